"""Every global name the host-side Python modules read is defined.

The benchmark modes and the server run only on a GPU machine; this catches
a name lost in an edit (a constant renamed, a helper removed) on the CPU."""
import builtins
import dis
import importlib
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _code_objects(co):
    yield co
    for c in co.co_consts:
        if isinstance(c, types.CodeType):
            yield from _code_objects(c)


def _global_reads(path):
    with open(path) as f:
        co = compile(f.read(), path, "exec")
    names = set()
    for c in _code_objects(co):
        for ins in dis.get_instructions(c):
            # LOAD_NAME outside module level reads a class body's namespace first
            if ins.opname == "LOAD_GLOBAL" or (ins.opname == "LOAD_NAME" and c is co):
                names.add(ins.argval)
    return names


@pytest.mark.parametrize("module", ["bench", "__graft_entry__", "paper_1605_00561_gb300.serving",
                                    "paper_1605_00561_gb300.dwt", "paper_1605_00561_gb300.build"])
def test_global_names_defined(module):
    mod = importlib.import_module(module)
    missing = sorted(n for n in _global_reads(mod.__file__)
                     if not hasattr(mod, n) and not hasattr(builtins, n) and n != "__file__")
    assert not missing, f"{module} reads undefined globals: {missing}"
