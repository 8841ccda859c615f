"""The bench's all-cores oracle baseline (CPU only): one spawned process per
core, each running the unchanged single-threaded oracle on its own image,
all starting together; the figure is every process's pixels over the
slowest one's duration."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_all_cores_baseline_runs_one_oracle_per_core():
    a = types.SimpleNamespace(wavelet="cdf97", levels=3)
    r = bench.cpu_baseline_all_cores(a, n=64)
    assert r is not None
    value, slowest, procs = r
    assert procs == (os.cpu_count() or 1)
    assert slowest > 0 and value > 0
    assert abs(value - 2.0 * 64 * 64 * procs / slowest / 1e9) < 1e-12
