"""Error paths on the GPU, made to happen without faulting or hanging it.

* A bounded device wait that runs out: the host injects a wait on something
  nothing provides (a batch row count one higher than its rows reach; a
  flag that nothing sets, taken before any load of the strip is issued),
  with a short wait limit.  The kernel raises its status word and returns;
  the status reaches the caller (batch status array, plan status query,
  no-alloc status query), and the next call on the same device is clean.
* Allocation failure: the host fakes cudaErrorMemoryAllocation at an
  allocation site of the library; the call returns DWT_ENOMEM, leaves no
  half-made state behind, and the next call succeeds.
"""
import numpy as np
import pytest

import oracle
from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_F32 = 2e-3
SHORT_SPINS = 2000  # polls of a few tens of ns each: a wait of well under a second


@pytest.fixture
def dwt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt as d
    d.lib()
    yield d
    d.dwt_debug_inject(d.DWT_INJECT_NONE)
    d.dwt_set_wait_limits(0, 0)


def _batch(dwt, shapes):
    plans, xs, outs, refs = [], [], [], []
    for h, w, wl, L in shapes:
        x = inputs.uniform_image(h, w, seed=h * 7 + w)
        plans.append(dwt.Plan(w, h, wl, L, "f32"))
        xs.append(torch.from_numpy(x).cuda())
        outs.append(torch.full_like(xs[-1], -3.0))
        refs.append(oracle.dwt2(x.astype(np.float64), {"cdf53": oracle.CDF53, "cdf97": oracle.CDF97}[wl], L))
    return plans, xs, outs, refs


def test_batch_row_wait_times_out_and_reports(dwt):
    shapes = [(300, 260, "cdf97", 3), (128, 200, "cdf53", 2), (97, 131, "cdf97", 2)]
    plans, xs, outs, refs = _batch(dwt, shapes)
    status = torch.full((len(shapes),), 77, dtype=torch.int32, device="cuda")
    dwt.dwt_set_wait_limits(0, SHORT_SPINS)
    dwt.dwt_debug_inject(dwt.DWT_INJECT_BATCH_DEP, 0, 1)
    dwt.submit([p.request(x, o) for p, x, o in zip(plans, xs, outs)], status=status)
    torch.cuda.synchronize()
    st = status.cpu().tolist()
    # request 0's second level waited for a row count nothing reaches
    assert st == [dwt.DWT_ETIMEOUT, dwt.DWT_OK, dwt.DWT_OK]
    for o, ref in zip(outs[1:], refs[1:]):
        assert np.abs(o.cpu().numpy() - ref).max() <= TOL_F32
    # the next batch on the same device is clean and correct, request 0 included
    dwt.dwt_set_wait_limits(0, 0)
    for o in outs:
        o.fill_(-3.0)
    dwt.submit([p.request(x, o) for p, x, o in zip(plans, xs, outs)], status=status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [dwt.DWT_OK] * 3
    for o, ref in zip(outs, refs):
        assert np.abs(o.cpu().numpy() - ref).max() <= TOL_F32
    for p in plans:
        p.close()


@pytest.mark.parametrize("fusion", [-1, 0])
@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_plan_wait_times_out_and_reports(dwt, dtype, fusion):
    """With the default fusion the whole pyramid is one fused-tail launch
    (the hold is CTA 0 of its first level); without it, one streaming launch
    per level (the hold is the second level's first strip)."""
    h, w, L = 257, 390, 3
    if dtype == "i32":
        x = inputs.int12_image(h, w, seed=3)
        ref = oracle.dwt2_int(x, L)
        plan = dwt.Plan(w, h, "cdf53", L, "i32")
    else:
        x = inputs.uniform_image(h, w, seed=3)
        ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, L)
        plan = dwt.Plan(w, h, "cdf97", L, "f32")
    dwt.dwt_plan_set_fusion(plan.handle, fusion)
    xd = torch.from_numpy(x).cuda()
    c = torch.empty_like(xd)
    plan.forward(xd, c)  # first call: the plan's allocations
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    dwt.dwt_set_wait_limits(0, SHORT_SPINS)
    dwt.dwt_debug_inject(dwt.DWT_INJECT_HOLD, 0 if fusion else 1, 1)
    plan.forward(xd, c)
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_ETIMEOUT
    # the query cleared the word; the next call is clean and correct
    dwt.dwt_set_wait_limits(0, 0)
    plan.forward(xd, c)
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    got = c.cpu().numpy()
    if dtype == "i32":
        assert np.array_equal(got, ref)
    else:
        assert np.abs(got - ref).max() <= TOL_F32
    plan.close()


def test_first_call_allocation_failure_then_recovery(dwt):
    h, w, L = 200, 333, 4
    x = inputs.uniform_image(h, w, seed=9)
    ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, L)
    xd = torch.from_numpy(x).cuda()
    c = torch.empty_like(xd)
    for skip in range(0, 4):  # status word, then each LL buffer
        plan = dwt.Plan(w, h, "cdf97", L, "f32")
        dwt.dwt_debug_inject(dwt.DWT_INJECT_ENOMEM, skip, 1)
        with pytest.raises(dwt.DwtError) as e:
            plan.forward(xd, c)
        assert e.value.status == dwt.DWT_ENOMEM
        dwt.dwt_debug_inject(dwt.DWT_INJECT_NONE)
        plan.forward(xd, c)
        torch.cuda.synchronize()
        assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
        assert np.abs(c.cpu().numpy() - ref).max() <= TOL_F32
        plan.close()


def test_host_call_staging_failure_leaves_no_half_state(dwt):
    """The host-buffer call allocates two staging planes; when the second
    fails, the first is freed and the next call allocates both again."""
    h, w, L = 120, 200, 3
    x = inputs.uniform_image(h, w, seed=21)
    ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, L)
    xh = torch.from_numpy(x).pin_memory()
    ch = torch.zeros_like(xh).pin_memory()
    plan = dwt.Plan(w, h, "cdf97", L, "f32")
    dwt.dwt_debug_inject(dwt.DWT_INJECT_ENOMEM, 1, 1)  # the input plane succeeds, the output plane fails
    with pytest.raises(dwt.DwtError) as e:
        plan.forward_host(xh, ch)
    assert e.value.status == dwt.DWT_ENOMEM
    dwt.dwt_debug_inject(dwt.DWT_INJECT_NONE)
    plan.forward_host(xh, ch)
    torch.cuda.synchronize()
    assert np.abs(ch.numpy() - ref).max() <= TOL_F32
    plan.close()


def test_batch_allocation_failure_then_recovery(dwt):
    shapes = [(300, 260, "cdf97", 3), (128, 200, "cdf53", 2)]
    plans, xs, outs, refs = _batch(dwt, shapes)
    status = torch.zeros(len(shapes), dtype=torch.int32, device="cuda")
    dwt.dwt_debug_inject(dwt.DWT_INJECT_ENOMEM, 0, 1)
    with pytest.raises(dwt.DwtError) as e:
        dwt.submit([p.request(x, o) for p, x, o in zip(plans, xs, outs)], status=status)
    assert e.value.status == dwt.DWT_ENOMEM
    dwt.submit([p.request(x, o) for p, x, o in zip(plans, xs, outs)], status=status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [dwt.DWT_OK] * 2
    for o, ref in zip(outs, refs):
        assert np.abs(o.cpu().numpy() - ref).max() <= TOL_F32
    for p in plans:
        p.close()
