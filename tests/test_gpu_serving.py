"""GPU tests of the continuous-batching server: every request's result is
the same whether it ran alone or mixed with others (bit for bit), when
memory pressure makes requests wait, and with one launch per request."""
import numpy as np
import pytest

import oracle
from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt, serving
    dwt.lib()
    return dwt, serving


def small_trace(n, seed):
    """Poisson-shaped requests scaled down (areas 64^2..512^2)."""
    tr = inputs.serving_trace(rate=4000.0, seconds=n / 4000.0 * 1.5, seed=seed, median_area=128 * 128,
                              lo=16, hi=512)
    return tr[:n]


@pytest.fixture(scope="module")
def pools(mods):
    f = torch.from_numpy(inputs.uniform_image(512, 512, seed=21)).cuda()
    i = torch.from_numpy(inputs.int12_image(512, 512, seed=22)).cuda()
    return f, i


def make_requests(serving, trace, pools, inverse_every=0):
    f, i = pools
    reqs = []
    for k, t in enumerate(trace):
        kind = t["kind"]
        dtype = "f32" if kind == "cdf97" else "i32"
        wl = "cdf97" if kind == "cdf97" else "cdf53"
        src = (f if dtype == "f32" else i)[: t["h"], : t["w"]]
        levels = min(t["levels"], oracle.max_levels(t["w"], t["h"]))
        inv = bool(inverse_every) and k % inverse_every == 0
        reqs.append(serving.Request(t["w"], t["h"], levels, wl, dtype, inv, src, tag=k))
    return reqs, [t["t"] for t in trace]


def alone(dwt, r):
    out = torch.empty((r.h, r.w), dtype=r.out.dtype, device="cuda")
    p = dwt.Plan(r.w, r.h, r.wavelet, r.levels, r.dtype)
    dwt.submit([p.request(r.src, out, r.inverse)])
    torch.cuda.synchronize()
    p.close()
    return out


def test_served_results_equal_alone(mods, pools):
    dwt, serving = mods
    reqs, offs = make_requests(serving, small_trace(300, seed=31), pools, inverse_every=5)
    srv = serving.Server(max_inflight=3)
    res = serving.replay(srv, reqs, offs)
    torch.cuda.synchronize()
    s = res.summary()
    assert s["requests"] == 300 and s["failed"] == 0
    assert res.batches < 300  # requests were grouped
    for r in reqs:
        assert torch.equal(r.out, alone(dwt, r)), r.tag
    # the oracle on a sample (forward requests)
    for r in reqs[1::41]:
        if r.inverse:
            continue
        x = r.src.cpu().numpy()
        if r.dtype == "i32":
            assert np.array_equal(r.out.cpu().numpy(), oracle.dwt2_int(x.astype(np.int64), r.levels))
        else:
            ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, r.levels)
            assert np.abs(r.out.cpu().numpy() - ref).max() <= 2e-3
    srv.close()


def test_memory_pressure_makes_requests_wait(mods, pools):
    dwt, serving = mods
    reqs, offs = make_requests(serving, small_trace(120, seed=32), pools)
    biggest = max(serving.request_bytes(r) for r in reqs)
    srv = serving.Server(budget_bytes=2 * biggest, max_inflight=4)
    peak = [0]
    orig = srv._launch

    def spy(take, cost):
        orig(take, cost)
        peak[0] = max(peak[0], srv.in_use)

    srv._launch = spy
    res = serving.replay(srv, reqs, [0.0] * len(reqs))
    assert res.summary()["failed"] == 0
    assert peak[0] <= srv.budget
    assert srv.in_use == 0
    for r in reqs[::7]:
        assert torch.equal(r.out, alone(dwt, r))
    srv.close()


def test_one_launch_per_request_mode(mods, pools):
    dwt, serving = mods
    reqs, offs = make_requests(serving, small_trace(60, seed=33), pools)
    srv = serving.Server(per_request=True)
    res = serving.replay(srv, reqs, offs)
    assert res.batches == 60 and res.summary()["failed"] == 0
    for r in reqs[::5]:
        assert torch.equal(r.out, alone(dwt, r))
    srv.close()
