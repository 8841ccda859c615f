"""The reversible integer non-separable lifting (the Iwahashi scheme of CDF
5/3 with each 2-D step rounded once; an int32 plan with DWT_IWAHASHI)
against its exact-integer oracle, bit for bit, forward, inverse and round
trip, streamed and in the fused tail; and the guards that keep it from
replacing the JPEG 2000 transform (DWT_AUTO, the autotuner, batches)."""
import numpy as np
import pytest

import oracle
from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(150, 261, 3), (64, 64, 6), (1, 37, 3), (37, 1, 3), (2, 3, 2), (5, 130, 2), (131, 9, 4),
          (333, 500, 5)]


@pytest.fixture(scope="module")
def dwt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt as d
    d.lib()
    return d


def run(dwt, x, L, fusion=-1, coef_in=None):
    h, w = x.shape
    plan = dwt.Plan(w, h, "cdf53", L, "i32", scheme="iwahashi")
    dwt.dwt_plan_set_fusion(plan.handle, fusion)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", torch.int32)
    c = torch.empty_like(xd)
    y = torch.empty_like(xd)
    plan.forward(xd, c)
    plan.inverse(c, y)
    yo = None
    if coef_in is not None:
        yo = torch.empty_like(xd)
        plan.inverse(torch.from_numpy(coef_in.astype(np.int32)).cuda(), yo)
    torch.cuda.synchronize()
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    plan.close()
    return c.cpu().numpy(), y.cpu().numpy(), None if yo is None else yo.cpu().numpy()


@pytest.mark.parametrize("fusion", [-1, 0])
@pytest.mark.parametrize("h,w,L", SHAPES)
def test_int_iwahashi_bit_exact(dwt, h, w, L, fusion):
    x = inputs.int12_image(h, w, seed=h + 5 * w)
    ref = oracle.dwt2_int_iwahashi(x, L)
    c, y, yo = run(dwt, x, L, fusion, coef_in=ref)
    assert np.array_equal(c, ref), "forward"
    assert np.array_equal(yo, x), "inverse of oracle coefficients"
    assert np.array_equal(y, x), "round trip"


@pytest.mark.parametrize("h,w", [(4096, 4096), (3333, 5001)])
def test_int_iwahashi_config_sizes(dwt, h, w):
    x = inputs.int12_image(h, w, seed=7)
    ref = oracle.dwt2_int_iwahashi(x, 5)
    c, y, _ = run(dwt, x, 5)
    assert np.array_equal(c, ref)
    assert np.array_equal(y, x)


def test_int_iwahashi_guards(dwt, tmp_path, monkeypatch):
    monkeypatch.setenv("DWT_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    # DWT_AUTO and the autotuner keep an int32 plan on the JPEG 2000 transform
    p = dwt.Plan(300, 200, "cdf53", 3, "i32")
    assert p.scheme == "sweldens"
    dwt.dwt_plan_autotune(p.handle)
    assert p.scheme in ("sweldens", "rowcol")
    # an int32 plan set to the integer Iwahashi lifting keeps it when tuned
    q = dwt.Plan(300, 200, "cdf53", 3, "i32", scheme="iwahashi")
    dwt.dwt_plan_autotune(q.handle)
    assert q.scheme == "iwahashi"
    # batches run the JPEG 2000 transform for int32 and refuse the other one
    x = torch.from_numpy(inputs.int12_image(200, 300, seed=3)).cuda()
    c = torch.empty_like(x)
    with pytest.raises(dwt.DwtError) as e:
        dwt.submit([q.request(x, c)])
    assert e.value.status == dwt.DWT_EUNSUPPORTED
    dwt.submit([p.request(x, c)])
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), oracle.dwt2_int(x.cpu().numpy(), 3))
    p.close()
    q.close()
