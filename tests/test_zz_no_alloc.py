"""dwt2_forward_noalloc, the forward transform for callers that cannot
allocate device memory (graph capture, real-time loops, hosts that own all
allocations): its LL scratch is a fixed device array inside the library.
Checked through the C ABI against dwt2_forward with a plan, twice in a row
(the shared array keeps the previous call's contents).  This file is
collected last on purpose."""
import numpy as np
import pytest

from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_F32 = 2e-3


@pytest.fixture(scope="module")
def dwt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt as d
    d.lib()
    return d


def _plan_forward(dwt, x, wavelet, levels, dtype):
    h, w = x.shape
    plan = dwt.Plan(w, h, wavelet, levels, dtype)
    out = torch.empty_like(x)
    plan.forward(x, out)
    torch.cuda.synchronize()
    plan.close()
    return out


@pytest.mark.parametrize("wavelet,dtype,h,w,levels", [
    ("cdf97", "f32", 300, 521, 4),
    ("cdf53", "f32", 64, 64, 6),
    ("cdf53", "i32", 333, 500, 5),
])
def test_noalloc_matches_plan_forward_twice(dwt, wavelet, dtype, h, w, levels):
    wl = {"cdf53": dwt.DWT_CDF53, "cdf97": dwt.DWT_CDF97}[wavelet]
    dt = {"f32": dwt.DWT_F32, "i32": dwt.DWT_I32}[dtype]
    for call, seed in enumerate((31, 32)):
        if dtype == "i32":
            x = torch.from_numpy(inputs.int12_image(h, w, seed=seed)).cuda()
        else:
            x = torch.from_numpy(inputs.uniform_image(h, w, seed=seed)).cuda()
        ref = _plan_forward(dwt, x, wavelet, levels, dtype).cpu().numpy()
        out = torch.full_like(x, -7)
        dwt.dwt2_forward_noalloc(w, h, wl, levels, dt, x.data_ptr(), x.stride(0) * x.element_size(),
                                 out.data_ptr(), out.stride(0) * out.element_size(),
                                 torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        if dtype == "i32":
            assert np.array_equal(got, ref), f"call {call}"
        else:
            assert np.abs(got.astype(np.float64) - ref).max() <= TOL_F32, f"call {call}"


def test_noalloc_rejects_images_beyond_its_scratch(dwt):
    n = 8192  # LL scratch 16 KiB x (4096 + 2048) rows = 96 MiB > 32 MiB
    x = torch.empty(n, n, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt2_forward_noalloc(n, n, dwt.DWT_CDF97, 6, dwt.DWT_F32, x.data_ptr(), n * 4, y.data_ptr(),
                                 n * 4, 0)
    assert e.value.status == dwt.DWT_EINVAL
