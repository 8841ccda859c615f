"""dwt2_forward_noalloc: the forward transform for callers that cannot
allocate device memory -- a real-time loop that must not call cudaMalloc
(which can synchronise the device and take unbounded time), or a plug-in
whose host application owns every device allocation.  Its LL scratch is a
fixed device array inside the library.  Checked through the C ABI against
dwt2_forward with a plan, twice in a row (the shared array keeps the
previous call's contents), and against the oracle on seeded random
configurations; the call's device memory use is checked too,
and a device wait that runs out is read back through
dwt_noalloc_device_status.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
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
    yield d
    d.dwt_debug_inject(d.DWT_INJECT_NONE)
    d.dwt_set_wait_limits(0, 0)


def _plan_forward(dwt, x, wavelet, levels, dtype):
    h, w = x.shape
    plan = dwt.Plan(w, h, wavelet, levels, dtype)
    out = torch.empty_like(x)
    plan.forward(x, out)
    torch.cuda.synchronize()
    plan.close()
    return out


def _noalloc(dwt, x, out, wl, levels, dt, stream=0):
    h, w = x.shape
    dwt.dwt2_forward_noalloc(w, h, wl, levels, dt, x.data_ptr(), x.stride(0) * x.element_size(),
                             out.data_ptr(), out.stride(0) * out.element_size(), stream)


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
        _noalloc(dwt, x, out, wl, levels, dt, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        if dtype == "i32":
            assert np.array_equal(got, ref), f"call {call}"
        else:
            assert np.abs(got.astype(np.float64) - ref).max() <= TOL_F32, f"call {call}"
    assert dwt.dwt_noalloc_device_status(0) == dwt.DWT_OK


def _random_cases():
    rng = np.random.default_rng(6061)
    out = []
    for i in range(40):
        h, w = (int(np.clip(np.round(np.exp(rng.uniform(0.0, np.log(1500.0)))), 1, 1500)) for _ in range(2))
        dtype = str(rng.choice(["f32", "f32", "f16s", "i32"]))
        wavelet = "cdf53" if dtype == "i32" else str(
            rng.choice(["cdf53", "cdf97", "dd137"] if dtype == "f32" else ["cdf53", "cdf97"]))
        levels = int(rng.integers(0, oracle.max_levels(w, h) + 1))
        pitch_pad = int(rng.choice([0, 0, 3, 16]))
        out.append((i, h, w, wavelet, dtype, levels, pitch_pad))
    return out


@pytest.mark.parametrize("case", _random_cases(), ids=lambda c: f"r{c[0]}")
def test_noalloc_random_against_oracle(dwt, case):
    """Seeded random sizes (1-1500 per side), level counts, wavelets and
    storage types, rows padded by 0, 3 or 16 elements, against the oracle:
    int32 bit for bit; float32 within 2e-3 (DD 13/7 included; the call
    runs Monolithic*); float16 storage within 1 + 0.3 L + 2e-3 of the
    largest coefficient (one float16 rounding of every band per level,
    amplified by the following levels' filters)."""
    i, h, w, wavelet, dtype, levels, pitch_pad = case
    what = f"h={h} w={w} {wavelet} {dtype} L={levels} pad={pitch_pad}"
    tdt = {"f32": torch.float32, "f16s": torch.float16, "i32": torch.int32}[dtype]
    if dtype == "i32":
        x = inputs.int12_image(h, w, seed=200 + i)
        ref = oracle.dwt2_int(x, levels)
    else:
        x = inputs.uniform_image(h, w, seed=200 + i)
        if dtype == "f16s":
            x = x.astype(np.float16).astype(np.float32)
        ref = oracle.dwt2(x.astype(np.float64), {"cdf53": oracle.CDF53, "cdf97": oracle.CDF97,
                                                 "dd137": oracle.DD137}[wavelet], levels)
    xb = torch.zeros(h, w + pitch_pad, dtype=tdt, device="cuda")
    xb[:, :w] = torch.from_numpy(x).to(tdt).cuda()
    ob = torch.full((h, w + pitch_pad), -7, dtype=tdt, device="cuda")
    xd, out = xb[:, :w], ob[:, :w]
    wl = {"cdf53": dwt.DWT_CDF53, "cdf97": dwt.DWT_CDF97, "dd137": dwt.DWT_DD137}[wavelet]
    dt = {"f32": dwt.DWT_F32, "f16s": dwt.DWT_F16S, "i32": dwt.DWT_I32}[dtype]
    _noalloc(dwt, xd, out, wl, levels, dt)
    assert dwt.dwt_noalloc_device_status(0) == dwt.DWT_OK, what
    got = out.cpu().numpy()
    if dtype == "i32":
        assert np.array_equal(got, ref), what
    else:
        err = float(np.abs(got.astype(np.float64) - ref).max(initial=0.0))
        tol = TOL_F32 if dtype == "f32" else 1.0 + 0.3 * levels + 2e-3 * float(np.abs(ref).max(initial=0.0))
        assert err <= tol, f"{what}: max|err| {err}"


def test_noalloc_call_takes_no_device_memory(dwt):
    """After a first call (which looks up the array and loads the kernels),
    a call leaves the device's free memory and torch's allocation as they
    were."""
    h, w, L = 1024, 768, 5
    x = torch.from_numpy(inputs.uniform_image(h, w, seed=5)).cuda()
    out = torch.empty_like(x)
    _noalloc(dwt, x, out, dwt.DWT_CDF97, L, dwt.DWT_F32)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    _noalloc(dwt, x, out, dwt.DWT_CDF97, L, dwt.DWT_F32)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0


def test_noalloc_wait_timeout_is_reported_then_clean(dwt):
    h, w, L = 300, 521, 4
    x = torch.from_numpy(inputs.uniform_image(h, w, seed=41)).cuda()
    ref = _plan_forward(dwt, x, "cdf97", L, "f32").cpu().numpy()
    out = torch.empty_like(x)
    dwt.dwt_set_wait_limits(0, 2000)
    dwt.dwt_debug_inject(dwt.DWT_INJECT_HOLD, 0, 1)  # the first level's launch waits on a flag nothing sets
    _noalloc(dwt, x, out, dwt.DWT_CDF97, L, dwt.DWT_F32)
    assert dwt.dwt_noalloc_device_status(0) == dwt.DWT_ETIMEOUT
    dwt.dwt_set_wait_limits(0, 0)
    _noalloc(dwt, x, out, dwt.DWT_CDF97, L, dwt.DWT_F32)
    assert dwt.dwt_noalloc_device_status(0) == dwt.DWT_OK
    assert np.abs(out.cpu().numpy().astype(np.float64) - ref).max() <= TOL_F32


def test_noalloc_rejects_images_beyond_its_scratch(dwt):
    n = 8192  # LL scratch 16 KiB x (4096 + 2048) rows = 96 MiB > 32 MiB
    x = torch.empty(n, n, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt2_forward_noalloc(n, n, dwt.DWT_CDF97, 6, dwt.DWT_F32, x.data_ptr(), n * 4, y.data_ptr(),
                                 n * 4, 0)
    assert e.value.status == dwt.DWT_EINVAL
