"""The fused tail: the small levels of a single-image call in one launch,
each level in 2-D shared-memory tiles (tile_kernel.cuh).

Each coefficient goes through the same steps in the same arithmetic order
in the tile kernel as in the streaming per-level kernels, so a fused call
must equal the unfused call of the same plan bit for bit, and both must
match the oracle.  Covered: every scheme that has a tile program, the
three wavelets, forward and inverse, float32, float16 storage and int32,
the paper's zeta scaling, odd sizes and a pyramid whose last levels have a
side of length 1 (those levels leave the tail)."""
import numpy as np
import pytest

import oracle
from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_F32 = 2e-3
OID = {"cdf53": oracle.CDF53, "cdf97": oracle.CDF97, "dd137": oracle.DD137}
TILE_SCHEMES = ["sweldens", "iwahashi", "iwahashi*", "explosive", "explosive*", "monolithic", "monolithic*",
                "polyphase", "polyphase*"]
DD_TILE = TILE_SCHEMES


@pytest.fixture(scope="module")
def dwt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt as d
    d.lib()
    return d


def same(a, b, what):
    if not torch.equal(a, b):
        d = float((a.double() - b.double()).abs().max())
        n = int((a != b).sum())
        raise AssertionError(f"{what}: fused and unfused differ at {n} values, max |diff| {d:.3e}")


def fwd_inv(dwt, x, wavelet, levels, dtype, scheme, fusion, zeta=False):
    h, w = x.shape
    plan = dwt.Plan(w, h, wavelet, levels, dtype, scheme=scheme)
    dwt.dwt_plan_set_fusion(plan.handle, fusion)
    if zeta:
        dwt.dwt_plan_set_normalization(plan.handle, dwt.DWT_NORM_ZETA)
    tdt = {"f32": torch.float32, "f16s": torch.float16, "i32": torch.int32}[dtype]
    xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", tdt)
    c = torch.empty_like(xd)
    y = torch.empty_like(xd)
    plan.forward(xd, c)
    plan.inverse(c, y)
    torch.cuda.synchronize()
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    plan.close()
    return c, y


@pytest.mark.parametrize("scheme", TILE_SCHEMES)
@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("h,w,L", [(1024, 1024, 6), (333, 517, 5), (70, 41, 7)])
def test_fused_equals_unfused_and_oracle(dwt, scheme, wavelet, h, w, L):
    x = inputs.uniform_image(h, w, seed=h + 3 * w)
    cf, yf = fwd_inv(dwt, x, wavelet, L, "f32", scheme, -1)
    cu, yu = fwd_inv(dwt, x, wavelet, L, "f32", scheme, 0)
    same(cf, cu, "forward")
    same(yf, yu, "inverse")
    ref = oracle.dwt2(x.astype(np.float64), OID[wavelet], L)
    assert np.abs(cf.cpu().numpy() - ref).max() <= TOL_F32
    assert float((yf - torch.from_numpy(x).cuda()).abs().max()) <= 2 * TOL_F32


@pytest.mark.parametrize("scheme", DD_TILE)
def test_fused_dd137(dwt, scheme):
    h, w, L = 601, 480, 5
    x = inputs.uniform_image(h, w, seed=9)
    cf, yf = fwd_inv(dwt, x, "dd137", L, "f32", scheme, -1)
    cu, yu = fwd_inv(dwt, x, "dd137", L, "f32", scheme, 0)
    same(cf, cu, "forward")
    same(yf, yu, "inverse")
    ref = oracle.dwt2(x.astype(np.float64), oracle.DD137, L)
    assert np.abs(cf.cpu().numpy() - ref).max() <= TOL_F32


@pytest.mark.parametrize("h,w,L", [(4096, 4096, 5), (3333, 5001, 5), (257, 390, 8), (2, 3, 2)])
def test_fused_int53_bit_exact(dwt, h, w, L):
    x = inputs.int12_image(h, w, seed=7 + h)
    cf, yf = fwd_inv(dwt, x, "cdf53", L, "i32", "sweldens", -1)
    ref = oracle.dwt2_int(x, L)
    assert np.array_equal(cf.cpu().numpy(), ref)
    assert torch.equal(yf, torch.from_numpy(x).cuda())


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_fused_float16_storage_and_zeta(dwt, wavelet):
    h, w, L = 700, 900, 6
    x = inputs.uniform_image(h, w, seed=11)
    cf, yf = fwd_inv(dwt, x, wavelet, L, "f16s", "monolithic*", -1)
    cu, yu = fwd_inv(dwt, x, wavelet, L, "f16s", "monolithic*", 0)
    same(cf, cu, "forward")
    same(yf, yu, "inverse")
    zf, zy = fwd_inv(dwt, x, wavelet, L, "f32", "monolithic*", -1, zeta=True)
    zu, _ = fwd_inv(dwt, x, wavelet, L, "f32", "monolithic*", 0, zeta=True)
    same(zf, zu, "forward, zeta")
    ref = oracle.dwt2(x.astype(np.float64), OID[wavelet], L, norm=oracle.NORM_ZETA)
    assert np.abs(zf.cpu().numpy() - ref).max() <= TOL_F32 + 2e-5 * float(np.abs(ref).max())


def test_fusion_threshold_and_profile(dwt):
    """The default threshold fuses every level whose input has at most
    512 x 512 samples: an 8192^2 six-level plan runs L0-L3 one launch each
    and L4-L5 in one launch; a larger threshold fuses more; 0 turns the
    fusion off."""
    n, L = 8192, 6
    plan = dwt.Plan(n, n, "cdf97", L, "f32", scheme="monolithic*")
    assert dwt.dwt_plan_get_fusion(plan.handle) == 512 * 512
    x = torch.rand(n, n, device="cuda")
    c = torch.empty_like(x)
    y = torch.empty_like(x)
    dwt.dwt_plan_set_profiling(plan.handle, True)
    plan.forward(x, c)
    plan.inverse(c, y)
    names = [p["name"] for p in dwt.dwt_plan_read_profile(plan.handle)]
    assert names == ["fwd/L0", "fwd/L1", "fwd/L2", "fwd/L3", "fwd/L4-5", "inv/L4-5", "inv/L3", "inv/L2",
                     "inv/L1", "inv/L0"]
    dwt.dwt_plan_set_fusion(plan.handle, 2048 * 2048)
    plan.forward(x, c)
    plan.inverse(c, y)
    names = [p["name"] for p in dwt.dwt_plan_read_profile(plan.handle)]
    assert names == ["fwd/L0", "fwd/L1", "fwd/L2-5", "inv/L2-5", "inv/L1", "inv/L0"]
    dwt.dwt_plan_set_fusion(plan.handle, 0)
    plan.forward(x, c)
    names = [p["name"] for p in dwt.dwt_plan_read_profile(plan.handle)]
    assert names == [f"fwd/L{k}" for k in range(L)]
    with pytest.raises(dwt.DwtError):
        dwt.dwt_plan_set_fusion(plan.handle, -2)
    plan.close()
