"""GPU parity: the CUDA path through the C ABI against the FP64 / exact-int
oracle, element by element, for every scheme, wavelet and direction, at
sizes spanning several warp strips with ragged tails, plus edge cases.

Tolerances: float32 max |err| <= 2e-3 against FP64 on 8-bit-range inputs
(up to 6 levels); reversible integer 5/3 bit-exact; float16 storage has no
precision bar (its error is printed and sanity-bounded)."""
import numpy as np
import pytest

import oracle
from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_F32 = 2e-3
# a GPU forward followed by a GPU inverse composes two FP32 transforms, each
# within TOL_F32 of the exact result
TOL_ROUND_TRIP = 2 * TOL_F32
FLOAT_SCHEMES = ["rowcol", "sweldens", "iwahashi", "iwahashi*", "explosive", "explosive*",
                 "monolithic", "monolithic*", "polyphase", "polyphase*", "convolution"]
OID = {"cdf53": oracle.CDF53, "cdf97": oracle.CDF97}
SHAPES = [(150, 261, 3), (64, 64, 6), (1, 37, 3), (37, 1, 3), (2, 3, 2), (5, 130, 2), (131, 9, 4)]


@pytest.fixture(scope="module")
def dwt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt as d
    d.lib()
    return d


def run_fwd_inv(dwt, x, wavelet, levels, dtype, scheme, coef_in=None):
    h, w = x.shape
    plan = dwt.Plan(w, h, wavelet, levels, dtype, scheme=scheme)
    tdt = {"f32": torch.float32, "f16s": torch.float16, "i32": torch.int32}[dtype]
    xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", tdt)
    c = torch.empty_like(xd)
    y = torch.empty_like(xd)
    plan.forward(xd, c)
    plan.inverse(c, y)
    yo = None
    if coef_in is not None:
        cd = torch.from_numpy(np.ascontiguousarray(coef_in)).to("cuda", tdt)
        yo = torch.empty_like(xd)
        plan.inverse(cd, yo)
        yo = yo.cpu().numpy()
    torch.cuda.synchronize()
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    plan.close()
    return c.cpu().numpy(), y.cpu().numpy(), yo


@pytest.mark.parametrize("scheme", FLOAT_SCHEMES)
@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("h,w,L", SHAPES)
def test_float32_forward_inverse_vs_oracle(dwt, scheme, wavelet, h, w, L):
    x = inputs.uniform_image(h, w, seed=h * 1000 + w)
    ref = oracle.dwt2(x.astype(np.float64), OID[wavelet], L)
    c, y, yo = run_fwd_inv(dwt, x, wavelet, L, "f32", scheme, coef_in=ref.astype(np.float32))
    assert np.abs(c - ref).max() <= TOL_F32, "forward"
    assert np.abs(yo - x).max() <= TOL_F32, "inverse of oracle coefficients"
    assert np.abs(y - x).max() <= TOL_ROUND_TRIP, "round trip"


# DD 13/7 (degree-3 predict and update, Sec. 5): every scheme, Polyphase(*)
# and Convolution with the degree-6 products of P and U
DD_SCHEMES = FLOAT_SCHEMES


@pytest.mark.parametrize("scheme", DD_SCHEMES)
@pytest.mark.parametrize("h,w,L", SHAPES)
def test_dd137_forward_inverse_vs_oracle(dwt, scheme, h, w, L):
    x = inputs.uniform_image(h, w, seed=h * 31 + w)
    ref = oracle.dwt2(x.astype(np.float64), oracle.DD137, L)
    c, y, yo = run_fwd_inv(dwt, x, "dd137", L, "f32", scheme, coef_in=ref.astype(np.float32))
    assert np.abs(c - ref).max() <= TOL_F32, "forward"
    assert np.abs(yo - x).max() <= TOL_F32, "inverse of oracle coefficients"
    assert np.abs(y - x).max() <= TOL_ROUND_TRIP, "round trip"


def zeta_tol(ref):
    # the paper's scaling grows LL by 2 per level (zeta^2 = 2): FP32 error
    # scales with the magnitudes, so the bar is relative to the largest
    return TOL_F32 + 2e-5 * float(np.abs(ref).max())


@pytest.mark.parametrize("scheme", FLOAT_SCHEMES)
@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("h,w,L", [(150, 261, 3), (131, 9, 4), (64, 64, 6)])
def test_zeta_normalisation_vs_oracle(dwt, scheme, wavelet, h, w, L):
    """The paper's scaling step (DWT_NORM_ZETA: low-pass x zeta, high-pass
    x 1/zeta per axis) against the oracle's, forward and inverse."""
    x = inputs.uniform_image(h, w, seed=h * 31 + w + L)
    ref = oracle.dwt2(x.astype(np.float64), OID[wavelet], L, norm=oracle.NORM_ZETA)
    plan = dwt.Plan(w, h, wavelet, L, "f32", scheme=scheme)
    dwt.dwt_plan_set_normalization(plan.handle, dwt.DWT_NORM_ZETA)
    xd = torch.from_numpy(x).cuda()
    c = torch.empty_like(xd)
    y = torch.empty_like(xd)
    plan.forward(xd, c)
    plan.inverse(c, y)
    torch.cuda.synchronize()
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    plan.close()
    assert np.abs(c.cpu().numpy() - ref).max() <= zeta_tol(ref)
    assert np.abs(y.cpu().numpy() - x).max() <= 2 * TOL_F32


def test_zeta_normalisation_in_a_batch(dwt):
    """Batched requests of plans with the paper's scaling take the batch
    kernel's runtime-coefficient kinds; each result matches the oracle."""
    shapes = [(301, 257, "cdf97", 3), (128, 96, "cdf53", 2), (77, 130, "cdf97", 1)]
    plans, xs, cs, refs = [], [], [], []
    for h, w, wl, L in shapes:
        x = inputs.uniform_image(h, w, seed=h + w)
        p = dwt.Plan(w, h, wl, L, "f32")
        dwt.dwt_plan_set_normalization(p.handle, dwt.DWT_NORM_ZETA)
        plans.append(p)
        xs.append(torch.from_numpy(x).cuda())
        cs.append(torch.empty_like(xs[-1]))
        refs.append(oracle.dwt2(x.astype(np.float64), OID[wl], L, norm=oracle.NORM_ZETA))
    status = torch.zeros(len(shapes), dtype=torch.int32, device="cuda")
    dwt.submit([p.request(x, c) for p, x, c in zip(plans, xs, cs)], status=status)
    torch.cuda.synchronize()
    assert int(status.abs().sum()) == 0
    for c, ref in zip(cs, refs):
        assert np.abs(c.cpu().numpy() - ref).max() <= zeta_tol(ref)
    for p in plans:
        p.close()


def test_dd137_every_scheme_and_batches(dwt):
    p = dwt.dwt_plan_create(64, 64, dwt.DWT_DD137, 2, dwt.DWT_F32)
    for name in FLOAT_SCHEMES:
        dwt.dwt_plan_set_scheme(p, dwt.SCHEMES[name])
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt_plan_create(64, 64, dwt.DWT_DD137, 2, dwt.DWT_F16S)
    assert e.value.status == dwt.DWT_EUNSUPPORTED
    # batches run DD 13/7 plans with their Monolithic* kind
    xh = inputs.uniform_image(64, 64, seed=5)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    req = dwt.DwtRequest(p, x.data_ptr(), 256, y.data_ptr(), 256, 0)
    dwt.dwt_batch_submit([req])
    torch.cuda.synchronize()
    ref = oracle.dwt2(xh.astype(np.float64), oracle.DD137, 2)
    assert np.abs(y.cpu().numpy() - ref).max() <= TOL_F32
    dwt.dwt_plan_destroy(p)


@pytest.mark.parametrize("scheme", ["rowcol", "sweldens"])
@pytest.mark.parametrize("h,w,L", SHAPES + [(333, 500, 5)])
def test_int32_bit_exact(dwt, scheme, h, w, L):
    x = inputs.int12_image(h, w, seed=h + 7 * w)
    ref = oracle.dwt2_int(x, L)
    c, y, yo = run_fwd_inv(dwt, x, "cdf53", L, "i32", scheme, coef_in=ref.astype(np.int32))
    assert np.array_equal(c, ref), "forward"
    assert np.array_equal(yo, x), "inverse of oracle coefficients"
    assert np.array_equal(y, x), "round trip"


@pytest.mark.parametrize("scheme", FLOAT_SCHEMES)
@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_float16_storage_error_reported(dwt, scheme, wavelet):
    h, w, L = 150, 261, 3
    x = inputs.uniform_image(h, w, seed=5)
    ref = oracle.dwt2(x.astype(np.float64), OID[wavelet], L)
    c, y, _ = run_fwd_inv(dwt, x, wavelet, L, "f16s", scheme)
    ef = float(np.abs(c.astype(np.float64) - ref).max())
    er = float(np.abs(y.astype(np.float64) - x).max())
    print(f"f16s {wavelet} {scheme}: forward max|err| {ef:.3f}, round trip {er:.3f}")
    assert ef < 2.0 and er < 2.0  # sanity bound, not a precision claim


def test_textured_8192_cdf97_six_levels_full_compare(dwt):
    n, L = 8192, 6
    x = inputs.textured_image(n, n, seed=2)
    ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, L)
    c, y, _ = run_fwd_inv(dwt, x, "cdf97", L, "f32", "monolithic*")
    assert np.abs(c - ref).max() <= TOL_F32
    assert np.abs(y - x).max() <= TOL_ROUND_TRIP


@pytest.mark.parametrize("scheme,wavelet", [("iwahashi*", "cdf97"), ("explosive", "cdf97"),
                                            ("polyphase", "cdf97"), ("convolution", "cdf97"),
                                            ("monolithic*", "dd137")])
def test_tall_strip_schemes_8192_full_compare(dwt, scheme, wavelet):
    """Schemes whose default strips are 24-48 rows tall: at 8192^2 their
    strip rows are dealt over several resident waves (the dispatch order of
    tall strips), which small images never reach.  Every coefficient and
    every reconstructed sample is compared."""
    n, L = 8192, 1
    x = inputs.textured_image(n, n, seed=3)
    ref = oracle.dwt2(x.astype(np.float64), {"cdf97": oracle.CDF97, "dd137": oracle.DD137}[wavelet], L)
    c, y, _ = run_fwd_inv(dwt, x, wavelet, L, "f32", scheme)
    assert np.abs(c - ref).max() <= TOL_F32
    assert np.abs(y - x).max() <= TOL_ROUND_TRIP


@pytest.mark.parametrize("scheme", ["monolithic*", "iwahashi*", "convolution"])
@pytest.mark.parametrize("h,w,L", [(131072, 3, 3), (3, 131072, 3), (70001, 1, 4), (1, 70001, 4)])
def test_extreme_aspect_ratios(dwt, scheme, h, w, L):
    """Lines and near-lines: one column of strips with thousands of rows of
    strips (for the 32-row Iwahashi* strips more than a wave, so their rows
    are dealt), one row of strips with thousands of columns, and length-1
    axes."""
    x = inputs.uniform_image(h, w, seed=h + w + L)
    ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, L)
    c, y, _ = run_fwd_inv(dwt, x, "cdf97", L, "f32", scheme)
    assert np.abs(c - ref).max() <= TOL_F32
    assert np.abs(y - x).max() <= TOL_ROUND_TRIP


@pytest.mark.parametrize("h,w", [(131072, 3), (3, 131072), (70001, 1)])
def test_int53_extreme_aspect_ratios_bit_exact(dwt, h, w):
    x = inputs.int12_image(h, w, seed=11)
    ref = oracle.dwt2_int(x, 3)
    c, y, _ = run_fwd_inv(dwt, x, "cdf53", 3, "i32", "sweldens")
    assert np.array_equal(c, ref)
    assert np.array_equal(y, x)


@pytest.mark.parametrize("h,w", [(4096, 4096), (3333, 5001)])
def test_int53_config_sizes_bit_exact(dwt, h, w):
    x = inputs.int12_image(h, w, seed=7)
    ref = oracle.dwt2_int(x, 5)
    c, y, _ = run_fwd_inv(dwt, x, "cdf53", 5, "i32", "sweldens")
    assert np.array_equal(c, ref)
    assert np.array_equal(y, x)


# ---------------------------------------------------------------------------
# layouts and edge cases
# ---------------------------------------------------------------------------

def test_pitched_and_unaligned_buffers_with_canaries(dwt):
    """Unaligned pitch and base (cp.async path instead of TMA); guard bands
    around the output must stay untouched."""
    h, w, L = 97, 203, 3
    x = inputs.uniform_image(h, w, seed=3)
    ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, L)
    big_in = torch.full((h + 4, w + 7), -1.0, device="cuda")
    big_in[2:2 + h, 3:3 + w] = torch.from_numpy(x).cuda()
    xin = big_in[2:2 + h, 3:3 + w]
    big_out = torch.full((h + 4, w + 7), 12345.0, device="cuda")
    cout = big_out[2:2 + h, 3:3 + w]
    plan = dwt.Plan(w, h, "cdf97", L, "f32", scheme="monolithic*")
    plan.forward(xin, cout)
    torch.cuda.synchronize()
    got = big_out.cpu().numpy()
    assert np.abs(got[2:2 + h, 3:3 + w] - ref).max() <= TOL_F32
    mask = np.ones_like(got, dtype=bool)
    mask[2:2 + h, 3:3 + w] = False
    assert np.all(got[mask] == 12345.0)
    plan.close()


def test_levels_zero_is_copy(dwt):
    x = inputs.uniform_image(33, 17, seed=4)
    c, y, _ = run_fwd_inv(dwt, x, "cdf97", 0, "f32", None)
    assert np.array_equal(c, x) and np.array_equal(y, x)


def test_invalid_calls_return_status(dwt):
    plan = dwt.Plan(64, 64, "cdf97", 2, "f32")
    a = torch.zeros(64, 64, device="cuda")
    b = torch.zeros(64, 64, device="cuda")
    host = torch.zeros(64, 64)
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt2_forward(plan.handle, host.data_ptr(), 256, b.data_ptr(), 256)
    assert e.value.status == dwt.DWT_EINVAL
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt2_forward(plan.handle, a.data_ptr(), 128, b.data_ptr(), 256)  # pitch < row
    assert e.value.status == dwt.DWT_EINVAL
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt2_forward(plan.handle, a.data_ptr(), 256, a.data_ptr(), 256)  # aliasing
    assert e.value.status == dwt.DWT_EINVAL
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt_plan_set_scheme(plan.handle, 99)
    assert e.value.status == dwt.DWT_EINVAL
    plan.close()
    pi = dwt.dwt_plan_create(8, 8, dwt.DWT_CDF53, 1, dwt.DWT_I32)
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt_plan_set_scheme(pi, dwt.SCHEMES["monolithic"])
    assert e.value.status == dwt.DWT_EUNSUPPORTED
    dwt.dwt_plan_destroy(pi)


def test_two_streams_same_result_as_alone(dwt):
    h, w, L = 300, 410, 4
    xs = [inputs.uniform_image(h, w, seed=s) for s in (11, 12)]
    alone = [run_fwd_inv(dwt, x, "cdf97", L, "f32", "monolithic*")[0] for x in xs]
    plans = [dwt.Plan(w, h, "cdf97", L, "f32", scheme="monolithic*") for _ in xs]
    streams = [torch.cuda.Stream() for _ in xs]
    outs = []
    for p, s, x in zip(plans, streams, xs):
        xd = torch.from_numpy(x).cuda()
        c = torch.empty_like(xd)
        torch.cuda.synchronize()
        p.forward(xd, c, stream=s.cuda_stream)
        outs.append(c)
    torch.cuda.synchronize()
    for a, o in zip(alone, outs):
        assert np.array_equal(a, o.cpu().numpy())
    for p in plans:
        p.close()


def test_host_buffer_entry_points(dwt):
    h, w, L = 120, 200, 3
    x = inputs.uniform_image(h, w, seed=21)
    ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, L)
    plan = dwt.Plan(w, h, "cdf97", L, "f32", scheme="monolithic*")
    xh = torch.from_numpy(x).pin_memory()
    ch = torch.empty_like(xh).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    plan.forward_host(xh, ch)
    plan.inverse_host(ch, yh)
    torch.cuda.synchronize()
    assert np.abs(ch.numpy() - ref).max() <= TOL_F32
    assert np.abs(yh.numpy() - x).max() <= TOL_ROUND_TRIP
    plan.close()


def test_profiling_reports_every_level(dwt):
    h, w, L = 256, 256, 3
    plan = dwt.Plan(w, h, "cdf97", L, "f32", scheme="monolithic*")
    dwt.dwt_plan_set_fusion(plan.handle, 0)  # one launch per level
    dwt.dwt_plan_set_profiling(plan.handle, True)
    x = torch.rand(h, w, device="cuda")
    c = torch.empty_like(x)
    plan.forward(x, c)
    prof = dwt.dwt_plan_read_profile(plan.handle)
    names = [p["name"] for p in prof]
    assert names == ["fwd/L0", "fwd/L1", "fwd/L2"]
    assert prof[0]["algorithmic_bytes"] == 2 * 256 * 256 * 4
    assert all(p["total_ms"] > 0 for p in prof)
    plan.close()


def test_autotune_scheme_and_tile_cached(dwt, tmp_path, monkeypatch):
    monkeypatch.setenv("DWT_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    h, w, L = 700, 1000, 3
    p = dwt.Plan(w, h, "cdf97", L, "f32")
    dwt.dwt_plan_autotune(p.handle)
    scheme = p.scheme
    rows, stages = dwt.dwt_plan_get_tile(p.handle)
    assert scheme in FLOAT_SCHEMES
    assert rows in (6, 8, 10, 12, 16, 24, 32, 48) and 1 <= stages <= 4
    # the tuned plan still computes the transform
    x = inputs.uniform_image(h, w, seed=77)
    ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, L)
    xd = torch.from_numpy(x).cuda()
    c = torch.empty_like(xd)
    p.forward(xd, c)
    torch.cuda.synchronize()
    assert np.abs(c.cpu().numpy() - ref).max() <= TOL_F32
    # a new plan of the same shape takes the cached choice
    q = dwt.Plan(w, h, "cdf97", L, "f32")
    assert q.scheme == scheme and dwt.dwt_plan_get_tile(q.handle) == (rows, stages)
    # a tile set by the caller wins over the cache
    r = dwt.Plan(w, h, "cdf97", L, "f32")
    dwt.dwt_plan_set_tile(r.handle, 8, 3)
    assert dwt.dwt_plan_get_tile(r.handle) == (8, 3)
    for plan in (p, q, r):
        plan.close()


def test_default_strip_rows_follow_the_scheme(dwt, tmp_path, monkeypatch):
    """Without a tile from the caller or the autotuner, each scheme takes its
    own default strip height; dwt_plan_set_tile(0, 0) returns to it."""
    monkeypatch.setenv("DWT_AUTOTUNE_CACHE", str(tmp_path / "empty.txt"))
    cases = [("monolithic*", "cdf97", 10), ("sweldens", "dd137", 10), ("iwahashi", "cdf53", 10),
             ("iwahashi*", "cdf97", 32), ("explosive", "dd137", 32), ("monolithic*", "dd137", 24),
             ("polyphase", "cdf53", 32), ("convolution", "cdf97", 48), ("convolution", "cdf53", 32)]
    for scheme, wavelet, rows in cases:
        p = dwt.Plan(512, 384, wavelet, 2, "f32", scheme=scheme)
        assert dwt.dwt_plan_get_tile(p.handle) == (rows, 2), (scheme, wavelet)
        dwt.dwt_plan_set_tile(p.handle, 6, 3)
        assert dwt.dwt_plan_get_tile(p.handle) == (6, 3)
        dwt.dwt_plan_set_tile(p.handle, 0, 0)
        assert dwt.dwt_plan_get_tile(p.handle) == (rows, 2)
        p.close()


def test_plan_calls_replay_from_a_cuda_graph(dwt):
    """After one eager call (which makes the plan's allocations), forward and
    inverse calls can be captured into a CUDA graph and replayed on new
    inputs with the eager results."""
    h, w, L = 523, 611, 4
    plan = dwt.Plan(w, h, "cdf97", L, "f32", scheme="monolithic*")
    x = torch.zeros((h, w), device="cuda")
    c = torch.empty_like(x)
    y = torch.empty_like(x)
    plan.forward(x, c)
    plan.inverse(c, y)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.forward(x, c, stream=s.cuda_stream)
            plan.inverse(c, y, stream=s.cuda_stream)
    for seed in (3, 4):
        x.copy_(torch.from_numpy(inputs.uniform_image(h, w, seed=seed)))
        g.replay()
        torch.cuda.synchronize()
        ce, ye = torch.empty_like(x), torch.empty_like(x)
        plan.forward(x, ce)
        plan.inverse(ce, ye)
        torch.cuda.synchronize()
        assert torch.equal(c, ce) and torch.equal(y, ye)
        ref = oracle.dwt2(x.cpu().numpy().astype(np.float64), oracle.CDF97, L)
        assert np.abs(c.cpu().numpy() - ref).max() <= TOL_F32
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    plan.close()


def _interior_bands(coef, k, levels, w, h):
    """(band name, array) of level k of a Mallat-packed array."""
    cw, ch = w, h
    for _ in range(k):
        cw, ch = (cw + 1) // 2, (ch + 1) // 2
    lw, lh = (cw + 1) // 2, (ch + 1) // 2
    bands = {"HL": coef[:lh, lw:cw], "LH": coef[lh:ch, :lw], "HH": coef[lh:ch, lw:cw]}
    if k == levels - 1:
        bands["LL"] = coef[:lh, :lw]
    return bands


@pytest.mark.parametrize("wavelet", ["cdf97"])
def test_largest_sweep_size_interior_against_oracle(dwt, wavelet):
    """16384 x 16384, 6 levels: the oracle cannot transform the whole image
    in seconds, but a level-k coefficient depends only on image samples
    within (filter radius) x 2^(k+1) of it.  The oracle runs on a 4096^2
    crop placed on a 2^6 grid; the GPU coefficients whose support lies
    inside the crop must match it."""
    n, L, S = 16384, 6, 4096
    r0, c0 = 7 * 1024, 5 * 1024  # multiples of 2^L: the crop keeps the polyphase grid
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    x = torch.randint(0, 256, (n, n), generator=g, device="cuda", dtype=torch.int32).float()
    c = torch.empty_like(x)
    plan = dwt.Plan(n, n, wavelet, L, "f32", scheme="monolithic*")
    plan.forward(x, c)
    torch.cuda.synchronize()
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    plan.close()
    crop = x[r0:r0 + S, c0:c0 + S].cpu().numpy().astype(np.float64)
    ref = oracle.dwt2(crop, OID[wavelet], L)
    cg = c.cpu().numpy()
    del x, c
    # A level-k coefficient depends on samples within sum_j 4 * 2^j < 4 *
    # 2^(k+1) of its position (the 9/7 analysis taps reach 4 samples at
    # every level): under 4 band units of level k.  The crop's own border
    # (mirrored) moves the crop's coefficients within that distance of its
    # edge, so 8 band units of margin are safe.
    margin = 8
    checked = 0
    for k in range(L):
        step = 2 ** (k + 1)
        gb = _interior_bands(cg, k, L, n, n)
        rb = _interior_bands(ref, k, L, S, S)
        br, bc = r0 // step, c0 // step  # crop origin in level-k band units
        m = S // step
        for name in rb:
            got = gb[name][br + margin:br + m - margin, bc + margin:bc + m - margin]
            exp = rb[name][margin:m - margin, margin:m - margin]
            assert got.shape == exp.shape and got.size > 0, (k, name)
            assert np.abs(got - exp).max() <= TOL_F32, (k, name)
            checked += got.size
    assert checked > 1_000_000


def test_misaligned_base_pointer_rejected(dwt):
    plan = dwt.Plan(64, 64, "cdf97", 2, "f32")
    buf = torch.zeros(64 * 64 + 4, device="cuda")
    out = torch.zeros(64, 64, device="cuda")
    raw = buf.data_ptr() + 2  # not on a 4-byte boundary
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt2_forward(plan.handle, raw, 256, out.data_ptr(), 256)
    assert e.value.status == dwt.DWT_EINVAL
    with pytest.raises(dwt.DwtError) as e:
        dwt.dwt2_forward(plan.handle, out.data_ptr(), 256, raw, 256)
    assert e.value.status == dwt.DWT_EINVAL
    plan.close()


@pytest.mark.parametrize("w", [1001, 1002, 1003])
def test_unaligned_pitches_all_offsets(dwt, w):
    """Row pitches of 4 w bytes put the rows (and the Mallat bands) at every
    offset from a 16-byte boundary: the box copies and split stores must
    agree with the oracle for each."""
    h, L = 203, 3
    for wl in ("cdf53", "cdf97"):
        x = inputs.uniform_image(h, w, seed=w + h)
        ref = oracle.dwt2(x.astype(np.float64), OID[wl], L)
        c, y, yo = run_fwd_inv(dwt, x, wl, L, "f32", "monolithic*", coef_in=ref.astype(np.float32))
        assert np.abs(c - ref).max() <= TOL_F32
        assert np.abs(yo - x).max() <= TOL_F32
    xi = inputs.int12_image(h, w, seed=w)
    refi = oracle.dwt2_int(xi, L)
    c, y, yo = run_fwd_inv(dwt, xi, "cdf53", L, "i32", "sweldens", coef_in=refi.astype(np.int32))
    assert np.array_equal(c, refi) and np.array_equal(yo, xi) and np.array_equal(y, xi)
