"""Seeded random configurations against the oracle: sizes from 1 to about
700 per side (odd, even, lines), every level count a size allows, every
float scheme with CDF 5/3, 9/7 and DD 13/7, the integer transforms, row
pitches packed, padded to 16 or 128 bytes or padded by an odd number of
elements, the fused tail on or off and random strip heights and ring
depths.  Each case checks the forward transform, the inverse of the
oracle's coefficients and the round trip; int32 bit for bit, float32
within the 8-bit-range bar, which is stated for up to six levels: deeper
pyramids (up to ten levels here) add one rounding of the LL band per
level, so the bar scales with L / 6 beyond six (the unstarred Polyphase
9/7 round trip reaches 4.7e-3 at ten levels).  A failure message carries
the configuration."""
import numpy as np
import pytest

import oracle
from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_F32 = 2e-3
OID = {"cdf53": oracle.CDF53, "cdf97": oracle.CDF97, "dd137": oracle.DD137}
FLOAT_SCHEMES = ["rowcol", "sweldens", "iwahashi", "iwahashi*", "explosive", "explosive*", "monolithic",
                 "monolithic*", "polyphase", "polyphase*", "convolution"]
NCASES = 160


def cases():
    rng = np.random.default_rng(20261204)
    out = []
    for i in range(NCASES):
        side = lambda: int(np.clip(np.round(np.exp(rng.uniform(0.0, np.log(720.0)))), 1, 720))
        h, w = side(), side()
        if rng.random() < 0.1:
            h = 1 if rng.random() < 0.5 else h
            w = 1 if h != 1 else w
        kind = rng.choice(["float", "float", "float", "int53", "intiw"])
        if kind == "float":
            wavelet = str(rng.choice(["cdf53", "cdf97", "dd137"]))
            scheme = str(rng.choice(FLOAT_SCHEMES))
        else:
            wavelet, scheme = "cdf53", ("sweldens" if rng.random() < 0.7 else "rowcol") if kind == "int53" else "iwahashi"
        L = int(rng.integers(0, oracle.max_levels(w, h) + 1))
        pad = str(rng.choice(["packed", "16", "128", "odd"]))
        fusion = int(rng.choice([-1, 0]))
        rows = int(rng.choice([0, 0, 2, 7, 16, 40]))
        stages = int(rng.choice([0, 0, 1, 3, 4]))
        out.append((i, h, w, L, kind, wavelet, scheme, pad, fusion, rows, stages))
    return out


@pytest.fixture(scope="module")
def dwt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt as d
    d.lib()
    return d


def buffer(a, tdt, pad):
    """A device copy of the 2-D array `a` with rows laid out per `pad`."""
    h, w = a.shape
    es = torch.empty((), dtype=tdt).element_size()
    if pad == "packed":
        pitch = w
    elif pad == "odd":
        pitch = w + 3
    else:
        q = int(pad)
        pitch = -(-w * es // q) * q // es
    buf = torch.zeros(h, pitch, dtype=tdt, device="cuda")
    buf[:, :w] = torch.from_numpy(np.ascontiguousarray(a)).to(tdt).cuda()
    return buf[:, :w]


@pytest.mark.parametrize("case", cases(), ids=lambda c: f"c{c[0]}")
def test_fuzz_against_oracle(dwt, case):
    i, h, w, L, kind, wavelet, scheme, pad, fusion, rows, stages = case
    what = (f"h={h} w={w} L={L} {kind} {wavelet} {scheme} pitch={pad} fusion={fusion} rows={rows} "
            f"stages={stages}")
    if kind == "float":
        x = inputs.uniform_image(h, w, seed=100 + i)
        ref = oracle.dwt2(x.astype(np.float64), OID[wavelet], L)
        dtype, tdt = "f32", torch.float32
    else:
        x = inputs.int12_image(h, w, seed=100 + i)
        ref = oracle.dwt2_int(x, L) if kind == "int53" else oracle.dwt2_int_iwahashi(x, L)
        dtype, tdt = "i32", torch.int32
    plan = dwt.Plan(w, h, wavelet, L, dtype, scheme=scheme)
    dwt.dwt_plan_set_fusion(plan.handle, fusion)
    if rows or stages:
        dwt.dwt_plan_set_tile(plan.handle, rows, stages)
    xd = buffer(x, tdt, pad)
    c = buffer(np.zeros((h, w)), tdt, pad)
    y = buffer(np.zeros((h, w)), tdt, pad)
    co = buffer(ref, tdt, pad)
    yo = buffer(np.zeros((h, w)), tdt, pad)
    plan.forward(xd, c)
    plan.inverse(c, y)
    plan.inverse(co, yo)
    torch.cuda.synchronize()
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK, what
    plan.close()
    c, y, yo = c.cpu().numpy(), y.cpu().numpy(), yo.cpu().numpy()
    if dtype == "i32":
        assert np.array_equal(c, ref), "forward: " + what
        assert np.array_equal(yo, x), "inverse of oracle coefficients: " + what
        assert np.array_equal(y, x), "round trip: " + what
    else:
        tol = TOL_F32 * max(1.0, L / 6.0)
        assert np.abs(c.astype(np.float64) - ref).max() <= tol, "forward: " + what
        assert np.abs(yo.astype(np.float64) - x).max() <= tol, "inverse of oracle coefficients: " + what
        assert np.abs(y.astype(np.float64) - x).max() <= 2 * tol, "round trip: " + what


def test_fuzz_batch_against_oracle(dwt):
    """48 seeded random requests in one batch: sizes 1-709, every level
    count, CDF 5/3, 9/7 and DD 13/7 in float32 and the integer 5/3, both
    directions, packed and padded pitches.  A batch runs Monolithic* for
    float and the JPEG 2000 order for int32, whatever scheme a plan names."""
    rng = np.random.default_rng(4120)
    reqs, keep, checks, plans = [], [], [], []
    for i in range(48):
        h, w = (int(np.clip(np.round(np.exp(rng.uniform(0.0, np.log(720.0)))), 1, 720)) for _ in range(2))
        kind = "int53" if rng.random() < 0.3 else "float"
        wavelet = "cdf53" if kind == "int53" else str(rng.choice(["cdf53", "cdf97", "dd137"]))
        L = int(rng.integers(0, oracle.max_levels(w, h) + 1))
        inverse = bool(rng.random() < 0.5)
        pad = str(rng.choice(["packed", "16", "128", "odd"]))
        if kind == "float":
            x = inputs.uniform_image(h, w, seed=500 + i)
            ref = oracle.dwt2(x.astype(np.float64), OID[wavelet], L)
            dtype, tdt = "f32", torch.float32
        else:
            x = inputs.int12_image(h, w, seed=500 + i)
            ref = oracle.dwt2_int(x, L)
            dtype, tdt = "i32", torch.int32
        p = dwt.Plan(w, h, wavelet, L, dtype, scheme=str(rng.choice(FLOAT_SCHEMES)) if kind == "float" else "sweldens")
        src = buffer(ref if inverse else x, tdt, pad)
        dst = buffer(np.zeros((h, w)), tdt, pad)
        reqs.append(p.request(src, dst, inverse=inverse))
        keep.append((src, dst))
        plans.append(p)
        checks.append((dst, x if inverse else ref, dtype, L,
                       f"request {i}: h={h} w={w} L={L} {kind} {wavelet} {'inv' if inverse else 'fwd'} pitch={pad}"))
    status = torch.zeros(len(reqs), dtype=torch.int32, device="cuda")
    dwt.submit(reqs, status=status)
    torch.cuda.synchronize()
    assert int(status.abs().max()) == 0
    for dst, want, dtype, L, what in checks:
        got = dst.cpu().numpy()
        if dtype == "i32":
            assert np.array_equal(got, want), what
        else:
            assert np.abs(got.astype(np.float64) - want).max() <= TOL_F32 * max(1.0, L / 6.0), what
    for p in plans:
        p.close()
