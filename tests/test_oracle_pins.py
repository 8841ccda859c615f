"""Pins of the FP64 / exact-integer oracle against what the paper and the
mathematics fix, independently of the oracle's own code paths:

* brute-force 2-D convolution with the CDF filter taps under whole-sample
  symmetric extension (tiny images, including 1xN, 2xN and odd sizes);
* the 9/7 constants against the values of the paper's reference;
* vanishing moments, constant images, perfect reconstruction;
* the normalisation reading (DC gain 1, Nyquist gain 2) and the paper's zeta;
* integer range, length-1 lines and argument validation.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
from oracle import scheme_algebra as sa


# ----------------------------------------------------------------------------
# helpers written for the tests (no oracle code)
# ----------------------------------------------------------------------------

def wss(i, n):
    """Whole-sample symmetric extension index (test's own statement)."""
    if n == 1:
        return 0
    while i < 0 or i >= n:
        i = -i if i < 0 else 2 * (n - 1) - i
    return i


def compose_1d(pairs, slo=1, shi=1):
    """Analysis filters of a lifting factorisation by multiplying the 2x2
    polyphase matrices of Sec. 2.2 (1-D Laurent polynomials as dicts)."""
    def mul(a, b):
        r = {}
        for e1, c1 in a.items():
            for e2, c2 in b.items():
                r[e1 + e2] = r.get(e1 + e2, 0) + c1 * c2
        return r

    def add(a, b):
        r = dict(a)
        for e, c in b.items():
            r[e] = r.get(e, 0) + c
        return r

    # rows: output (L, H); columns: input polyphase component (even, odd)
    m = [[{0: 1}, {}], [{}, {0: 1}]]
    for p, u in pairs:
        m[1] = [add(m[1][0], mul(p, m[0][0])), add(m[1][1], mul(p, m[0][1]))]  # H += P L
        m[0] = [add(m[0][0], mul(u, m[1][0])), add(m[0][1], mul(u, m[1][1]))]  # L += U H
    lo, hi = {}, {}
    for e, c in m[0][0].items():
        lo[2 * e] = lo.get(2 * e, 0) + c * slo
    for e, c in m[0][1].items():
        lo[2 * e + 1] = lo.get(2 * e + 1, 0) + c * slo
    for e, c in m[1][0].items():  # centred on the odd sample 2n+1
        hi[2 * e - 1] = hi.get(2 * e - 1, 0) + c * shi
    for e, c in m[1][1].items():
        hi[2 * e] = hi.get(2 * e, 0) + c * shi
    return ({k: v for k, v in lo.items() if v != 0}, {k: v for k, v in hi.items() if v != 0})


def brute_force_level(x, lo, hi):
    """One level of the 2-D transform as four separable FIR filters with
    subsampling on the WSS-extended image; length-1 axes are untouched."""
    H, W = len(x), len(x[0])
    cw, ch = (W + 1) // 2, (H + 1) // 2
    out = [[0] * W for _ in range(H)]

    def taps_and_origin(i, n, nlo):
        if n == 1:
            return {0: 1}, 0
        return (lo, 2 * i) if i < nlo else (hi, 2 * (i - nlo) + 1)

    for r in range(H):
        ty, oy = taps_and_origin(r, H, ch)
        for c in range(W):
            tx, ox = taps_and_origin(c, W, cw)
            s = 0
            for dy, cy in ty.items():
                for dx, cx in tx.items():
                    s += cy * cx * x[wss(oy + dy, H)][wss(ox + dx, W)]
            out[r][c] = s
    return out


def golden_filters(golden, name):
    lo, hi = {}, {}
    for band, off, tap in golden(name):
        v = Fraction(tap) if "/" in tap or tap.isdigit() or tap.lstrip("-").isdigit() else float(tap)
        k = int(off)
        (lo if band == "low" else hi)[k] = v
    return lo, hi


def symmetric_full(taps, centre_odd=False):
    full = {}
    for k, v in taps.items():
        full[k] = v
        full[-k] = v
    return full


SIZES = [(1, 1), (1, 4), (4, 1), (2, 2), (2, 5), (3, 7), (5, 6), (7, 9), (8, 8), (11, 3)]


# ----------------------------------------------------------------------------
# CDF 5/3: exact
# ----------------------------------------------------------------------------

def paper_pair(golden, wavelet):
    """(P, U) of `wavelet` as the paper prints them (Sec. 5), converted from
    powers of z to quad offsets (z^e reads offset -e)."""
    ops = {"P": {}, "U": {}}
    for wl, op, e, c in golden("paper_lifting_pairs.txt"):
        if wl == wavelet:
            ops[op][-int(e)] = Fraction(c)
    return ops["P"], ops["U"]


def test_cdf53_filters_follow_from_paper_lifting(golden):
    lo_g, hi_g = golden_filters(golden, "cdf53_filters.txt")
    lo, hi = compose_1d([paper_pair(golden, "CDF 5/3")])
    assert lo == lo_g
    assert hi == hi_g


def test_scheme_algebra_pairs_are_the_papers(golden):
    # the step matrices of oracle/scheme_algebra.py are built from these pairs
    assert sa.cdf53() == [paper_pair(golden, "CDF 5/3")]
    assert sa.dd137() == [paper_pair(golden, "DD 13/7")]


@pytest.mark.parametrize("h,w", SIZES)
def test_cdf53_bruteforce_convolution_exact(golden, h, w):
    lo, hi = golden_filters(golden, "cdf53_filters.txt")
    rng = np.random.default_rng(100 + 7 * h + w)
    x = rng.integers(0, 256, (h, w))
    ref = brute_force_level([[Fraction(int(v)) for v in row] for row in x], lo, hi)
    got = oracle.dwt2(x.astype(float), oracle.CDF53, 1 if max(h, w) > 1 else 0)
    if max(h, w) == 1:
        ref = [[Fraction(int(x[0, 0]))]]
    # 5/3 taps are dyadic rationals: FP64 reproduces them exactly here
    assert [[Fraction(v) for v in row] for row in got.tolist()] == ref


# ----------------------------------------------------------------------------
# CDF 9/7
# ----------------------------------------------------------------------------

def test_cdf97_constants_match_reference(golden):
    a, b, g, d, K, res = oracle.cdf97_constants()
    ref = {k: float(v) for k, v in golden("cdf97_lifting_constants.txt")}
    assert res < 1e-13
    for name, got in zip(("alpha", "beta", "gamma", "delta"), (a, b, g, d)):
        assert abs(got - ref[name]) < 2e-9, name
    # the paper's zeta makes the low-pass DC gain sqrt(2): zeta = sqrt(2) / K
    assert abs(math.sqrt(2) / K - ref["zeta"]) < 2e-9


def test_cdf97_filters_from_constants(golden):
    a, b, g, d, K, _ = oracle.cdf97_constants()
    lo, hi = compose_1d(sa.cdf97(a, b, g, d), 1 / K, K)
    lo_g, hi_g = golden_filters(golden, "cdf97_filters.txt")
    for k, v in symmetric_full(lo_g).items():
        assert abs(lo.get(k, 0) - v) < 1e-11
    for k, v in symmetric_full(hi_g).items():
        assert abs(hi.get(k, 0) - v) < 1e-10
    assert set(lo) == set(symmetric_full(lo_g)) and set(hi) == set(symmetric_full(hi_g))
    # normalisation reading: DC gain of the low-pass 1, Nyquist gain of the high-pass 2
    assert abs(sum(lo.values()) - 1) < 1e-13
    assert abs(sum(v * (-1) ** k for k, v in hi.items()) - 2) < 1e-12


@pytest.mark.parametrize("h,w", SIZES)
def test_cdf97_bruteforce_convolution(h, w):
    a, b, g, d, K, _ = oracle.cdf97_constants()
    lo, hi = compose_1d(sa.cdf97(a, b, g, d), 1 / K, K)
    rng = np.random.default_rng(200 + 7 * h + w)
    x = rng.integers(0, 256, (h, w)).astype(float)
    L = 1 if max(h, w) > 1 else 0
    ref = np.array(brute_force_level(x.tolist(), lo, hi)) if L else x
    got = oracle.dwt2(x, oracle.CDF97, L)
    assert np.max(np.abs(got - ref)) < 1e-11


@pytest.mark.parametrize("h,w", [(2, 9), (6, 5), (9, 9)])
def test_dd137_bruteforce_convolution(golden, h, w):
    lo, hi = compose_1d([paper_pair(golden, "DD 13/7")])
    rng = np.random.default_rng(300 + h * w)
    x = rng.integers(0, 256, (h, w))
    ref = brute_force_level([[Fraction(int(v)) for v in row] for row in x], lo, hi)
    got = oracle.dwt2(x.astype(float), oracle.DD137, 1)
    assert np.max(np.abs(got - np.array(ref, dtype=float))) < 1e-10


# ----------------------------------------------------------------------------
# properties
# ----------------------------------------------------------------------------

def test_vanishing_moments_cdf53_linear():
    H, W = 24, 30
    r, c = np.mgrid[0:H, 0:W].astype(float)
    x = 3.0 + 2.0 * c - 5.0 * r
    y = oracle.dwt2(x, oracle.CDF53, 1)
    ch, cw = H // 2, W // 2
    m = 2  # quads away from the borders
    assert np.all(y[m:ch - m, cw + m:W - m] == 0)      # HL
    assert np.all(y[ch + m:H - m, m:cw - m] == 0)      # LH
    assert np.all(y[ch + m:H - m, cw + m:W - m] == 0)  # HH
    assert np.abs(y[m:ch - m, m:cw - m]).max() > 0


def test_vanishing_moments_cdf97_cubic():
    H, W = 40, 44
    r, c = np.mgrid[0:H, 0:W].astype(float)
    f = lambda t: 0.001 * t ** 3 - 0.05 * t ** 2 + 0.7 * t + 4
    x = f(c) + 0.5 * f(r)
    y = oracle.dwt2(x, oracle.CDF97, 1)
    ch, cw = H // 2, W // 2
    m = 3
    scale = np.abs(x).max()
    for blk in (y[m:ch - m, cw + m:W - m], y[ch + m:H - m, m:cw - m], y[ch + m:H - m, cw + m:W - m]):
        assert np.abs(blk).max() < 1e-11 * scale
    # a quartic is not annihilated: the pin is not vacuous
    y4 = oracle.dwt2((c / 4) ** 4, oracle.CDF97, 1)
    assert np.abs(y4[m:ch - m, cw + m:W - m]).max() > 1e-3


@pytest.mark.parametrize("wl", [oracle.CDF53, oracle.CDF97])
@pytest.mark.parametrize("h,w", [(37, 50), (64, 64), (1, 17)])
def test_constant_image_every_level(wl, h, w):
    L = oracle.max_levels(w, h)
    y = oracle.dwt2(np.full((h, w), 117.0), wl, L)
    # all detail bands vanish and the final LL is the constant (DC gain 1)
    assert abs(y[0, 0] - 117.0) < 1e-11
    y[0, 0] = 0.0
    assert np.abs(y).max() < 1e-10


@pytest.mark.parametrize("wl", [oracle.CDF53, oracle.CDF97, oracle.DD137])
@pytest.mark.parametrize("h,w,L", [(33, 47, 4), (64, 64, 6), (2, 3, 2), (1, 9, 4), (9, 1, 4)])
def test_perfect_reconstruction_float(wl, h, w, L):
    x = np.random.default_rng(h * 31 + w).integers(0, 256, (h, w)).astype(float)
    y = oracle.dwt2(x, wl, L)
    assert np.abs(oracle.dwt2(y, wl, L, inverse=True) - x).max() < 1e-10


@pytest.mark.parametrize("wl", [oracle.CDF53, oracle.CDF97])
def test_zeta_normalisation(wl):
    # paper's scaling (Sec. 2.2, zeta = sqrt(2) for 5/3, Sec. 5): the low-pass
    # gain becomes sqrt(2) per axis, so a constant image's LL is 2c per level
    x = np.full((16, 16), 5.0)
    y = oracle.dwt2(x, wl, 1, norm=oracle.NORM_ZETA)
    assert abs(y[0, 0] - 10.0) < 1e-12
    z = oracle.dwt2(y, wl, 1, inverse=True, norm=oracle.NORM_ZETA)
    assert np.abs(z - x).max() < 1e-12


def test_length1_lines_untouched():
    x = np.arange(9, dtype=float).reshape(1, 9) * 3 + 1
    y1 = oracle.dwt2(x, oracle.CDF97, 1)
    # a 1x9 image: the vertical length-1 transform is the identity, the
    # horizontal one is the plain 1-D transform
    assert np.allclose(y1[0], oracle.dwt1(x[0], oracle.CDF97))
    assert np.array_equal(oracle.dwt1([5.0], oracle.CDF97), [5.0])
    assert np.array_equal(oracle.dwt1_int([5]), [5])


# ----------------------------------------------------------------------------
# reversible integer 5/3
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("h,w,L", [(33, 47, 5), (64, 64, 6), (5, 2, 3), (1, 13, 4), (13, 1, 4), (1, 1, 0)])
def test_integer_exact_round_trip(h, w, L):
    x = np.random.default_rng(h * 7 + w).integers(0, 4096, (h, w))
    y = oracle.dwt2_int(x, L)
    assert np.array_equal(oracle.dwt2_int(y, L, inverse=True), x)


def test_integer_linear_ramps_and_constants_exact():
    r, c = np.mgrid[0:20, 0:22]
    y = oracle.dwt2_int(3 * c + 7 * r + 11, 1)
    assert np.all(y[2:8, 13:19] == 0) and np.all(y[12:18, 2:9] == 0)
    yc = oracle.dwt2_int(np.full((20, 22), 1234), 3)
    # after 3 levels LL is ceil(20/8) x ceil(22/8) = 3 x 3
    assert np.all(yc[:3, :3] == 1234) and np.count_nonzero(yc) == 9


def _ints(field):
    return [int(v) for v in field.split()]


def test_integer_golden_lines(golden):
    # hand-derived JPEG 2000 reversible 5/3 lines (tests/golden/int53_vectors.txt)
    rows = [r for r in golden("int53_vectors.txt") if len(r) == 3]
    assert len(rows) == 5
    for name, x, y in rows:
        got = oracle.dwt1_int(_ints(x))
        assert got.tolist() == _ints(y), name
        assert oracle.dwt1_int(got, inverse=True).tolist() == _ints(x), name


def test_integer_golden_image(golden):
    (name, h, w, L, x, y), = [r for r in golden("int53_vectors.txt") if len(r) == 6]
    h, w, L = int(h), int(w), int(L)
    x = np.array(_ints(x)).reshape(h, w)
    want = np.array(_ints(y)).reshape(h, w)
    got = oracle.dwt2_int(x, L)
    assert np.array_equal(got, want), name
    assert np.array_equal(oracle.dwt2_int(got, L, inverse=True), x)


def _lift53_int_variant(x, plus2=True, predict="floor", update="floor"):
    """The test's own statement of the reversible 5/3 forward line, with a
    rounding mistake planted on request: the update without its +2, the
    predict rounding half up (floor((a + b + 1)/2)) or truncating toward
    zero, the update truncating toward zero."""
    def trunc_div(a, b):
        q = abs(a) // b
        return q if a >= 0 else -q

    n, t = len(x), list(x)
    if n == 1:
        return t
    for i in range(1, n, 2):
        a = t[wss(i - 1, n)] + t[wss(i + 1, n)]
        t[i] -= {"floor": a // 2, "half_up": (a + 1) // 2, "trunc": trunc_div(a, 2)}[predict]
    for i in range(0, n, 2):
        a = t[wss(i - 1, n)] + t[wss(i + 1, n)] + (2 if plus2 else 0)
        t[i] += a // 4 if update == "floor" else trunc_div(a, 4)
    return t[0::2] + t[1::2]


@pytest.mark.parametrize("mistake", [dict(plus2=False), dict(predict="half_up"), dict(predict="trunc"),
                                     dict(update="trunc")])
def test_integer_golden_lines_catch_rounding_mistakes(golden, mistake):
    # the vectors are not vacuous: each plausible rounding mistake changes
    # the result of at least one golden line (the unplanted statement
    # reproduces all of them)
    rows = [r for r in golden("int53_vectors.txt") if len(r) == 3]
    assert all(_lift53_int_variant(_ints(x)) == _ints(y) for _, x, y in rows)
    assert any(_lift53_int_variant(_ints(x), **mistake) != _ints(y) for _, x, y in rows)


def test_integer_1d_rounding_error_intervals():
    # Float 5/3 (JPEG 2000 normalisation leaves it unscaled) is the reversible
    # transform without its floors.  From the two equations: the high-pass
    # error is (a + b)/2 - floor((a + b)/2), which is 0 or 1/2; the low-pass
    # error is floor((D + 2)/4) - D/4 + (e1 + e2)/4 with D = d1 + d2 and e1,
    # e2 the two high-pass errors, which lies in [-1/4, 3/4].  A dropped +2
    # moves the low band to [-3/4, 1/4], half-up rounding the high band to
    # [-1/2, 0]: random lines hit those outside the intervals.
    rng = np.random.default_rng(17)
    for n in (2, 3, 8, 9, 64, 65):
        for _ in range(200 // n + 5):
            x = rng.integers(-4096, 4096, n)
            ei = oracle.dwt1_int(x) - oracle.dwt1(x.astype(float), oracle.CDF53)
            nlo = (n + 1) // 2
            lo, hi = ei[:nlo], ei[nlo:]
            assert np.all((hi == 0) | (hi == 0.5))
            assert lo.min() >= -0.25 and lo.max() <= 0.75


def test_integer_2d_rounding_error_intervals():
    # One 2-D level: the column pass leaves errors in [-1/4, 3/4] (low rows)
    # and [0, 1/2] (high rows); the row pass adds its own and maps the column
    # errors through the float filters.  The high-pass filter (-1/2, 1, -1/2)
    # maps [a, b] to [-(b - a), b - a]; the low-pass filter (-1/8, 1/4, 3/4,
    # 1/4, -1/8; positive taps 5/4, negative -1/4) maps [a, b] to
    # [5a/4 - b/4, 5b/4 - a/4].  So LL in [-3/4, 7/4], HL in [-1, 3/2], LH in
    # [-3/8, 11/8], HH in [-1/2, 1].
    rng = np.random.default_rng(5)
    for h, w in ((40, 36), (33, 47), (2, 9), (64, 64)):
        x = rng.integers(0, 4096, (h, w))
        e = oracle.dwt2_int(x, 1) - oracle.dwt2(x.astype(float), oracle.CDF53, 1)
        ch, cw = (h + 1) // 2, (w + 1) // 2
        bands = {"LL": (e[:ch, :cw], -0.75, 1.75), "HL": (e[:ch, cw:], -1.0, 1.5),
                 "LH": (e[ch:, :cw], -0.375, 1.375), "HH": (e[ch:, cw:], -0.5, 1.0)}
        for name, (b, lo, hi) in bands.items():
            assert b.min() >= lo and b.max() <= hi, (name, h, w, b.min(), b.max())
        assert np.abs(e).max() > 0


def test_integer_range_12bit_five_levels_and_overflow_detected():
    x = np.random.default_rng(9).integers(0, 4096, (97, 113))
    y = oracle.dwt2_int(x, 5)
    assert np.abs(y).max() < 2 ** 16
    big = np.full((8, 8), 2 ** 31 - 1)
    big[::2, ::2] = -(2 ** 31)
    with pytest.raises(oracle.OracleRangeError):
        oracle.dwt2_int(big, 1)


def test_integer_step_order_matters():
    # the three plausible 2-D orders give different integer results, so the
    # column-then-row order (JPEG 2000) is a fixed part of the contract
    x = np.random.default_rng(11).integers(0, 4096, (9, 12))
    cols_first = oracle.dwt2_int(x, 1)
    rows_first = oracle.dwt2_int(x.T.copy(), 1).T
    assert not np.array_equal(cols_first, rows_first)


# ----------------------------------------------------------------------------
# argument validation
# ----------------------------------------------------------------------------

def test_max_levels_and_invalid_arguments():
    assert oracle.max_levels(1, 1) == 0
    assert oracle.max_levels(2, 1) == 1
    assert oracle.max_levels(8192, 8192) == 13
    assert oracle.max_levels(5001, 3333) == 13
    with pytest.raises(ValueError):
        oracle.dwt2(np.zeros((4, 4)), oracle.CDF53, 3)
    with pytest.raises(ValueError):
        oracle.dwt2(np.zeros((4, 4)), oracle.CDF53, -1)


# ----------------------------------------------------------------------------
# reversible integer non-separable lifting (the integer Iwahashi scheme)
# ----------------------------------------------------------------------------

def test_integer_iwahashi_golden(golden):
    rows = golden("int_iwahashi_vectors.txt")
    assert len(rows) == 2
    for name, h, w, L, x, y in rows:
        h, w, L = int(h), int(w), int(L)
        x = np.array(_ints(x)).reshape(h, w)
        want = np.array(_ints(y)).reshape(h, w)
        got = oracle.dwt2_int_iwahashi(x, L)
        assert np.array_equal(got, want), name
        assert np.array_equal(oracle.dwt2_int_iwahashi(got, L, inverse=True), x), name


@pytest.mark.parametrize("h,w,L", [(33, 47, 5), (64, 64, 6), (5, 2, 3), (1, 13, 4), (13, 1, 4), (2, 2, 1)])
def test_integer_iwahashi_exact_round_trip(h, w, L):
    x = np.random.default_rng(h * 11 + w).integers(0, 4096, (h, w))
    y = oracle.dwt2_int_iwahashi(x, L)
    assert np.array_equal(oracle.dwt2_int_iwahashi(y, L, inverse=True), x)
    # a different reversible transform from the JPEG 2000 one
    if h > 2 and w > 2:
        assert not np.array_equal(y, oracle.dwt2_int(x, L))


def test_integer_iwahashi_linear_ramps_and_constants():
    r, c = np.mgrid[0:20, 0:22]
    y = oracle.dwt2_int_iwahashi(3 * c + 7 * r + 11, 1)
    # the predict of a linear ramp is exact away from the borders
    assert np.all(y[2:8, 13:19] == 0) and np.all(y[12:18, 2:9] == 0) and np.all(y[12:18, 13:19] == 0)
    yc = oracle.dwt2_int_iwahashi(np.full((20, 22), 1234), 3)
    assert np.all(yc[:3, :3] == 1234) and np.count_nonzero(yc) == 9


def test_integer_iwahashi_error_intervals_against_float():
    # Each step rounds its whole update once, half up: an error in (-1/2,
    # 1/2] per step.  T leaves HH within 1/2 of the float transform; R adds
    # u (two HH errors) to its own, so HL, LH within 3/4; S adds u (four
    # HL/LH errors, 3/4 in all) and u^2 (four HH errors, 1/8 in all) to its
    # own, so LL within 11/8.  Without the rounding offsets the intervals
    # shift by 1/2 and random images leave them.
    rng = np.random.default_rng(23)
    for h, w in ((40, 36), (33, 47), (2, 9), (64, 64), (9, 2)):
        x = rng.integers(0, 4096, (h, w))
        e = oracle.dwt2_int_iwahashi(x, 1) - oracle.dwt2(x.astype(float), oracle.CDF53, 1)
        ch, cw = (h + 1) // 2, (w + 1) // 2
        assert np.abs(e[ch:, cw:]).max() <= 0.5
        assert np.abs(e[:ch, cw:]).max() <= 0.75 and np.abs(e[ch:, :cw]).max() <= 0.75
        assert np.abs(e[:ch, :cw]).max() <= 11 / 8
        assert np.abs(e).max() > 0
