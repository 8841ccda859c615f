"""Inverse transforms whose HL and HH planes start off a 16-byte boundary in
coefficient rows padded to a 16-byte multiple (odd ceil(w/2), the Mallat
layout of most odd widths).  Such planes load by TMA from the aligned column
before their start, the kernel reading each lane's elements from the
shifted box (encode_level_maps, Strip::set_box_cols).  Every residue of
ceil(w/2) mod 4 is covered, for the per-level kernels of several schemes
(boxes as wide as the span and boxes with room), float16 storage, the
integer 5/3 (bit-exact), a batch, and rows packed without padding (no
tensor map: lane copies), all against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_F32 = 2e-3
OID = {"cdf53": oracle.CDF53, "cdf97": oracle.CDF97, "dd137": oracle.DD137}
TDT = {"f32": torch.float32, "f16s": torch.float16, "i32": torch.int32}

# ceil(w/2) = 501, 502, 503, 504: HL starts 1, 2, 3, 0 elements past a
# 16-byte boundary (4-byte samples)
WIDTHS = [1001, 1003, 1005, 1007]


@pytest.fixture(scope="module")
def dwt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt as d
    d.lib()
    return d


def padded(a, dtype, pad_bytes=128):
    """A device copy of the 2-D array `a` in rows padded to pad_bytes."""
    h, w = a.shape
    es = torch.empty((), dtype=TDT[dtype]).element_size()
    pitch = -(-w * es // pad_bytes) * pad_bytes // es
    buf = torch.zeros(h, pitch, dtype=TDT[dtype], device="cuda")
    buf[:, :w] = torch.from_numpy(np.ascontiguousarray(a)).to(TDT[dtype]).cuda()
    return buf[:, :w]


def inverse_of_oracle(dwt, x, wavelet, L, dtype, scheme, pad):
    h, w = x.shape
    ref = oracle.dwt2_int(x, L) if dtype == "i32" else oracle.dwt2(x.astype(np.float64), OID[wavelet], L)
    plan = dwt.Plan(w, h, wavelet, L, dtype, scheme=scheme)
    c = padded(ref, dtype) if pad else torch.from_numpy(np.ascontiguousarray(ref)).to(TDT[dtype]).cuda()
    y = torch.empty(h, w, dtype=TDT[dtype], device="cuda")
    plan.inverse(c, y)
    # and a round trip through coefficients in padded rows
    c2 = padded(np.zeros_like(ref), dtype) if pad else torch.empty_like(c)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(TDT[dtype]).cuda()
    y2 = torch.empty_like(y)
    plan.forward(xd, c2)
    plan.inverse(c2, y2)
    torch.cuda.synchronize()
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK
    plan.close()
    return y.cpu().numpy(), y2.cpu().numpy(), x


@pytest.mark.parametrize("w", WIDTHS)
@pytest.mark.parametrize("scheme,wavelet", [("monolithic*", "cdf97"), ("monolithic*", "cdf53"),
                                            ("sweldens", "cdf97"), ("polyphase", "cdf53"),
                                            ("convolution", "cdf97"), ("iwahashi", "cdf97"),
                                            ("monolithic*", "dd137")])
def test_inverse_padded_odd_widths_float32(dwt, w, scheme, wavelet):
    x = inputs.uniform_image(517, w, seed=w)
    y, y2, x = inverse_of_oracle(dwt, x, wavelet, 3, "f32", scheme, pad=True)
    assert np.abs(y.astype(np.float64) - x).max() <= TOL_F32
    assert np.abs(y2.astype(np.float64) - x).max() <= 2 * TOL_F32


@pytest.mark.parametrize("w", WIDTHS)
def test_inverse_padded_odd_widths_int53(dwt, w):
    x = inputs.int12_image(333, w, seed=w)
    y, y2, x = inverse_of_oracle(dwt, x, "cdf53", 4, "i32", "sweldens", pad=True)
    assert np.array_equal(y, x) and np.array_equal(y2, x)


@pytest.mark.parametrize("w", [1001, 1003, 1005, 1007, 1011, 1013])
def test_inverse_padded_odd_widths_float16(dwt, w):
    # float16: ceil(w/2) mod 8 takes other residues; boxes have room for any
    x = inputs.uniform_image(300, w, seed=w)
    y, y2, x = inverse_of_oracle(dwt, x, "cdf97", 3, "f16s", "monolithic*", pad=True)
    # the coefficients are rounded to float16 on the way in: compare with
    # the same plan on packed rows (lane copies), which must agree exactly
    yp, y2p, _ = inverse_of_oracle(dwt, x, "cdf97", 3, "f16s", "monolithic*", pad=False)
    assert np.array_equal(y, yp) and np.array_equal(y2, y2p)


@pytest.mark.parametrize("w", WIDTHS)
def test_padded_equals_packed_bit_for_bit(dwt, w):
    # the realigned TMA path and the lane-copy path put the same values in
    # the same shared-memory layout before the same arithmetic
    x = inputs.uniform_image(400, w, seed=3 * w)
    y, y2, _ = inverse_of_oracle(dwt, x, "cdf97", 3, "f32", "monolithic*", pad=True)
    yp, y2p, _ = inverse_of_oracle(dwt, x, "cdf97", 3, "f32", "monolithic*", pad=False)
    assert np.array_equal(y, yp) and np.array_equal(y2, y2p)


def test_batch_inverse_padded_odd_widths(dwt):
    reqs, ins, outs, refs, plans = [], [], [], [], []
    for i, w in enumerate([1001, 1003, 1005, 1007, 701, 333]):
        h = 300 + 7 * i
        x = inputs.uniform_image(h, w, seed=i)
        ref = oracle.dwt2(x.astype(np.float64), oracle.CDF97, 3)
        p = dwt.Plan(w, h, "cdf97", 3, "f32")
        c = padded(ref, "f32")
        y = padded(np.zeros((h, w)), "f32")
        reqs.append(p.request(c, y, inverse=True))
        ins.append(c)  # a request holds raw pointers: keep its buffers alive
        outs.append(y)
        refs.append(x)
        plans.append(p)
    dwt.submit(reqs)
    torch.cuda.synchronize()
    for y, x in zip(outs, refs):
        assert np.abs(y.cpu().numpy().astype(np.float64) - x).max() <= TOL_F32
    for p in plans:
        p.close()
