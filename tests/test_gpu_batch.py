"""GPU tests of dwt_batch_submit, the persistent kernel that runs every
level of many mixed requests in one launch: each request's result must be
bit-identical to the same plan's own call with the batch's scheme
(Monolithic* for float storage, the separable JPEG 2000 order for int32),
whatever else shares the batch, and within the oracle's tolerance."""
import numpy as np
import pytest

import oracle
from paper_1605_00561_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_F32 = 2e-3
TDT = {"f32": torch.float32, "f16s": torch.float16, "i32": torch.int32}
OID = {"cdf53": oracle.CDF53, "cdf97": oracle.CDF97, "dd137": oracle.DD137}


@pytest.fixture(scope="module")
def dwt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00561_gb300 import dwt as d
    d.lib()
    return d


def make_input(h, w, dtype, seed):
    if dtype == "i32":
        x = inputs.int12_image(h, w, seed=seed)
    else:
        x = inputs.uniform_image(h, w, seed=seed)
    return x


class Job:
    """One request: plan, device input, device output, host input."""

    def __init__(self, dwt, h, w, wavelet, levels, dtype, inverse, seed, pitch_pad=0):
        self.h, self.w, self.wavelet, self.levels, self.dtype, self.inverse = h, w, wavelet, levels, dtype, inverse
        self.plan = dwt.Plan(w, h, wavelet, levels, dtype,
                             scheme="sweldens" if dtype == "i32" else "monolithic*")
        x = make_input(h, w, dtype, seed)
        self.x = x
        if inverse:  # feed the oracle's coefficients of x
            if dtype == "i32":
                x = oracle.dwt2_int(x, levels).astype(np.int32)
            else:
                x = oracle.dwt2(x.astype(np.float64), OID[wavelet], levels).astype(np.float32)
        self.host_in = x
        t = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", TDT[dtype])
        if pitch_pad:
            buf = torch.zeros((h, w + pitch_pad), dtype=TDT[dtype], device="cuda")
            buf[:, :w] = t
            t = buf[:, :w]
        self.src = t
        self.dst = torch.full((h, w), 7, dtype=TDT[dtype], device="cuda")

    def request(self):
        return self.plan.request(self.src, self.dst, self.inverse)

    def alone(self):
        out = torch.full((self.h, self.w), 7, dtype=TDT[self.dtype], device="cuda")
        (self.plan.inverse if self.inverse else self.plan.forward)(self.src, out)
        return out

    def close(self):
        self.plan.close()


def check_vs_oracle(job, got):
    """Forward: the oracle's coefficients; inverse (fed the oracle's
    coefficients): the original image.  float16 storage has no bar."""
    if job.dtype == "i32":
        ref = job.x if job.inverse else oracle.dwt2_int(job.x, job.levels)
        assert np.array_equal(got.cpu().numpy(), ref)
    elif job.dtype == "f32":
        wl = OID[job.wavelet]
        ref = job.x.astype(np.float64) if job.inverse else oracle.dwt2(job.x.astype(np.float64), wl, job.levels)
        assert np.abs(got.cpu().numpy() - ref).max() <= TOL_F32


MIX = [  # h, w, wavelet, levels, dtype, inverse
    (150, 261, "cdf97", 3, "f32", False),
    (261, 150, "cdf97", 4, "f32", True),
    (64, 64, "cdf53", 6, "f32", False),
    (333, 500, "cdf53", 5, "f32", True),
    (1, 37, "cdf97", 3, "f32", False),
    (37, 1, "cdf53", 3, "f32", True),
    (2, 3, "cdf97", 2, "f32", False),
    (131, 9, "cdf97", 4, "f32", False),
    (333, 500, "cdf53", 5, "i32", False),
    (500, 333, "cdf53", 4, "i32", True),
    (5, 130, "cdf53", 2, "i32", False),
    (97, 203, "cdf97", 3, "f16s", False),
    (203, 97, "cdf97", 3, "f16s", True),
    (120, 77, "cdf53", 2, "f16s", False),
    (77, 120, "cdf53", 3, "f16s", True),
    (40, 50, "cdf97", 0, "f32", False),
    (1200, 1500, "cdf97", 6, "f32", False),
    (150, 261, "dd137", 3, "f32", False),
    (261, 150, "dd137", 2, "f32", True),
    (1, 37, "dd137", 2, "f32", False),
    (600, 700, "dd137", 4, "f32", False),
    (65536, 3, "cdf97", 3, "f32", False),
    (3, 65536, "cdf53", 3, "i32", True),
]


def make_jobs(dwt, spec, seed0=0):
    jobs = []
    for i, (h, w, wl, L, dt, inv) in enumerate(spec):
        jobs.append(Job(dwt, h, w, wl, L, dt, inv, seed=seed0 + 31 * i + 5, pitch_pad=(i % 3) * 8))
    return jobs


def test_mixed_batch_equals_single_calls_and_oracle(dwt):
    jobs = make_jobs(dwt, MIX)
    status = torch.full((len(jobs),), -1, dtype=torch.int32, device="cuda")
    dwt.submit([j.request() for j in jobs], status=status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [dwt.DWT_OK] * len(jobs)
    for j in jobs:
        alone = j.alone()
        torch.cuda.synchronize()
        assert torch.equal(j.dst, alone), (j.h, j.w, j.wavelet, j.levels, j.dtype, j.inverse)
        check_vs_oracle(j, j.dst)
    for j in jobs:
        j.close()


def test_request_alone_in_batch_equals_in_mix(dwt):
    jobs = make_jobs(dwt, MIX, seed0=100)
    dwt.submit([j.request() for j in jobs])
    torch.cuda.synchronize()
    mixed = [j.dst.clone() for j in jobs]
    for j, m in zip(jobs, mixed):
        j.dst.fill_(3)
        dwt.submit([j.request()])
        torch.cuda.synchronize()
        assert torch.equal(j.dst, m)
    for j in jobs:
        j.close()


def test_batch_of_256_images_mixed_sizes(dwt):
    shapes = inputs.batch_shapes(n=256, seed=8, lo=64, hi=1024)
    spec = [(h, w, "cdf97" if k == "cdf97" else "cdf53", 5, "f32" if k == "cdf97" else "i32", i % 4 == 3)
            for i, (w, h, k) in enumerate(shapes)]
    jobs = make_jobs(dwt, spec, seed0=1000)
    status = torch.full((len(jobs),), -1, dtype=torch.int32, device="cuda")
    dwt.submit([j.request() for j in jobs], status=status)
    torch.cuda.synchronize()
    assert int(status.abs().sum()) == 0
    for j in jobs:
        alone = j.alone()
        torch.cuda.synchronize()
        assert torch.equal(j.dst, alone)
    # the oracle on a sample of them
    for j in jobs[::37]:
        check_vs_oracle(j, j.dst)
    for j in jobs:
        j.close()


def test_one_plan_in_many_requests(dwt):
    """A plan only supplies parameters to a batch: one plan may serve many
    requests of its shape, each with its own buffers."""
    plan = dwt.Plan(203, 97, "cdf97", 4, "f32", scheme="monolithic*")
    xs = [torch.from_numpy(inputs.uniform_image(97, 203, seed=50 + i)).cuda() for i in range(5)]
    outs = [torch.empty_like(x) for x in xs]
    dwt.submit([plan.request(x, o) for x, o in zip(xs, outs)])
    for x, o in zip(xs, outs):
        alone = torch.empty_like(x)
        plan.forward(x, alone)
        torch.cuda.synchronize()
        assert torch.equal(o, alone)
    plan.close()


def test_back_to_back_batches_on_two_streams(dwt):
    a = make_jobs(dwt, MIX[:8], seed0=7)
    b = make_jobs(dwt, MIX[8:], seed0=9)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(3):
        with torch.cuda.stream(s1):
            dwt.submit([j.request() for j in a], stream=s1.cuda_stream)
        with torch.cuda.stream(s2):
            dwt.submit([j.request() for j in b], stream=s2.cuda_stream)
    torch.cuda.synchronize()
    for j in a + b:
        alone = j.alone()
        torch.cuda.synchronize()
        assert torch.equal(j.dst, alone)
        j.close()


def test_batch_rejections(dwt):
    j1, j2 = make_jobs(dwt, [(64, 80, "cdf97", 2, "f32", False), (64, 80, "cdf97", 2, "f32", False)])
    # two outputs in one buffer
    r2 = j2.plan.request(j2.src, j1.dst)
    with pytest.raises(dwt.DwtError) as e:
        dwt.submit([j1.request(), r2])
    assert e.value.status == dwt.DWT_EINVAL
    # an output over another request's input
    r2 = j2.plan.request(j2.src, j1.src)
    with pytest.raises(dwt.DwtError) as e:
        dwt.submit([j1.request(), r2])
    assert e.value.status == dwt.DWT_EINVAL
    dwt.submit([])
    for j in (j1, j2):
        j.close()
