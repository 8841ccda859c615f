"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no wavelet arithmetic; the oracle and the CUDA path both
consume what it returns.  The paper names no image data set, so these stand
in for it:

* ``uniform_image``: 8-bit grayscale, integers uniform in 0..255 (float32);
* ``textured_image``: uniform 0..255 plus a smooth component, the sum of 4
  sinusoids with random direction, frequency 0.5-8 cycles per image and
  phase, each of amplitude 16 (so the smooth part stays within +-64);
* ``int12_image``: int32 samples uniform in 0..4095 (12-bit);
* ``batch_shapes``: sizes of a mixed batch, widths and heights uniform in
  [256, 4096] (odd sizes included), half CDF 9/7 and half integer 5/3;
* ``serving_trace``: Poisson arrivals with log-normal image areas.
"""
from __future__ import annotations

import math

import numpy as np


def uniform_image(h: int, w: int, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(h, w), dtype=np.int32).astype(np.float32)


def textured_image(h: int, w: int, seed: int = 2, chunk_rows: int = 1024) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = rng.integers(0, 256, size=(h, w), dtype=np.int32).astype(np.float32)
    n = max(h, w)
    theta = rng.uniform(0.0, 2.0 * math.pi, 4)
    freq = rng.uniform(0.5, 8.0, 4)
    phase = rng.uniform(0.0, 2.0 * math.pi, 4)
    xs = np.arange(w, dtype=np.float32)
    for r0 in range(0, h, chunk_rows):
        ys = np.arange(r0, min(h, r0 + chunk_rows), dtype=np.float32)[:, None]
        acc = np.zeros((ys.shape[0], w), dtype=np.float32)
        for k in range(4):
            kx = np.float32(2.0 * math.pi * freq[k] * math.cos(theta[k]) / n)
            ky = np.float32(2.0 * math.pi * freq[k] * math.sin(theta[k]) / n)
            acc += np.float32(16.0) * np.sin(kx * xs[None, :] + ky * ys + np.float32(phase[k]))
        out[r0:r0 + ys.shape[0]] += acc
    return out


def int12_image(h: int, w: int, seed: int = 7) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 4096, size=(h, w), dtype=np.int32)


def batch_shapes(n: int = 256, seed: int = 8, lo: int = 256, hi: int = 4096):
    """[(w, h, kind)] with kind "cdf97" (float32) for the first half and
    "int53" (int32) for the second half."""
    rng = np.random.default_rng(seed)
    ws = rng.integers(lo, hi + 1, size=n)
    hs = rng.integers(lo, hi + 1, size=n)
    return [(int(ws[i]), int(hs[i]), "cdf97" if i < n // 2 else "int53") for i in range(n)]


def serving_trace(rate: float = 2000.0, seconds: float = 60.0, seed: int = 9, median_area: float = 1 << 20,
                  sigma: float = 1.0, lo: int = 64, hi: int = 8192, frac97: float = 0.7):
    """Poisson arrival stream: list of dicts (t, w, h, levels, kind)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        area = median_area * math.exp(sigma * rng.standard_normal())
        aspect = rng.uniform(0.5, 2.0)
        w = int(min(hi, max(lo, round(math.sqrt(area * aspect)))))
        h = int(min(hi, max(lo, round(math.sqrt(area / aspect)))))
        levels = int(rng.integers(1, 7))
        kind = "cdf97" if rng.random() < frac97 else "int53"
        out.append(dict(t=t, w=w, h=h, levels=levels, kind=kind))
    return out
