/*
 * Oracle for the multi-level 2-D DWT -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow CPU code that states the transform the way the paper defines
 * it: separable 1-D lifting (Sec. 2.2, the factorisation of M into K
 * predict/update pairs and a scaling step), the 2-D transform as the tensor
 * product of 1-D transforms (Sec. 2.2, last paragraph), and the multi-level
 * pyramid applied to LL (Sec. 1).  Floating point is FP64; the reversible
 * 5/3 is exact int64 with an int32 range check.  No blocking, fusion or
 * reordering: every line is transformed on its own, in the order stated.
 *
 * Only tests/, __graft_entry__.smoke() and the benchmark's CPU-baseline leg
 * may load this; the CUDA library never does.  See dwt_oracle.h for the
 * readings taken where the paper is silent.
 */
#include "dwt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

long oracle_mirror(long i, long n) {
  /* Whole-sample symmetric extension: ... x2 x1 | x0 x1 ... x(n-1) | x(n-2) ...
   * repeated as often as needed (period 2(n-1)). */
  if (n <= 1) return 0;
  long period = 2 * (n - 1);
  i %= period;
  if (i < 0) i += period;
  if (i >= n) i = period - i;
  return i;
}

/* ------------------------------------------------------------------ */
/* Lifting coefficients (Sec. 5).                                      */
/* ------------------------------------------------------------------ */

/* One unscaled forward lifting pass of a 9/7-shaped transform with the given
 * constants, on an interleaved line of length n, mirrored reads. */
static void lift97_unscaled(const double c[4], double* t, long n) {
  for (int k = 0; k < 2; ++k) {
    double p = c[2 * k], u = c[2 * k + 1];
    for (long i = 1; i < n; i += 2)
      t[i] += p * (t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)]);
    for (long i = 0; i < n; i += 2)
      t[i] += u * (t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)]);
  }
}

/* Impulse responses of the unscaled analysis filters of the 9/7 lifting:
 * h[k+4] for k=-4..4 (low-pass, centred on an even sample) and g[k+3] for
 * k=-3..3 (high-pass, centred on an odd sample). */
static void filters97(const double c[4], double h[9], double g[7]) {
  enum { N = 41, C = 20 };
  double t[N];
  for (int k = -4; k <= 4; ++k) {
    memset(t, 0, sizeof t);
    t[C + k] = 1.0;
    lift97_unscaled(c, t, N);
    h[k + 4] = t[C];
  }
  for (int k = -3; k <= 3; ++k) {
    memset(t, 0, sizeof t);
    t[C + 1 + k] = 1.0;
    lift97_unscaled(c, t, N);
    g[k + 3] = t[C + 1];
  }
}

/* The four conditions that fix the 9/7 constants: the analysis high-pass has
 * vanishing moments 0 and 2 (odd ones vanish by symmetry), and the analysis
 * low-pass has vanishing alternating moments 0 and 2 (zeros at z = -1). */
static void residual97(const double c[4], double f[4]) {
  double h[9], g[7];
  filters97(c, h, g);
  f[0] = f[1] = f[2] = f[3] = 0.0;
  for (int k = -3; k <= 3; ++k) {
    f[0] += g[k + 3];
    f[1] += g[k + 3] * k * k;
  }
  for (int k = -4; k <= 4; ++k) {
    double s = (k & 1) ? -1.0 : 1.0;
    f[2] += s * h[k + 4];
    f[3] += s * h[k + 4] * k * k;
  }
}

static int solve4(double a[4][4], double b[4], double x[4]) {
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (fabs(a[piv][col]) < 1e-300) return -1;
    if (piv != col) {
      for (int j = 0; j < 4; ++j) {
        double tmp = a[col][j];
        a[col][j] = a[piv][j];
        a[piv][j] = tmp;
      }
      double tb = b[col];
      b[col] = b[piv];
      b[piv] = tb;
    }
    for (int r = col + 1; r < 4; ++r) {
      double f = a[r][col] / a[col][col];
      for (int j = col; j < 4; ++j) a[r][j] -= f * a[col][j];
      b[r] -= f * b[col];
    }
  }
  for (int r = 3; r >= 0; --r) {
    double s = b[r];
    for (int j = r + 1; j < 4; ++j) s -= a[r][j] * x[j];
    x[r] = s / a[r][r];
  }
  return 0;
}

double oracle_cdf97_constants(double out[5]) {
  static int done = 0;
  static double cached[5], cached_res;
  if (!done) {
    double c[4] = {-1.58, -0.05, 0.88, 0.44}; /* starting point near the root */
    double f[4];
    for (int it = 0; it < 60; ++it) {
      residual97(c, f);
      double jac[4][4];
      for (int j = 0; j < 4; ++j) {
        double step = 1e-6, cp[4], cm[4], fp[4], fm[4];
        memcpy(cp, c, sizeof cp);
        memcpy(cm, c, sizeof cm);
        cp[j] += step;
        cm[j] -= step;
        residual97(cp, fp);
        residual97(cm, fm);
        for (int i = 0; i < 4; ++i) jac[i][j] = (fp[i] - fm[i]) / (2 * step);
      }
      double rhs[4] = {-f[0], -f[1], -f[2], -f[3]}, dx[4];
      if (solve4(jac, rhs, dx) != 0) break;
      for (int j = 0; j < 4; ++j) c[j] += dx[j];
    }
    residual97(c, f);
    double h[9], g[7], dc = 0.0;
    filters97(c, h, g);
    for (int k = 0; k < 9; ++k) dc += h[k];
    for (int j = 0; j < 4; ++j) cached[j] = c[j];
    cached[4] = dc;
    cached_res = fabs(f[0]) + fabs(f[1]) + fabs(f[2]) + fabs(f[3]);
    done = 1;
  }
  memcpy(out, cached, 5 * sizeof(double));
  return cached_res;
}

int oracle_lifting(int wavelet, double pred1[2], double pred3[2],
                   double upd1[2], double upd3[2], double* scale_lo,
                   double* scale_hi, int norm) {
  int K;
  double dc; /* DC gain of the unscaled analysis low-pass */
  pred3[0] = pred3[1] = upd3[0] = upd3[1] = 0.0;
  pred1[1] = upd1[1] = 0.0;
  switch (wavelet) {
    case ORACLE_CDF53: /* P = -1/2(1+z^-1), U = 1/4(1+z) */
      K = 1;
      pred1[0] = -0.5;
      upd1[0] = 0.25;
      dc = 1.0;
      break;
    case ORACLE_CDF97: {
      double c[5];
      oracle_cdf97_constants(c);
      K = 2;
      pred1[0] = c[0];
      upd1[0] = c[1];
      pred1[1] = c[2];
      upd1[1] = c[3];
      dc = c[4];
      break;
    }
    case ORACLE_DD137: /* P = 1/16(z+z^-2) - 9/16(1+z^-1); U = 9/32(1+z) - 1/32(z^-1+z^2) */
      K = 1;
      pred1[0] = -9.0 / 16.0;
      pred3[0] = 1.0 / 16.0;
      upd1[0] = 9.0 / 32.0;
      upd3[0] = -1.0 / 32.0;
      dc = 1.0;
      break;
    default:
      return -1;
  }
  if (norm == ORACLE_NORM_ZETA) {
    double zeta = sqrt(2.0) / dc; /* 5/3: zeta = sqrt(2) (Sec. 5) */
    *scale_lo = zeta;
    *scale_hi = 1.0 / zeta;
  } else {
    *scale_lo = 1.0 / dc;
    *scale_hi = dc;
  }
  return K;
}

/* ------------------------------------------------------------------ */
/* 1-D transforms                                                      */
/* ------------------------------------------------------------------ */

int oracle_dwt1_f64(int wavelet, int norm, int inverse, long n, double* x,
                    long stride) {
  double p1[2], p3[2], u1[2], u3[2], slo, shi;
  int K = oracle_lifting(wavelet, p1, p3, u1, u3, &slo, &shi, norm);
  if (K < 0 || n < 1) return -1;
  if (n == 1) return 0; /* a length-1 line is left as it is */
  long nlo = (n + 1) / 2;
  double* t = (double*)malloc(sizeof(double) * n);
  if (!t) return -1;
  if (!inverse) {
    for (long i = 0; i < n; ++i) t[i] = x[i * stride];
    for (int k = 0; k < K; ++k) {
      for (long i = 1; i < n; i += 2) /* predict: odd samples from even */
        t[i] += p1[k] * (t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)]) +
                p3[k] * (t[oracle_mirror(i - 3, n)] + t[oracle_mirror(i + 3, n)]);
      for (long i = 0; i < n; i += 2) /* update: even samples from odd */
        t[i] += u1[k] * (t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)]) +
                u3[k] * (t[oracle_mirror(i - 3, n)] + t[oracle_mirror(i + 3, n)]);
    }
    for (long j = 0; 2 * j < n; ++j) x[j * stride] = t[2 * j] * slo;
    for (long j = 0; 2 * j + 1 < n; ++j) x[(nlo + j) * stride] = t[2 * j + 1] * shi;
  } else {
    for (long j = 0; 2 * j < n; ++j) t[2 * j] = x[j * stride] / slo;
    for (long j = 0; 2 * j + 1 < n; ++j) t[2 * j + 1] = x[(nlo + j) * stride] / shi;
    for (int k = K - 1; k >= 0; --k) {
      for (long i = 0; i < n; i += 2)
        t[i] -= u1[k] * (t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)]) +
                u3[k] * (t[oracle_mirror(i - 3, n)] + t[oracle_mirror(i + 3, n)]);
      for (long i = 1; i < n; i += 2)
        t[i] -= p1[k] * (t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)]) +
                p3[k] * (t[oracle_mirror(i - 3, n)] + t[oracle_mirror(i + 3, n)]);
    }
    for (long i = 0; i < n; ++i) x[i * stride] = t[i];
  }
  free(t);
  return 0;
}

static int64_t floor_div(int64_t a, int64_t b) { /* b > 0 */
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}

static int g_range_error;

static int64_t chk(int64_t v) {
  if (v > 2147483647LL || v < -2147483648LL) g_range_error = 1;
  return v;
}

/* JPEG 2000 reversible 5/3:
 *   odd:  y(2n+1) = x(2n+1) - floor((x(2n) + x(2n+2)) / 2)
 *   even: y(2n)   = x(2n)   + floor((y(2n-1) + y(2n+1) + 2) / 4)          */
int oracle_dwt1_i64(int inverse, long n, int64_t* x, long stride) {
  if (n < 1) return -1;
  if (n == 1) return 0;
  long nlo = (n + 1) / 2;
  int64_t* t = (int64_t*)malloc(sizeof(int64_t) * n);
  if (!t) return -1;
  if (!inverse) {
    for (long i = 0; i < n; ++i) t[i] = x[i * stride];
    for (long i = 1; i < n; i += 2)
      t[i] = chk(t[i] - floor_div(chk(t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)]), 2));
    for (long i = 0; i < n; i += 2)
      t[i] = chk(t[i] + floor_div(chk(t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)] + 2), 4));
    for (long j = 0; 2 * j < n; ++j) x[j * stride] = t[2 * j];
    for (long j = 0; 2 * j + 1 < n; ++j) x[(nlo + j) * stride] = t[2 * j + 1];
  } else {
    for (long j = 0; 2 * j < n; ++j) t[2 * j] = x[j * stride];
    for (long j = 0; 2 * j + 1 < n; ++j) t[2 * j + 1] = x[(nlo + j) * stride];
    for (long i = 0; i < n; i += 2)
      t[i] = chk(t[i] - floor_div(chk(t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)] + 2), 4));
    for (long i = 1; i < n; i += 2)
      t[i] = chk(t[i] + floor_div(chk(t[oracle_mirror(i - 1, n)] + t[oracle_mirror(i + 1, n)]), 2));
    for (long i = 0; i < n; ++i) x[i * stride] = t[i];
  }
  free(t);
  return 0;
}

/* ------------------------------------------------------------------ */
/* 2-D multi-level                                                     */
/* ------------------------------------------------------------------ */

int oracle_max_levels(int w, int h) {
  int L = 0;
  while (w > 1 || h > 1) {
    w = (w + 1) / 2;
    h = (h + 1) / 2;
    ++L;
  }
  return L;
}

static int check_args(int w, int h, int levels) {
  if (w < 1 || h < 1 || levels < 0) return -1;
  if (levels > oracle_max_levels(w, h)) return -1;
  return 0;
}

int oracle_dwt2_f64(int wavelet, int norm, int inverse, int w, int h,
                    int levels, const double* in, double* out) {
  if (check_args(w, h, levels) != 0) return -1;
  double p1[2], p3[2], u1[2], u3[2], slo, shi;
  if (oracle_lifting(wavelet, p1, p3, u1, u3, &slo, &shi, norm) < 0) return -1;
  if (out != in) memcpy(out, in, sizeof(double) * (size_t)w * (size_t)h);
  int wk[64], hk[64];
  wk[0] = w;
  hk[0] = h;
  for (int k = 1; k <= levels; ++k) {
    wk[k] = (wk[k - 1] + 1) / 2;
    hk[k] = (hk[k - 1] + 1) / 2;
  }
  if (!inverse) {
    for (int k = 0; k < levels; ++k) {
      for (int c = 0; c < wk[k]; ++c) /* every column, then every row */
        if (oracle_dwt1_f64(wavelet, norm, 0, hk[k], out + c, w)) return -1;
      for (int r = 0; r < hk[k]; ++r)
        if (oracle_dwt1_f64(wavelet, norm, 0, wk[k], out + (size_t)r * w, 1)) return -1;
    }
  } else {
    for (int k = levels - 1; k >= 0; --k) {
      for (int r = 0; r < hk[k]; ++r)
        if (oracle_dwt1_f64(wavelet, norm, 1, wk[k], out + (size_t)r * w, 1)) return -1;
      for (int c = 0; c < wk[k]; ++c)
        if (oracle_dwt1_f64(wavelet, norm, 1, hk[k], out + c, w)) return -1;
    }
  }
  return 0;
}

int oracle_dwt2_i64(int inverse, int w, int h, int levels, const int64_t* in,
                    int64_t* out) {
  if (check_args(w, h, levels) != 0) return -1;
  if (out != in) memcpy(out, in, sizeof(int64_t) * (size_t)w * (size_t)h);
  g_range_error = 0;
  for (size_t i = 0; i < (size_t)w * (size_t)h; ++i) chk(out[i]);
  int wk[64], hk[64];
  wk[0] = w;
  hk[0] = h;
  for (int k = 1; k <= levels; ++k) {
    wk[k] = (wk[k - 1] + 1) / 2;
    hk[k] = (hk[k - 1] + 1) / 2;
  }
  if (!inverse) {
    for (int k = 0; k < levels; ++k) {
      for (int c = 0; c < wk[k]; ++c) oracle_dwt1_i64(0, hk[k], out + c, w);
      for (int r = 0; r < hk[k]; ++r) oracle_dwt1_i64(0, wk[k], out + (size_t)r * w, 1);
    }
  } else {
    for (int k = levels - 1; k >= 0; --k) {
      for (int r = 0; r < hk[k]; ++r) oracle_dwt1_i64(1, wk[k], out + (size_t)r * w, 1);
      for (int c = 0; c < wk[k]; ++c) oracle_dwt1_i64(1, hk[k], out + c, w);
    }
  }
  return g_range_error ? -2 : 0;
}

/* ------------------------------------------------------------------ */
/* Reversible integer non-separable lifting (Iwahashi scheme, CDF 5/3)  */
/* ------------------------------------------------------------------ */

/* Sample (r, c) of a w x h plane with whole-sample symmetric extension; on
 * an axis of length 1 the samples of odd parity do not exist and read 0. */
static int64_t iw_get(const int64_t* t, long w, long h, long r, long c) {
  if ((w == 1 && c != 0) || (h == 1 && r != 0)) return 0;
  return t[oracle_mirror(r, h) * w + oracle_mirror(c, w)];
}

/* Neighbour sums of sample (r, c): horizontal (left + right), vertical
 * (above + below) and diagonal (the four corners). */
static int64_t iw_h(const int64_t* t, long w, long h, long r, long c) {
  return iw_get(t, w, h, r, c - 1) + iw_get(t, w, h, r, c + 1);
}
static int64_t iw_v(const int64_t* t, long w, long h, long r, long c) {
  return iw_get(t, w, h, r - 1, c) + iw_get(t, w, h, r + 1, c);
}
static int64_t iw_d(const int64_t* t, long w, long h, long r, long c) {
  return iw_get(t, w, h, r - 1, c - 1) + iw_get(t, w, h, r - 1, c + 1) + iw_get(t, w, h, r + 1, c - 1) +
         iw_get(t, w, h, r + 1, c + 1);
}

/* The rounded update of one sample in step `step` (0: T, 1: R, 2: S), read
 * from the current plane: the Iwahashi step matrices (Sec. 2.6) with
 * p = -1/2 and u = 1/4, each step's whole update rounded once (half up). */
static int64_t iw_delta(int step, const int64_t* t, long w, long h, long r, long c) {
  const int ro = (int)(r & 1), co = (int)(c & 1);
  if (step == 0) /* T^I_P: HH += p h(LH) + p v(HL) + p^2 d(LL) */
    return floor_div(chk(iw_d(t, w, h, r, c) - 2 * (iw_h(t, w, h, r, c) + iw_v(t, w, h, r, c)) + 2), 4);
  if (step == 1) {
    if (!ro && co) /* R^I, HL += p h(LL) + u v(HH) */
      return floor_div(chk(iw_v(t, w, h, r, c) - 2 * iw_h(t, w, h, r, c) + 2), 4);
    /* R^I, LH += p v(LL) + u h(HH) */
    return floor_div(chk(iw_h(t, w, h, r, c) - 2 * iw_v(t, w, h, r, c) + 2), 4);
  }
  /* S^I_U: LL += u h(HL) + u v(LH) - u^2 d(HH) */
  return floor_div(chk(4 * (iw_h(t, w, h, r, c) + iw_v(t, w, h, r, c)) - iw_d(t, w, h, r, c) + 8), 16);
}

/* Whether sample (r, c) is a target of step `step`: T writes HH (odd,
 * odd), R writes HL (even, odd) and LH (odd, even), S writes LL. */
static int iw_target(int step, long r, long c) {
  const int ro = (int)(r & 1), co = (int)(c & 1);
  if (step == 0) return ro && co;
  if (step == 1) return ro != co;
  return !ro && !co;
}

/* One step on the whole plane: every update is computed from the pre-step
 * plane (a step's targets are not among its sources), then applied. */
static int iw_step(int step, int sign, int64_t* t, long w, long h) {
  int64_t* dlt = (int64_t*)malloc(sizeof(int64_t) * (size_t)w * (size_t)h);
  if (!dlt) return -1;
  for (long r = 0; r < h; ++r)
    for (long c = 0; c < w; ++c)
      dlt[r * w + c] = iw_target(step, r, c) ? iw_delta(step, t, w, h, r, c) : 0;
  for (long i = 0; i < w * h; ++i) t[i] = chk(t[i] + sign * dlt[i]);
  free(dlt);
  return 0;
}

int oracle_dwt2_iwahashi_i64(int inverse, int w, int h, int levels, const int64_t* in, int64_t* out) {
  if (check_args(w, h, levels) != 0) return -1;
  if (out != in) memcpy(out, in, sizeof(int64_t) * (size_t)w * (size_t)h);
  g_range_error = 0;
  for (size_t i = 0; i < (size_t)w * (size_t)h; ++i) chk(out[i]);
  int wk[64], hk[64];
  wk[0] = w;
  hk[0] = h;
  for (int k = 1; k <= levels; ++k) {
    wk[k] = (wk[k - 1] + 1) / 2;
    hk[k] = (hk[k - 1] + 1) / 2;
  }
  int64_t* t = (int64_t*)malloc(sizeof(int64_t) * (size_t)w * (size_t)h);
  if (!t) return -1;
  for (int s = 0; s < levels; ++s) {
    const int k = inverse ? levels - 1 - s : s;
    const long W = wk[k], H = hk[k], cw = (W + 1) / 2, ch = (H + 1) / 2;
    if (!inverse) {
      for (long r = 0; r < H; ++r)
        for (long c = 0; c < W; ++c) t[r * W + c] = out[r * (size_t)w + c];
      for (int step = 0; step < 3; ++step)
        if (iw_step(step, 1, t, W, H)) return -1;
      /* Mallat packing: even rows / columns to the low halves */
      for (long r = 0; r < H; ++r)
        for (long c = 0; c < W; ++c)
          out[((r & 1) ? ch + r / 2 : r / 2) * (size_t)w + ((c & 1) ? cw + c / 2 : c / 2)] = t[r * W + c];
    } else {
      for (long r = 0; r < H; ++r)
        for (long c = 0; c < W; ++c)
          t[r * W + c] = out[((r & 1) ? ch + r / 2 : r / 2) * (size_t)w + ((c & 1) ? cw + c / 2 : c / 2)];
      for (int step = 2; step >= 0; --step)
        if (iw_step(step, -1, t, W, H)) return -1;
      for (long r = 0; r < H; ++r)
        for (long c = 0; c < W; ++c) out[r * (size_t)w + c] = t[r * W + c];
    }
  }
  free(t);
  return g_range_error ? -2 : 0;
}
