/*
 * Oracle for the multi-level 2-D discrete wavelet transform.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct CPU
 * restatement of what the paper's transform computes.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may call it; the
 * product path (the CUDA library) never links or calls anything here.
 *
 * What it computes (paper, Sec. 2.1-2.2 and Sec. 5):
 *   - one level = the separable 2-D transform: the 1-D lifting transform
 *     (K predict/update pairs followed by the scaling step, Sec. 2.2 Eq. of M)
 *     applied to every column, then to every row ("tensor product of 1-D
 *     transforms", Sec. 2.2);
 *   - CDF 5/3: P = -1/2(1+z^-1), U = 1/4(1+z)          (Sec. 5)
 *     CDF 9/7: two pairs (alpha,beta),(gamma,delta)     (Sec. 5)
 *     DD 13/7: degree-3 P and U                         (Sec. 5)
 *   - multi-level: the level is re-applied to the LL band (Sec. 1).
 *
 * Readings where the paper is silent (readings, not statements of the paper):
 *   - whole-sample symmetric (WSS) boundary extension; a length-1 line is
 *     left untouched (no lifting, no scaling);
 *   - H samples are the odd ones and are predicted from both even
 *     neighbours (JPEG 2000 origin convention);
 *   - normalisation: JPEG 2000 (low-pass DC gain 1, high-pass Nyquist gain 2):
 *     9/7 low x 1/K, high x K; 5/3 and DD 13/7 unscaled.  The paper's own
 *     zeta scaling (low x zeta, high x 1/zeta) is available as norm = 1;
 *   - the 9/7 constants, not printed in the paper, are derived here by
 *     Newton's method from the vanishing-moment conditions;
 *   - reversible integer 5/3 (JPEG 2000 floor rounding), per level columns
 *     first then rows; the inverse does rows first then columns;
 *   - Mallat-packed output: LL top-left (ceil(W/2) x ceil(H/2)), HL top-right,
 *     LH bottom-left, HH bottom-right, recursively inside LL.
 */
#ifndef DWT_ORACLE_H
#define DWT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_CDF53 = 0, ORACLE_CDF97 = 1, ORACLE_DD137 = 2 };
enum { ORACLE_NORM_JPEG2000 = 0, ORACLE_NORM_ZETA = 1 };

/* Whole-sample symmetric index for a line of length n >= 1. */
long oracle_mirror(long i, long n);

/* Derive the CDF 9/7 lifting constants (alpha, beta, gamma, delta) and the
 * DC gain K of the unscaled low-pass filter; returns the Newton residual. */
double oracle_cdf97_constants(double out[5]);

/* Lifting coefficients of a wavelet: number of pairs K, and per pair the
 * odd-step (predict) and even-step (update) taps at distance 1 and 3.
 * Returns K, or -1 for an unknown wavelet. */
int oracle_lifting(int wavelet, double pred1[2], double pred3[2],
                   double upd1[2], double upd3[2], double* scale_lo,
                   double* scale_hi, int norm);

/* 1-D transform of one line of length n (n >= 1), stride in elements.
 * Forward output is deinterleaved: ceil(n/2) lows then floor(n/2) highs. */
int oracle_dwt1_f64(int wavelet, int norm, int inverse, long n, double* x,
                    long stride);
int oracle_dwt1_i64(int inverse, long n, int64_t* x, long stride);

/* L-level 2-D transform of a w x h row-major image (pitch = w elements).
 * Forward: in = samples, out = Mallat-packed coefficients.
 * Inverse: in = Mallat-packed coefficients, out = samples.
 * Returns 0 on success, -1 on invalid arguments, -2 (integer only) if an
 * intermediate value leaves the int32 range. */
int oracle_dwt2_f64(int wavelet, int norm, int inverse, int w, int h,
                    int levels, const double* in, double* out);
int oracle_dwt2_i64(int inverse, int w, int h, int levels, const int64_t* in,
                    int64_t* out);

/* Reversible integer non-separable lifting: the Iwahashi scheme (Sec. 2.6)
 * of CDF 5/3 (p = -1/2, u = 1/4) with each step's whole update rounded once,
 * half up -- a different reversible transform from the JPEG 2000 one above
 * (whose every 1-D step rounds on its own).  In sample coordinates, with
 * h, v, d the horizontal, vertical and diagonal neighbour sums (whole-sample
 * symmetric extension; absent samples of a length-1 axis read 0):
 *   T: odd row, odd col    += floor((d - 2 (h + v) + 2) / 4)
 *   R: even row, odd col   += floor((v - 2 h + 2) / 4)
 *      odd row, even col   += floor((h - 2 v + 2) / 4)
 *   S: even row, even col  += floor((4 (h + v) - d + 8) / 16)
 * Each step reads only samples it does not write, so the inverse subtracts
 * the same updates in the order S, R, T.  Mallat packing as above. */
int oracle_dwt2_iwahashi_i64(int inverse, int w, int h, int levels, const int64_t* in, int64_t* out);

/* Largest valid level count: halvings until both dimensions are 1. */
int oracle_max_levels(int w, int h);

#ifdef __cplusplus
}
#endif
#endif
