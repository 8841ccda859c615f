// Lifting steps of the paper as compile-time stencil stages.
//
// A quadruple (n, m) holds the samples of rows 2n..2n+1 and columns
// 2m..2m+1: LL (even, even), HL (even, odd), LH (odd, even), HH (odd, odd)
// (Sec. 2.3).  A lane of a warp holds QL horizontally adjacent quadruples
// (QL*l .. QL*l + QL-1 relative to the warp's first quad), so a horizontal
// neighbour at distance <= QL is either in the lane or one shuffle away.
// Vertical neighbours come from the stage's window of rows.
//
// A linear stage is one step matrix of the paper: every target subband
// receives sum(sign * (vertical op (x) horizontal op) applied to a source
// subband), all sources read from the pre-step state (the matrices act on
// the whole vector at once, Sec. 2.4).  The 1-D operators are the predict P
// and update U of Sec. 2.2 / Sec. 5, their scalar split P = P0 + P1,
// U = U0 + U1 (Sec. 4), V = PU + 1 (Sec. 2.3) and the identity.  With P
// placed after L (JPEG 2000 origin) the predict reads quads at offsets
// {0, +1} and the update reads {-1, 0}.
#pragma once

#include <type_traits>

#include "dwt_internal.h"

namespace dwt {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B <= E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
template <class... A>
__host__ __device__ constexpr int vmax(int a, A... b) {
  int r = a;
  ((r = b > r ? b : r), ...);
  return r;
}
template <class... A>
__host__ __device__ constexpr int vmin(int a, A... b) {
  int r = a;
  ((r = b < r ? b : r), ...);
  return r;
}

enum Sub : int { LL = 0, HL = 1, LH = 2, HH = 3 };

template <typename V, int QL>
struct Row {
  V s[4][QL];
};

// The value of the quad at position P, where 0..QL-1 are this lane's quads,
// negative positions the previous lanes' and QL.. the next lanes' (one or
// two lanes away).
template <int P, typename V, int QL>
__device__ __forceinline__ V hpos(const V (&x)[QL]) {
  static_assert(P >= -2 * QL && P < 3 * QL, "horizontal reach beyond two lanes");
  if constexpr (P >= 0 && P < QL) return x[P];
  else if constexpr (P >= -QL && P < 0) return __shfl_up_sync(kFull, x[QL + P], 1);
  else if constexpr (P < 0) return __shfl_up_sync(kFull, x[2 * QL + P], 2);
  else if constexpr (P < 2 * QL) return __shfl_down_sync(kFull, x[P - QL], 1);
  else return __shfl_down_sync(kFull, x[P - 2 * QL], 2);
}

// ---------------------------------------------------------------------------
// Where a stage reads its inputs.  A stage evaluates one lane's QL quads;
// it asks its accessor for subband S of the quad DY rows below and DX
// columns right of the lane's quad J (all compile-time), and starts from
// the lane's own pre-step values `own`.  WinAcc serves the streaming
// kernels: vertical neighbours from the stage's window of rows (row UP is
// the lane's own), horizontal ones by warp shuffles.  The tile kernels use
// an accessor into a shared-memory plane (tile_kernel.cuh).  Both evaluate
// every stage with the same arithmetic in the same order.
// ---------------------------------------------------------------------------
template <typename V, int QL, int UP>
struct WinAcc {
  const Row<V, QL>* w;
  template <int S, int DY, int DX, int J>
  __device__ __forceinline__ V at() const {
    return hpos<J + DX>(w[UP + DY].s[S]);
  }
};

// ---------------------------------------------------------------------------
// 1-D operators
// ---------------------------------------------------------------------------
enum Op : int { OP_I, OP_P, OP_U, OP_P0, OP_P1, OP_U0, OP_U1, OP_V, OP_V1 };

// Degree-1 lifting (CDF 5/3 and 9/7): P = p(1 + z), U = u(1 + z^-1) in the
// quad-offset convention above.  Degree 3 (DD 13/7): P has taps p1 at 0, +1
// and p3 at -1, +2; U has u1 at -1, 0 and u3 at -2, +1.  V = PU + 1 (the
// Polyphase scheme's diagonal operator, Sec. 2.3) spans -1..1 for degree 1
// and -3..3 for degree 3; V1 = P1 U1 + 1 (Polyphase*) is the single tap
// 1 + pu for degree 1 and spans -3..3 for degree 3.
template <int DEG, int OP>
struct OpShape {
  static constexpr int lo = (OP == OP_I || OP == OP_P0 || OP == OP_U0) ? 0
                            : (OP == OP_V1) ? (DEG == 1 ? 0 : -3)
                            : (OP == OP_P)  ? (DEG == 1 ? 0 : -1)
                            : (OP == OP_P1) ? (DEG == 1 ? 1 : -1)
                            : (OP == OP_U)  ? (DEG == 1 ? -1 : -2)
                            : (OP == OP_U1) ? (DEG == 1 ? -1 : -2)
                                            : (DEG == 1 ? -1 : -3);  // OP_V
  static constexpr int hi = (OP == OP_I || OP == OP_P0 || OP == OP_U0) ? 0
                            : (OP == OP_V1) ? (DEG == 1 ? 0 : 3)
                            : (OP == OP_P)  ? (DEG == 1 ? 1 : 2)
                            : (OP == OP_P1) ? (DEG == 1 ? 1 : 2)
                            : (OP == OP_U)  ? (DEG == 1 ? 0 : 1)
                            : (OP == OP_U1) ? (DEG == 1 ? -1 : 1)
                                            : (DEG == 1 ? 1 : 3);  // OP_V
  // The split operators P1, U1 of degree 3 have a zero tap at offset 0.
  __host__ __device__ static constexpr bool has(int off) {
    return !((OP == OP_P1 || OP == OP_U1) && DEG == 3 && off == 0);
  }
  // Taps with equal coefficients form a class: P and U have one class of
  // two taps (degree 1) or two classes (degree 3: distance 1 and 3); V has
  // its centre 1 + 2pu and the pair pu (degree 1) or one class per
  // distance 0..3 (degree 3); V1 of degree 3 has {0}, {-3, 3}, {-2, 1} and
  // {-1, 2} (P1 U1 is not symmetric).  Class 0 holds the centre tap when the
  // operator has one.
  __host__ __device__ static constexpr int cls(int off) {
    return OP == OP_V ? (DEG == 1 ? (off == 0 ? 0 : 1) : (off < 0 ? -off : off))
           : OP == OP_V1 ? (DEG == 1 ? 0
                                     : off == 0 ? 0 : (off == 3 || off == -3) ? 1 : (off == -2 || off == 1) ? 2 : 3)
           : (DEG == 3 && (OP == OP_P || OP == OP_P1)) ? ((off == 0 || off == 1) ? 0 : 1)
           : (DEG == 3 && (OP == OP_U || OP == OP_U1)) ? ((off == -1 || off == 0) ? 0 : 1)
                                                       : 0;
  }
  static constexpr int NCLS = OP == OP_V ? (DEG == 1 ? 2 : 4)
                              : OP == OP_V1 ? (DEG == 1 ? 1 : 4)
                              : (DEG == 3 && (OP == OP_P || OP == OP_P1 || OP == OP_U || OP == OP_U1)) ? 2
                                                                                                       : 1;
  // a representative offset of each class (for its coefficient)
  __host__ __device__ static constexpr int rep(int c) {
    return OP == OP_V ? (DEG == 1 ? (c == 0 ? 0 : 1) : c)
           : OP == OP_V1 ? (DEG == 1 ? 0 : c == 0 ? 0 : c == 1 ? 3 : c == 2 ? 1 : 2)
           : (DEG == 3 && (OP == OP_P || OP == OP_P1)) ? (c == 0 ? 1 : 2)
           : (DEG == 3 && (OP == OP_U || OP == OP_U1)) ? (c == 0 ? -1 : 1)
                                                       : lo;
  }
};

// ---------------------------------------------------------------------------
// Coefficient sources.  RtCoefs reads a Coefs structure (kernel parameter or
// batch descriptor): any normalisation, and zero taps / unit scales on an
// axis of length 1.  StCoefs<WL, INV> holds the wavelet's constants with
// JPEG 2000 normalisation and both axes longer than one sample as
// compile-time values, which the compiler folds into the instructions
// (no registers, no loads).  Both give bit-identical coefficients: the
// same literals rounded the same way as the host's coefficient tables.
// ---------------------------------------------------------------------------
struct RtCoefs {
  const Coefs& c;
  __device__ __forceinline__ float p1(int k, int axis) const { return axis ? c.ph1[k] : c.pv1[k]; }
  __device__ __forceinline__ float p3(int k, int axis) const { return axis ? c.ph3[k] : c.pv3[k]; }
  __device__ __forceinline__ float u1(int k, int axis) const { return axis ? c.uh1[k] : c.uv1[k]; }
  __device__ __forceinline__ float u3(int k, int axis) const { return axis ? c.uh3[k] : c.uv3[k]; }
  __device__ __forceinline__ float scale(int s) const { return c.scale[s]; }
  __device__ __forceinline__ bool v_on() const { return c.v_on != 0; }
  __device__ __forceinline__ bool h_on() const { return c.h_on != 0; }
};

template <int WL, bool INV>
struct StCoefs {
  __host__ __device__ constexpr float p1(int k, int) const {
    return WL == W97 ? float(k == 0 ? kAlpha : kGamma) : WL == W53 ? -0.5f : float(-9.0 / 16.0);
  }
  __host__ __device__ constexpr float p3(int, int) const { return WL == WDD ? float(1.0 / 16.0) : 0.0f; }
  __host__ __device__ constexpr float u1(int k, int) const {
    return WL == W97 ? float(k == 0 ? kBeta : kDelta) : WL == W53 ? 0.25f : float(9.0 / 32.0);
  }
  __host__ __device__ constexpr float u3(int, int) const { return WL == WDD ? float(-1.0 / 32.0) : 0.0f; }
  // JPEG 2000 band gains: low x 1/K, high x K per axis (K = 1 but for 9/7);
  // s = LL, HL, LH, HH; the inverse divides
  __host__ __device__ constexpr float scale(int s) const {
    const double lo = WL == W97 ? 1.0 / kK97 : 1.0, hi = WL == W97 ? kK97 : 1.0;
    const double v = ((s & 2) ? hi : lo) * ((s & 1) ? hi : lo);
    return float(INV ? 1.0 / v : v);
  }
  __host__ __device__ constexpr bool v_on() const { return true; }
  __host__ __device__ constexpr bool h_on() const { return true; }
};

// Configuration tag of a kernel that reads its coefficients at run time.
struct RtTag {};

template <class SRC>
struct CoefSource {
  __device__ __forceinline__ static SRC make(const Coefs&) { return SRC{}; }
};
template <>
struct CoefSource<RtTag> {
  __device__ __forceinline__ static RtCoefs make(const Coefs& c) { return RtCoefs{c}; }
};

// Coefficient of operator OP (pair K, axis: 0 vertical, 1 horizontal) at
// quad offset OFF.
template <int DEG, int OP, int K, int AXIS, int OFF, class CS>
__device__ __forceinline__ float op_tap(const CS& c) {
  const float p1 = c.p1(K, AXIS);
  const float u1 = c.u1(K, AXIS);
  if constexpr (OP == OP_I) {
    return 1.0f;
  } else if constexpr (OP == OP_P || OP == OP_P1) {
    if constexpr (DEG == 1) return p1;
    else return (OFF == 0 || OFF == 1) ? p1 : c.p3(K, AXIS);
  } else if constexpr (OP == OP_P0) {
    return p1;
  } else if constexpr (OP == OP_U || OP == OP_U1) {
    if constexpr (DEG == 1) return u1;
    else return (OFF == -1 || OFF == 0) ? u1 : c.u3(K, AXIS);
  } else if constexpr (OP == OP_U0) {
    return u1;
  } else if constexpr (OP == OP_V) {
    // V = PU + 1, the convolution of the taps above plus one at the centre.
    // Rounded products and sums (no contraction into an FMA), so that every
    // kernel folds the same coefficient whatever its inlining context.
    if constexpr (DEG == 1) {  // pu z^-1 + (1 + 2pu) + pu z
      return OFF == 0 ? __fadd_rn(1.0f, __fmul_rn(__fmul_rn(2.0f, p1), u1)) : __fmul_rn(p1, u1);
    } else {  // distance 0: 1 + 2 p1 u1 + 2 p3 u3; 1: p1 u1 + p1 u3 + p3 u1; 2: p1 u3 + p3 u1; 3: p3 u3
      const float p3 = c.p3(K, AXIS), u3 = c.u3(K, AXIS);
      if constexpr (OFF == 0)
        return __fadd_rn(1.0f, __fadd_rn(__fmul_rn(__fmul_rn(2.0f, p1), u1), __fmul_rn(__fmul_rn(2.0f, p3), u3)));
      else if constexpr (OFF == 1)
        return __fadd_rn(__fadd_rn(__fmul_rn(p1, u1), __fmul_rn(p1, u3)), __fmul_rn(p3, u1));
      else if constexpr (OFF == 2)
        return __fadd_rn(__fmul_rn(p1, u3), __fmul_rn(p3, u1));
      else
        return __fmul_rn(p3, u3);
    }
  } else {  // OP_V1 = P1 U1 + 1
    if constexpr (DEG == 1) {  // 1 + pu
      return __fadd_rn(1.0f, __fmul_rn(p1, u1));
    } else {  // 0: 1 + p1 u1 + 2 p3 u3; +-3: p3 u3; -2, 1: p3 u1; -1, 2: p1 u3
      const float p3 = c.p3(K, AXIS), u3 = c.u3(K, AXIS);
      if constexpr (OFF == 0)
        return __fadd_rn(1.0f, __fadd_rn(__fmul_rn(p1, u1), __fmul_rn(__fmul_rn(2.0f, p3), u3)));
      else if constexpr (OFF == 3 || OFF == -3)
        return __fmul_rn(p3, u3);
      else if constexpr (OFF == -2 || OFF == 1)
        return __fmul_rn(p3, u1);
      else
        return __fmul_rn(p1, u3);
    }
  }
}

// ---------------------------------------------------------------------------
// Linear stages (one step matrix)
// ---------------------------------------------------------------------------
template <int TGT, int SRC, int VOP, int HOP, int SGN = 1>
struct Term {
  static constexpr int tgt = TGT, src = SRC, vop = VOP, hop = HOP, sgn = SGN;
};

template <int DEG, int K, bool REPLACE, class... Ts>
struct Lin {
  static constexpr int UP = -vmin(0, OpShape<DEG, Ts::vop>::lo...);
  static constexpr int DOWN = vmax(0, OpShape<DEG, Ts::vop>::hi...);
  static constexpr int LEFT = -vmin(0, OpShape<DEG, Ts::hop>::lo...);
  static constexpr int RIGHT = vmax(0, OpShape<DEG, Ts::hop>::hi...);
  static constexpr unsigned TARGETS = (0u | ... | (1u << Ts::tgt));

  // One term.  Taps of equal coefficient are summed first and multiplied
  // once (P x = p (x0 + x1), P P* x = p^2 (sum of four), ...): fewer
  // roundings at the magnitude of the target than one FMA per tap.  The
  // class holding the centre tap, whose coefficient is the largest in the
  // products of V, is accumulated in the second pass, after all others.
  // Subbands this step reads at another quad's position (published by the
  // tile kernels before the step): sources of terms that reach beyond the
  // quad itself.  A step with none is local and needs no barrier.
  static constexpr unsigned NEIGHBOUR_SRCS =
      (0u | ... | ((OpShape<DEG, Ts::vop>::lo < 0 || OpShape<DEG, Ts::vop>::hi > 0 ||
                    OpShape<DEG, Ts::hop>::lo < 0 || OpShape<DEG, Ts::hop>::hi > 0)
                       ? (1u << Ts::src)
                       : 0u));

  template <class T, bool CENTRE_PASS, int QL, class A, class CS>
  __device__ __forceinline__ static void term(const A& acc, Row<float, QL>& o, const CS& c) {
    using VS = OpShape<DEG, T::vop>;
    using HS = OpShape<DEG, T::hop>;
    static_for<0, VS::NCLS - 1>([&](auto cvi) {
      constexpr int CV = decltype(cvi)::value;
      static_for<0, HS::NCLS - 1>([&](auto chi) {
        constexpr int CH = decltype(chi)::value;
        constexpr bool centre = VS::has(0) && HS::has(0) && VS::cls(0) == CV && HS::cls(0) == CH &&
                                VS::lo <= 0 && VS::hi >= 0 && HS::lo <= 0 && HS::hi >= 0;
        if constexpr (centre == CENTRE_PASS) {
          float s[QL];
#pragma unroll
          for (int j = 0; j < QL; ++j) s[j] = 0.0f;  // overwritten by the first tap
          bool first = true;
          static_for<VS::lo, VS::hi>([&](auto dy) {
            constexpr int DY = decltype(dy)::value;
            if constexpr (VS::has(DY) && VS::cls(DY) == CV) {
              static_for<HS::lo, HS::hi>([&](auto dx) {
                constexpr int DX = decltype(dx)::value;
                if constexpr (HS::has(DX) && HS::cls(DX) == CH) {
                  static_for<0, QL - 1>([&](auto jj) {
                    constexpr int J = decltype(jj)::value;
                    const float v = acc.template at<T::src, DY, DX, J>();
                    s[J] = first ? v : s[J] + v;
                  });
                  first = false;
                }
              });
            }
          });
          const float cf = (T::sgn > 0 ? 1.0f : -1.0f) * op_tap<DEG, T::vop, K, 0, VS::rep(CV), CS>(c) *
                           op_tap<DEG, T::hop, K, 1, HS::rep(CH), CS>(c);
#pragma unroll
          for (int j = 0; j < QL; ++j) o.s[T::tgt][j] = fmaf(cf, s[j], o.s[T::tgt][j]);
        }
      });
    });
  }

  template <int QL, class A, class CS>
  __device__ __forceinline__ static void eval(const Row<float, QL>& own, const A& acc, Row<float, QL>& o,
                                              const CS& c, const ConvTaps&) {
    o = own;
    if constexpr (REPLACE) {
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (TARGETS & (1u << s))
#pragma unroll
          for (int j = 0; j < QL; ++j) o.s[s][j] = 0.0f;
    }
    (term<Ts, false, QL>(acc, o, c), ...);
    (term<Ts, true, QL>(acc, o, c), ...);
  }
};

// Scaling step (Sec. 2.2, the diagonal matrix of M): per-subband factors.
struct Scale {
  static constexpr int UP = 0, DOWN = 0, LEFT = 0, RIGHT = 0;
  static constexpr unsigned NEIGHBOUR_SRCS = 0;
  template <int QL, class A, class CS>
  __device__ __forceinline__ static void eval(const Row<float, QL>& own, const A&, Row<float, QL>& o,
                                              const CS& c, const ConvTaps&) {
    // a rounded product: never contracted into the next step's sums (which
    // would make the result depend on how a kernel passes values between
    // steps, in registers or through shared memory)
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int j = 0; j < QL; ++j) o.s[s][j] = __fmul_rn(own.s[s][j], c.scale(s));
  }
};

// ---------------------------------------------------------------------------
// Convolution scheme (Sec. 2.3): each output polyphase component is a 2-D
// FIR of the four input components; the taps (scaling folded in) are the
// products of the 1-D polyphase entries of the whole factorisation, indexed
// [out row][out col][in row][in col][dy][dx].
// ---------------------------------------------------------------------------
template <int WL, bool INV>
struct ConvShape {
  // [out][in] ranges of the 1-D polyphase entries (quad offsets).  DD 13/7:
  // forward L <- even 1 + UP (-3..3), L <- odd U (-2..1), H <- even P
  // (-1..2), H <- odd 1; inverse even <- L 1, even <- H U, odd <- L P,
  // odd <- H 1 + PU.
  __host__ __device__ static constexpr int lo(int o, int i) {
    return WL == W53 ? (!INV ? (o == 0 ? -1 : 0) : (i == 0 ? 0 : -1))
           : WL == W97 ? (!INV ? (o == 0 ? -2 : -1) : (i == 0 ? -1 : -2))
                       : (!INV ? (o == 0 ? (i == 0 ? -3 : -2) : (i == 0 ? -1 : 0))
                               : (o == 0 ? (i == 0 ? 0 : -2) : (i == 0 ? -1 : -3)));
  }
  __host__ __device__ static constexpr int hi(int o, int i) {
    return WL == W53 ? (!INV ? (o == 0 ? (i == 0 ? 1 : 0) : (i == 0 ? 1 : 0))
                             : (o == 0 ? 0 : (i == 0 ? 1 : 1)))
           : WL == W97 ? (!INV ? (o == 0 ? (i == 0 ? 2 : 1) : (i == 0 ? 2 : 1))
                               : (o == 0 ? 1 : 2))
                       : (!INV ? (o == 0 ? (i == 0 ? 3 : 1) : (i == 0 ? 2 : 0))
                               : (o == 0 ? (i == 0 ? 0 : 1) : (i == 0 ? 2 : 3)));
  }
};

// The 1-D polyphase matrix of the whole factorisation (rows: outputs,
// columns: inputs, Laurent polynomials in the quad offset -4..4), computed
// at compile time from the lifting constants with JPEG 2000 normalisation:
// forward (L, H) <- (even, odd), H += P L and L += U H per pair, then the
// band gains; inverse (even, odd) <- (L, H), the steps undone in reverse
// order.  The same arithmetic in the same order as the host's tap table
// for the runtime path.
struct ConvPoly {
  double c[9];
};
struct ConvMat {
  ConvPoly m[2][2];
};
__host__ __device__ constexpr ConvPoly conv_pmul(const ConvPoly& a, const ConvPoly& b) {
  ConvPoly r{};
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) {
      const int k = i + j - 4;
      if (a.c[i] != 0 && b.c[j] != 0 && k >= 0 && k < 9) r.c[k] += a.c[i] * b.c[j];
    }
  return r;
}
__host__ __device__ constexpr void conv_padd(ConvPoly& a, const ConvPoly& b, double s) {
  for (int i = 0; i < 9; ++i) a.c[i] += s * b.c[i];
}
template <int WL, bool INV>
__host__ __device__ constexpr ConvMat conv_matrix() {
  const int npairs = WL == W97 ? 2 : 1;
  const double p1[2] = {WL == W97 ? kAlpha : WL == W53 ? -0.5 : -9.0 / 16.0, kGamma};
  const double u1[2] = {WL == W97 ? kBeta : WL == W53 ? 0.25 : 9.0 / 32.0, kDelta};
  const double p3 = WL == WDD ? 1.0 / 16.0 : 0.0, u3 = WL == WDD ? -1.0 / 32.0 : 0.0;
  const double dc = WL == W97 ? kK97 : 1.0;
  const double lo = 1.0 / dc, hi = dc;
  ConvMat r{};
  if (!INV) {
    r.m[0][0].c[4] = r.m[1][1].c[4] = 1.0;
    for (int k = 0; k < npairs; ++k) {
      ConvPoly P{}, U{};
      P.c[4] = P.c[5] = p1[k];
      P.c[3] = P.c[6] = k == 0 ? p3 : 0.0;
      U.c[3] = U.c[4] = u1[k];
      U.c[2] = U.c[5] = k == 0 ? u3 : 0.0;
      for (int j = 0; j < 2; ++j) conv_padd(r.m[1][j], conv_pmul(P, r.m[0][j]), 1.0);
      for (int j = 0; j < 2; ++j) conv_padd(r.m[0][j], conv_pmul(U, r.m[1][j]), 1.0);
    }
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 9; ++i) {
        r.m[0][j].c[i] *= lo;
        r.m[1][j].c[i] *= hi;
      }
  } else {
    r.m[0][0].c[4] = 1.0 / lo;
    r.m[1][1].c[4] = 1.0 / hi;
    for (int k = npairs - 1; k >= 0; --k) {
      ConvPoly P{}, U{};
      P.c[4] = P.c[5] = p1[k];
      P.c[3] = P.c[6] = k == 0 ? p3 : 0.0;
      U.c[3] = U.c[4] = u1[k];
      U.c[2] = U.c[5] = k == 0 ? u3 : 0.0;
      for (int j = 0; j < 2; ++j) conv_padd(r.m[0][j], conv_pmul(U, r.m[1][j]), -1.0);
      for (int j = 0; j < 2; ++j) conv_padd(r.m[1][j], conv_pmul(P, r.m[0][j]), -1.0);
    }
  }
  return r;
}
template <int WL, bool INV>
struct ConvStatic {
  static constexpr ConvMat M = conv_matrix<WL, INV>();
  // tap of output (SO, SX) from input (TI, TX) at quad offset (DY, DX)
  template <int SO, int SX, int TI, int TX, int DY, int DX>
  __device__ __forceinline__ static constexpr float tap() {
    return float(M.m[SO][TI].c[DY + 4] * M.m[SX][TX].c[DX + 4]);
  }
};

template <class CS>
struct IsStaticCoefs : std::false_type {};
template <int WL, bool INV>
struct IsStaticCoefs<StCoefs<WL, INV>> : std::true_type {};

template <int WL, bool INV>
struct Conv {
  using S = ConvShape<WL, INV>;
  static constexpr int UP = -cmin(cmin(S::lo(0, 0), S::lo(0, 1)), cmin(S::lo(1, 0), S::lo(1, 1)));
  static constexpr int DOWN = cmax(cmax(S::hi(0, 0), S::hi(0, 1)), cmax(S::hi(1, 0), S::hi(1, 1)));
  static constexpr int LEFT = UP, RIGHT = DOWN;
  static constexpr unsigned NEIGHBOUR_SRCS = 15u;

  template <int QL, class A, class CS>
  __device__ __forceinline__ static void eval(const Row<float, QL>&, const A& acc, Row<float, QL>& o,
                                              const CS&, const ConvTaps& t) {
    static_for<0, 3>([&](auto so_sx) {
      constexpr int SO = decltype(so_sx)::value >> 1, SX = decltype(so_sx)::value & 1;
      float sum[QL];
#pragma unroll
      for (int j = 0; j < QL; ++j) sum[j] = 0.0f;
      static_for<0, 3>([&](auto ti_tx) {
        constexpr int TI = decltype(ti_tx)::value >> 1, TX = decltype(ti_tx)::value & 1;
        static_for<S::lo(SO, TI), S::hi(SO, TI)>([&](auto dy) {
          constexpr int DY = decltype(dy)::value;
          static_for<S::lo(SX, TX), S::hi(SX, TX)>([&](auto dx) {
            constexpr int DX = decltype(dx)::value;
            // compile-time taps for levels with static coefficients
            // (JPEG 2000 normalisation, both sides >= 2), else the table
            float cf;
            if constexpr (IsStaticCoefs<CS>::value) {
              constexpr float k = ConvStatic<WL, INV>::template tap<SO, SX, TI, TX, DY, DX>();
              cf = k;
            } else {
              cf = t.t[SO][SX][TI][TX][DY + kConvReach][DX + kConvReach];
            }
            static_for<0, QL - 1>([&](auto jj) {
              constexpr int J = decltype(jj)::value;
              sum[J] = fmaf(cf, acc.template at<2 * TI + TX, DY, DX, J>(), sum[J]);
            });
          });
        });
      });
#pragma unroll
      for (int j = 0; j < QL; ++j) o.s[2 * SO + SX][j] = sum[j];
    });
  }
};

// ---------------------------------------------------------------------------
// Reversible integer 5/3, JPEG 2000 floor rounding, separable order:
// vertical predict, vertical update, horizontal predict, horizontal update.
// ---------------------------------------------------------------------------
template <int KIND, bool INV>
struct Int53 {
  // KIND 0: vertical predict (reads rows n, n+1), 1: vertical update
  // (rows n-1, n), 2: horizontal predict (quads m, m+1), 3: horizontal update.
  static constexpr int UP = KIND == 1 ? 1 : 0;
  static constexpr int DOWN = KIND == 0 ? 1 : 0;
  static constexpr int LEFT = KIND == 3 ? 1 : 0;
  static constexpr int RIGHT = KIND == 2 ? 1 : 0;

  static constexpr unsigned NEIGHBOUR_SRCS = KIND == 0   ? (1u << LL) | (1u << HL)
                                             : KIND == 1 ? (1u << LH) | (1u << HH)
                                             : KIND == 2 ? (1u << LL) | (1u << LH)
                                                         : (1u << HL) | (1u << HH);

  template <int QL, class A, class CS>
  __device__ __forceinline__ static void eval(const Row<int, QL>& own, const A& acc, Row<int, QL>& o,
                                              const CS& c, const ConvTaps&) {
    o = own;
    const int sg = INV ? -1 : 1;
    if constexpr (KIND == 0) {  // odd rows -= floor((even above + even below) / 2)
      if (c.v_on()) {
        static_for<0, QL - 1>([&](auto jj) {
          constexpr int J = decltype(jj)::value;
          o.s[LH][J] -= sg * ((acc.template at<LL, 0, 0, J>() + acc.template at<LL, 1, 0, J>()) >> 1);
          o.s[HH][J] -= sg * ((acc.template at<HL, 0, 0, J>() + acc.template at<HL, 1, 0, J>()) >> 1);
        });
      }
    } else if constexpr (KIND == 1) {  // even rows += floor((odd above + odd below + 2) / 4)
      if (c.v_on()) {
        static_for<0, QL - 1>([&](auto jj) {
          constexpr int J = decltype(jj)::value;
          o.s[LL][J] += sg * ((acc.template at<LH, -1, 0, J>() + acc.template at<LH, 0, 0, J>() + 2) >> 2);
          o.s[HL][J] += sg * ((acc.template at<HH, -1, 0, J>() + acc.template at<HH, 0, 0, J>() + 2) >> 2);
        });
      }
    } else if constexpr (KIND == 2) {  // odd columns from the even ones at m, m+1
      if (c.h_on()) {
        static_for<0, QL - 1>([&](auto jj) {
          constexpr int J = decltype(jj)::value;
          o.s[HL][J] -= sg * ((acc.template at<LL, 0, 0, J>() + acc.template at<LL, 0, 1, J>()) >> 1);
          o.s[HH][J] -= sg * ((acc.template at<LH, 0, 0, J>() + acc.template at<LH, 0, 1, J>()) >> 1);
        });
      }
    } else {  // even columns from the odd ones at m-1, m
      if (c.h_on()) {
        static_for<0, QL - 1>([&](auto jj) {
          constexpr int J = decltype(jj)::value;
          o.s[LL][J] += sg * ((acc.template at<HL, 0, -1, J>() + acc.template at<HL, 0, 0, J>() + 2) >> 2);
          o.s[LH][J] += sg * ((acc.template at<HH, 0, -1, J>() + acc.template at<HH, 0, 0, J>() + 2) >> 2);
        });
      }
    }
  }
};

// ---------------------------------------------------------------------------
// Reversible integer non-separable lifting: the Iwahashi scheme (Sec. 2.6)
// of CDF 5/3 (p = -1/2, u = 1/4) with each step's whole update rounded once,
// half up -- a different reversible transform from the JPEG 2000 one, whose
// 1-D steps round one by one.  Every step reads only subbands it does not
// write, so the inverse subtracts the same updates in reverse order.  On an
// axis of length 1 the absent subbands stay 0: their updates are skipped.
//   KIND 0, T^I_P: HH += (d(LL) - 2 (h(LH) + v(HL)) + 2) >> 2
//   KIND 1, R^I:   HL += (v(HH) - 2 h(LL) + 2) >> 2,  LH += (h(HH) - 2 v(LL) + 2) >> 2
//   KIND 2, S^I_U: LL += (4 (h(HL) + v(LH)) - d(HH) + 8) >> 4
// with h, v, d the horizontal, vertical and diagonal neighbour sums in
// quad offsets of the JPEG 2000 origin (predicts read {0, +1}, updates
// {-1, 0}).
// ---------------------------------------------------------------------------
template <int KIND, bool INV>
struct IntIw {
  static constexpr int UP = KIND == 0 ? 0 : 1;
  static constexpr int DOWN = KIND == 2 ? 0 : 1;
  static constexpr int LEFT = KIND == 0 ? 0 : 1;
  static constexpr int RIGHT = KIND == 2 ? 0 : 1;
  static constexpr unsigned NEIGHBOUR_SRCS = KIND == 0   ? (1u << LL) | (1u << HL) | (1u << LH)
                                             : KIND == 1 ? (1u << LL) | (1u << HH)
                                                         : (1u << HL) | (1u << LH) | (1u << HH);

  template <int QL, class A, class CS>
  __device__ __forceinline__ static void eval(const Row<int, QL>& own, const A& acc, Row<int, QL>& o,
                                              const CS& c, const ConvTaps&) {
    o = own;
    const int sg = INV ? -1 : 1;
    if constexpr (KIND == 0) {
      if (c.h_on() && c.v_on()) {
        static_for<0, QL - 1>([&](auto jj) {
          constexpr int J = decltype(jj)::value;
          const int d = acc.template at<LL, 0, 0, J>() + acc.template at<LL, 0, 1, J>() +
                        acc.template at<LL, 1, 0, J>() + acc.template at<LL, 1, 1, J>();
          const int hv = acc.template at<LH, 0, 0, J>() + acc.template at<LH, 0, 1, J>() +
                         acc.template at<HL, 0, 0, J>() + acc.template at<HL, 1, 0, J>();
          o.s[HH][J] += sg * ((d - 2 * hv + 2) >> 2);
        });
      }
    } else if constexpr (KIND == 1) {
      const bool hon = c.h_on(), von = c.v_on();
      static_for<0, QL - 1>([&](auto jj) {
        constexpr int J = decltype(jj)::value;
        if (hon) {
          const int v = acc.template at<HH, -1, 0, J>() + acc.template at<HH, 0, 0, J>();
          const int hl = acc.template at<LL, 0, 0, J>() + acc.template at<LL, 0, 1, J>();
          o.s[HL][J] += sg * ((v - 2 * hl + 2) >> 2);
        }
        if (von) {
          const int h = acc.template at<HH, 0, -1, J>() + acc.template at<HH, 0, 0, J>();
          const int vl = acc.template at<LL, 0, 0, J>() + acc.template at<LL, 1, 0, J>();
          o.s[LH][J] += sg * ((h - 2 * vl + 2) >> 2);
        }
      });
    } else {
      static_for<0, QL - 1>([&](auto jj) {
        constexpr int J = decltype(jj)::value;
        const int hv = acc.template at<HL, 0, -1, J>() + acc.template at<HL, 0, 0, J>() +
                       acc.template at<LH, -1, 0, J>() + acc.template at<LH, 0, 0, J>();
        const int d = acc.template at<HH, -1, -1, J>() + acc.template at<HH, -1, 0, J>() +
                      acc.template at<HH, 0, -1, J>() + acc.template at<HH, 0, 0, J>();
        o.s[LL][J] += sg * ((4 * hv - d + 8) >> 4);
      });
    }
  }
};

// ---------------------------------------------------------------------------
// Type lists and the streaming pipeline
// ---------------------------------------------------------------------------
template <class... S>
struct List {};

template <class A, class B>
struct Cat;
template <class... A, class... B>
struct Cat<List<A...>, List<B...>> {
  using type = List<A..., B...>;
};

template <class L>
struct Totals;
template <class... S>
struct Totals<List<S...>> {
  static constexpr int UP = (0 + ... + S::UP);
  static constexpr int DOWN = (0 + ... + S::DOWN);
  static constexpr int LEFT = (0 + ... + S::LEFT);
  static constexpr int RIGHT = (0 + ... + S::RIGHT);
};

// A chain of stages; each keeps the rows of its input state it still needs.
// push() takes the next input row and returns the last stage's output for
// the row sum(DOWN) positions behind it.
template <typename V, int QL, class L>
struct Pipe;

template <typename V, int QL>
struct Pipe<V, QL, List<>> {
  __device__ __forceinline__ void reset() {}
  template <class CS>
  __device__ __forceinline__ Row<V, QL> push(const Row<V, QL>& r, const CS&, const ConvTaps&) {
    return r;
  }
};

template <typename V, int QL, class S0, class... S>
struct Pipe<V, QL, List<S0, S...>> {
  static constexpr int NW = S0::UP + 1 + S0::DOWN;
  Row<V, QL> win[NW];
  Pipe<V, QL, List<S...>> rest;

  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int k = 0; k < NW; ++k)
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int j = 0; j < QL; ++j) win[k].s[s][j] = V(0);
    rest.reset();
  }

  template <class CS>
  __device__ __forceinline__ Row<V, QL> push(const Row<V, QL>& r, const CS& c, const ConvTaps& t) {
#pragma unroll
    for (int k = 0; k + 1 < NW; ++k) win[k] = win[k + 1];
    win[NW - 1] = r;
    Row<V, QL> o;
    S0::template eval<QL>(win[S0::UP], WinAcc<V, QL, S0::UP>{win}, o, c, t);
    return rest.push(o, c, t);
  }
};

}  // namespace dev
}  // namespace dwt
