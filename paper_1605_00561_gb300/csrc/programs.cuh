// The paper's schemes as stage lists, per predict/update pair (pair K of
// degree DEG), in the order the matrices are applied (right to left in the
// paper's equations).  Inverses apply the inverse step matrices in reverse
// order; a step whose targets are not among its sources inverts by negating
// every term; the Monolithic steps invert to T_{-P} and S_{-U}; the
// Polyphase step inverts to N^{-1} = T_{-P} S_{-U}.
#pragma once

#include "stages.cuh"

namespace dwt {
namespace dev {

// --- Sweldens (Sec. 2.5): T^H_P, T^V_P, S^H_U, S^V_U ------------------------
template <int D, int K, int PO, int S = 1>
using TH = Lin<D, K, false, Term<HL, LL, OP_I, PO, S>, Term<HH, LH, OP_I, PO, S>>;
template <int D, int K, int PO, int S = 1>
using TV = Lin<D, K, false, Term<LH, LL, PO, OP_I, S>, Term<HH, HL, PO, OP_I, S>>;
template <int D, int K, int UO, int S = 1>
using SH = Lin<D, K, false, Term<LL, HL, OP_I, UO, S>, Term<LH, HH, OP_I, UO, S>>;
template <int D, int K, int UO, int S = 1>
using SV = Lin<D, K, false, Term<LL, LH, UO, OP_I, S>, Term<HL, HH, UO, OP_I, S>>;

// --- Iwahashi (Sec. 2.6): T^I_P, R^I_{P,U}, S^I_U ---------------------------
template <int D, int K, int PO, int S = 1>
using TI = Lin<D, K, false, Term<HH, LL, PO, PO, S>, Term<HH, HL, PO, OP_I, S>,
               Term<HH, LH, OP_I, PO, S>>;
template <int D, int K, int PO, int UO, int S = 1>
using RI = Lin<D, K, false, Term<HL, LL, OP_I, PO, S>, Term<HL, HH, UO, OP_I, S>,
               Term<LH, LL, PO, OP_I, S>, Term<LH, HH, OP_I, UO, S>>;
template <int D, int K, int UO, int S = 1>
using SI = Lin<D, K, false, Term<LL, HL, OP_I, UO, S>, Term<LL, LH, UO, OP_I, S>,
               Term<LL, HH, UO, UO, -S>>;

// --- Explosive (Sec. 3.1): T^E_P, R^E_{P,U}, S^E_U --------------------------
template <int D, int K, int PO, int S = 1>
using TE = Lin<D, K, false, Term<HL, LL, OP_I, PO, S>, Term<LH, LL, PO, OP_I, S>,
               Term<HH, LL, PO, PO, -S>>;
template <int D, int K, int PO, int UO, int S = 1>
using RE = Lin<D, K, false, Term<LL, HL, OP_I, UO, S>, Term<LL, LH, UO, OP_I, S>,
               Term<HH, HL, PO, OP_I, S>, Term<HH, LH, OP_I, PO, S>>;
template <int D, int K, int UO, int S = 1>
using SE = Lin<D, K, false, Term<LL, HH, UO, UO, S>, Term<HL, HH, UO, OP_I, S>,
               Term<LH, HH, OP_I, UO, S>>;

// --- Monolithic (Sec. 3.2): T_P, S_U; S = -1 gives T_{-P}, S_{-U} ----------
template <int D, int K, int PO, int S = 1>
using TM = Lin<D, K, false, Term<HL, LL, OP_I, PO, S>, Term<LH, LL, PO, OP_I, S>,
               Term<HH, LL, PO, PO, 1>, Term<HH, HL, PO, OP_I, S>, Term<HH, LH, OP_I, PO, S>>;
template <int D, int K, int UO, int S = 1>
using SM = Lin<D, K, false, Term<LL, HL, OP_I, UO, S>, Term<LL, LH, UO, OP_I, S>,
               Term<LL, HH, UO, UO, 1>, Term<HL, HH, UO, OP_I, S>, Term<LH, HH, OP_I, UO, S>>;

// --- Polyphase (Sec. 2.3): N_{P,U} with V = PU + 1, and its inverse --------
// Terms are listed with the same-subband (diagonal) entry of each row last,
// so that its large contribution is accumulated after the smaller ones.
template <int D, int K, int PO, int UO, int VO>
using NP = Lin<D, K, true,
               Term<LL, HL, VO, UO>, Term<LL, LH, UO, VO>, Term<LL, HH, UO, UO>, Term<LL, LL, VO, VO>,
               Term<HL, LL, VO, PO>, Term<HL, LH, UO, PO>, Term<HL, HH, UO, OP_I>, Term<HL, HL, VO, OP_I>,
               Term<LH, LL, PO, VO>, Term<LH, HL, PO, UO>, Term<LH, HH, OP_I, UO>, Term<LH, LH, OP_I, VO>,
               Term<HH, LL, PO, PO>, Term<HH, HL, PO, OP_I>, Term<HH, LH, OP_I, PO>, Term<HH, HH, OP_I, OP_I>>;
// N^{-1} = [[1, -U, -U*, UU*], [-P, V, PU*, -U*V], [-P*, P*U, V*, -UV*], [PP*, -P*V, -PV*, V*V]]
template <int D, int K, int PO, int UO, int VO>
using NPinv = Lin<D, K, true,
               Term<LL, HL, OP_I, UO, -1>, Term<LL, LH, UO, OP_I, -1>, Term<LL, HH, UO, UO>, Term<LL, LL, OP_I, OP_I>,
               Term<HL, LL, OP_I, PO, -1>, Term<HL, LH, UO, PO>, Term<HL, HH, UO, VO, -1>, Term<HL, HL, OP_I, VO>,
               Term<LH, LL, PO, OP_I, -1>, Term<LH, HL, PO, UO>, Term<LH, HH, VO, UO, -1>, Term<LH, LH, VO, OP_I>,
               Term<HH, LL, PO, PO>, Term<HH, HL, PO, VO, -1>, Term<HH, LH, VO, PO, -1>, Term<HH, HH, VO, VO>>;

// ---------------------------------------------------------------------------
// One pair of a scheme, forward and inverse.
// ---------------------------------------------------------------------------
template <int SCHEME, int D, int K>
struct PairProg;

template <int D, int K>
struct PairProg<SWELDENS, D, K> {
  using fwd = List<TH<D, K, OP_P>, TV<D, K, OP_P>, SH<D, K, OP_U>, SV<D, K, OP_U>>;
  using inv = List<SV<D, K, OP_U, -1>, SH<D, K, OP_U, -1>, TV<D, K, OP_P, -1>, TH<D, K, OP_P, -1>>;
};
template <int D, int K>
struct PairProg<IWAHASHI, D, K> {
  using fwd = List<TI<D, K, OP_P>, RI<D, K, OP_P, OP_U>, SI<D, K, OP_U>>;
  using inv = List<SI<D, K, OP_U, -1>, RI<D, K, OP_P, OP_U, -1>, TI<D, K, OP_P, -1>>;
};
template <int D, int K>
struct PairProg<IWAHASHI_S, D, K> {  // S^V_U0 S^H_U0 S^I_U1 | R^I | T^I_P1 | T^V_P0 T^H_P0
  using fwd = List<TH<D, K, OP_P0>, TV<D, K, OP_P0>, TI<D, K, OP_P1>, RI<D, K, OP_P1, OP_U1>,
                   SI<D, K, OP_U1>, SH<D, K, OP_U0>, SV<D, K, OP_U0>>;
  using inv = List<SV<D, K, OP_U0, -1>, SH<D, K, OP_U0, -1>, SI<D, K, OP_U1, -1>,
                   RI<D, K, OP_P1, OP_U1, -1>, TI<D, K, OP_P1, -1>, TV<D, K, OP_P0, -1>,
                   TH<D, K, OP_P0, -1>>;
};
template <int D, int K>
struct PairProg<EXPLOSIVE, D, K> {
  using fwd = List<TE<D, K, OP_P>, RE<D, K, OP_P, OP_U>, SE<D, K, OP_U>>;
  using inv = List<SE<D, K, OP_U, -1>, RE<D, K, OP_P, OP_U, -1>, TE<D, K, OP_P, -1>>;
};
template <int D, int K>
struct PairProg<EXPLOSIVE_S, D, K> {
  using fwd = List<TH<D, K, OP_P0>, TV<D, K, OP_P0>, TE<D, K, OP_P1>, RE<D, K, OP_P1, OP_U1>,
                   SE<D, K, OP_U1>, SH<D, K, OP_U0>, SV<D, K, OP_U0>>;
  using inv = List<SV<D, K, OP_U0, -1>, SH<D, K, OP_U0, -1>, SE<D, K, OP_U1, -1>,
                   RE<D, K, OP_P1, OP_U1, -1>, TE<D, K, OP_P1, -1>, TV<D, K, OP_P0, -1>,
                   TH<D, K, OP_P0, -1>>;
};
template <int D, int K>
struct PairProg<MONOLITHIC, D, K> {
  using fwd = List<TM<D, K, OP_P>, SM<D, K, OP_U>>;
  using inv = List<SM<D, K, OP_U, -1>, TM<D, K, OP_P, -1>>;
};
template <int D, int K>
struct PairProg<MONOLITHIC_S, D, K> {  // S^V_U0 S^H_U0 S_U1 | T^V_P0 T^H_P0 T_P1
  using fwd = List<TM<D, K, OP_P1>, TH<D, K, OP_P0>, TV<D, K, OP_P0>, SM<D, K, OP_U1>,
                   SH<D, K, OP_U0>, SV<D, K, OP_U0>>;
  using inv = List<SV<D, K, OP_U0, -1>, SH<D, K, OP_U0, -1>, SM<D, K, OP_U1, -1>,
                   TV<D, K, OP_P0, -1>, TH<D, K, OP_P0, -1>, TM<D, K, OP_P1, -1>>;
};
template <int D, int K>
struct PairProg<POLYPHASE, D, K> {
  using fwd = List<NP<D, K, OP_P, OP_U, OP_V>>;
  using inv = List<NPinv<D, K, OP_P, OP_U, OP_V>>;
};
template <int D, int K>
struct PairProg<POLYPHASE_S, D, K> {  // S^V_U0 S^H_U0 N_{P1,U1} | T^V_P0 T^H_P0
  using fwd = List<TH<D, K, OP_P0>, TV<D, K, OP_P0>, NP<D, K, OP_P1, OP_U1, OP_V1>,
                   SH<D, K, OP_U0>, SV<D, K, OP_U0>>;
  using inv = List<SV<D, K, OP_U0, -1>, SH<D, K, OP_U0, -1>, NPinv<D, K, OP_P1, OP_U1, OP_V1>,
                   TV<D, K, OP_P0, -1>, TH<D, K, OP_P0, -1>>;
};

// Row-column baseline: the vertical and the horizontal 1-D transforms as two
// separate passes through global memory.
template <int PASS, int D, int K>
struct PassProg;
template <int D, int K>
struct PassProg<PASS_VERT, D, K> {
  using fwd = List<TV<D, K, OP_P>, SV<D, K, OP_U>>;
  using inv = List<SV<D, K, OP_U, -1>, TV<D, K, OP_P, -1>>;
};
template <int D, int K>
struct PassProg<PASS_HORZ, D, K> {
  using fwd = List<TH<D, K, OP_P>, SH<D, K, OP_U>>;
  using inv = List<SH<D, K, OP_U, -1>, TH<D, K, OP_P, -1>>;
};

// ---------------------------------------------------------------------------
// Whole programs: all pairs, scaling, direction.
// ---------------------------------------------------------------------------
template <int WL>
constexpr int kPairs = WL == W97 ? 2 : 1;
template <int WL>
constexpr int kDeg = WL == WDD ? 3 : 1;

template <class P0, class P1, int NPAIRS, bool INV>
struct JoinPairs;
template <class P0, class P1>
struct JoinPairs<P0, P1, 1, false> {
  using type = typename Cat<typename P0::fwd, List<Scale>>::type;
};
template <class P0, class P1>
struct JoinPairs<P0, P1, 2, false> {
  using type = typename Cat<typename Cat<typename P0::fwd, typename P1::fwd>::type, List<Scale>>::type;
};
template <class P0, class P1>
struct JoinPairs<P0, P1, 1, true> {
  using type = typename Cat<List<Scale>, typename P0::inv>::type;
};
template <class P0, class P1>
struct JoinPairs<P0, P1, 2, true> {
  using type = typename Cat<typename Cat<List<Scale>, typename P1::inv>::type, typename P0::inv>::type;
};

template <int SCHEME, int WL, bool INV>
struct FusedProgram {
  using type = typename JoinPairs<PairProg<SCHEME, kDeg<WL>, 0>, PairProg<SCHEME, kDeg<WL>, 1>,
                                  kPairs<WL>, INV>::type;
};
template <int WL, bool INV>
struct FusedProgram<CONVOLUTION, WL, INV> {
  using type = List<Conv<WL, INV>>;
};

template <int PASS, int WL, bool INV>
struct PassProgram {
  using type = typename JoinPairs<PassProg<PASS, kDeg<WL>, 0>, PassProg<PASS, kDeg<WL>, 1>,
                                  kPairs<WL>, INV>::type;
};

// Reversible integer 5/3 in the JPEG 2000 order (columns, then rows).
template <bool INV>
struct IntFused {
  using type = typename std::conditional<
      !INV, List<Int53<0, false>, Int53<1, false>, Int53<2, false>, Int53<3, false>>,
      List<Int53<3, true>, Int53<2, true>, Int53<1, true>, Int53<0, true>>>::type;
};
// Reversible integer Iwahashi lifting (its own rounding): T, R, S.
template <bool INV>
struct IntIwFused {
  using type = typename std::conditional<!INV, List<IntIw<0, false>, IntIw<1, false>, IntIw<2, false>>,
                                         List<IntIw<2, true>, IntIw<1, true>, IntIw<0, true>>>::type;
};
template <int PASS, bool INV>
struct IntPass {
  using type = typename std::conditional<
      PASS == PASS_VERT,
      typename std::conditional<!INV, List<Int53<0, false>, Int53<1, false>>,
                                List<Int53<1, true>, Int53<0, true>>>::type,
      typename std::conditional<!INV, List<Int53<2, false>, Int53<3, false>>,
                                List<Int53<3, true>, Int53<2, true>>>::type>::type;
};

}  // namespace dev
}  // namespace dwt
