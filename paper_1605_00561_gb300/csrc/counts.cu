// Operation and barrier counts of the programs the kernels run, computed at
// compile time from the same stage lists (programs.cuh), for comparison with
// the paper's Table of operations and barriers (Sec. 5): multiply-
// accumulates per quadruple (every tap of every term of every step; the
// unit diagonal of the merged Polyphase matrix and the scaling step are not
// operations) and barriers (steps that read other quadruples).  Also the
// shared-memory words the tile kernel publishes per quadruple (the
// subbands each such step reads from other quadruples).
#include "dwt.h"

#include "dispatch.cuh"

namespace dwt {
namespace dev {
namespace {

template <int DEG, int OP>
constexpr int ntaps() {
  int n = 0;
  for (int o = OpShape<DEG, OP>::lo; o <= OpShape<DEG, OP>::hi; ++o) n += OpShape<DEG, OP>::has(o) ? 1 : 0;
  return n;
}

template <int DEG, class T>
constexpr int term_taps() {
  // a term of the identity on both axes into its own subband is the unit
  // diagonal of a merged matrix: a copy, not an operation
  return (T::vop == OP_I && T::hop == OP_I && T::tgt == T::src) ? 0 : ntaps<DEG, T::vop>() * ntaps<DEG, T::hop>();
}

constexpr int popcount4(unsigned m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

struct Count {
  int macs, barriers, words;
};

template <class S>
struct StepCount;
template <int DEG, int K, bool R, class... Ts>
struct StepCount<Lin<DEG, K, R, Ts...>> {
  static constexpr unsigned N = Lin<DEG, K, R, Ts...>::NEIGHBOUR_SRCS;
  static constexpr Count v{(0 + ... + term_taps<DEG, Ts>()), N ? 1 : 0, popcount4(N)};
};
template <>
struct StepCount<Scale> {
  static constexpr Count v{0, 0, 0};
};
template <int WL, bool INV>
struct StepCount<Conv<WL, INV>> {
  using S = ConvShape<WL, INV>;
  static constexpr int n1() {
    int n = 0;
    for (int o = 0; o < 2; ++o)
      for (int i = 0; i < 2; ++i) n += S::hi(o, i) - S::lo(o, i) + 1;
    return n;
  }
  // every output subband is a 2-D filter of every input subband
  static constexpr Count v{n1() * n1(), 1, 4};
};

template <class L>
struct ProgCount;
template <class... S>
struct ProgCount<List<S...>> {
  static constexpr Count v{(0 + ... + StepCount<S>::v.macs), (0 + ... + StepCount<S>::v.barriers),
                           (0 + ... + StepCount<S>::v.words)};
};

template <int SCHEME, int WL>
Count fused() {
  return ProgCount<typename FusedProgram<SCHEME, WL, false>::type>::v;
}

template <int WL>
Count of_scheme(int scheme) {
  switch (scheme) {
    case ROWCOL: {
      const Count v = ProgCount<typename PassProgram<PASS_VERT, WL, false>::type>::v;
      const Count h = ProgCount<typename PassProgram<PASS_HORZ, WL, false>::type>::v;
      return Count{v.macs + h.macs, v.barriers + h.barriers, v.words + h.words};
    }
    case SWELDENS: return fused<SWELDENS, WL>();
    case IWAHASHI: return fused<IWAHASHI, WL>();
    case IWAHASHI_S: return fused<IWAHASHI_S, WL>();
    case EXPLOSIVE: return fused<EXPLOSIVE, WL>();
    case EXPLOSIVE_S: return fused<EXPLOSIVE_S, WL>();
    case MONOLITHIC: return fused<MONOLITHIC, WL>();
    case MONOLITHIC_S: return fused<MONOLITHIC_S, WL>();
    case POLYPHASE: return fused<POLYPHASE, WL>();
    case POLYPHASE_S: return fused<POLYPHASE_S, WL>();
    case CONVOLUTION: return fused<CONVOLUTION, WL>();
  }
  return Count{-1, -1, -1};
}

}  // namespace
}  // namespace dev
}  // namespace dwt

extern "C" dwt_status dwt_scheme_counts(dwt_wavelet wavelet, dwt_scheme scheme, int* macs, int* barriers,
                                        int* smem_words) {
  using namespace dwt;
  if ((int)scheme <= DWT_AUTO || (int)scheme >= NUM_SCHEMES) return DWT_EINVAL;
  dev::Count c;
  switch ((int)wavelet) {
    case W53: c = dev::of_scheme<W53>((int)scheme); break;
    case W97: c = dev::of_scheme<W97>((int)scheme); break;
    case WDD: c = dev::of_scheme<WDD>((int)scheme); break;
    default: return DWT_EINVAL;
  }
  if (macs) *macs = c.macs;
  if (barriers) *barriers = c.barriers;
  if (smem_words) *smem_words = c.words;
  return DWT_OK;
}
