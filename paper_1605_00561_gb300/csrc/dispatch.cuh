// Instantiation helpers shared by the kernel translation units.  Each unit
// owns a group of schemes and answers "kernel info" and "launch" requests
// for the (wavelet, dtype, direction) combinations of its group.
#pragma once

#include <type_traits>

#include "level_kernel.cuh"

namespace dwt {

namespace dev {

template <class C>
inline bool run(int nstages, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  using I = Instance<C>;
  if (info) *info = I::info(nstages);
  if (call) *err = I::launch(*call->a, *call->maps, *call->cf, *call->ct, call->stream);
  return true;
}

// Quadruples per lane: four for the light schemes (128-bit vectors, fewer
// instructions per pixel); two for the schemes whose windows or stencils
// would otherwise exceed the register file (Polyphase, Convolution, and the
// three-step schemes of two pairs).  A ring stage holds the same bytes
// either way.
template <int SCHEME, int WL>
constexpr int kQuadsPerLane =
    (SCHEME == POLYPHASE || SCHEME == POLYPHASE_S || SCHEME == CONVOLUTION ||
     (WL == W97 && (SCHEME == IWAHASHI || SCHEME == IWAHASHI_S || SCHEME == EXPLOSIVE ||
                    SCHEME == EXPLOSIVE_S)))
        ? 2
        : 4;

// STATIC: coefficients folded in at compile time (StCoefs), for levels with
// JPEG 2000 normalisation and both axes longer than one sample.
template <int SCHEME, int WL, typename ST, bool INV, bool STATIC = false>
using FusedCfg = Cfg<ST, float, typename FusedProgram<SCHEME, WL, INV>::type, INV ? SUBBANDS : SAMPLES,
                     INV ? SAMPLES : SUBBANDS, kQuadsPerLane<SCHEME, WL>, 8 / kQuadsPerLane<SCHEME, WL>,
                     SCHEME == CONVOLUTION ? 8 : 16, std::conditional_t<STATIC, StCoefs<WL, INV>, RtTag>>;

template <int SCHEME, int WL, typename ST, bool STATIC>
inline bool fused_dir(bool inv, int ns, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  return inv ? run<FusedCfg<SCHEME, WL, ST, true, STATIC>>(ns, info, call, err)
             : run<FusedCfg<SCHEME, WL, ST, false, STATIC>>(ns, info, call, err);
}

// The float combinations of one fused scheme; schemes listed with
// WITH_STATIC also carry compile-time-coefficient kernels, taken when the
// launch allows them.
template <int SCHEME, bool WITH_STATIC = false>
inline bool fused_float(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call,
                        cudaError_t* err) {
  if (k.pass != PASS_FUSED || k.scheme != SCHEME) return false;
  const bool inv = k.inverse != 0;
  if constexpr (WITH_STATIC) {
    if (k.static_coefs) {
      if (k.wavelet == W53 && k.dtype == F32) return fused_dir<SCHEME, W53, float, true>(inv, ns, info, call, err);
      if (k.wavelet == W97 && k.dtype == F32) return fused_dir<SCHEME, W97, float, true>(inv, ns, info, call, err);
      if (k.wavelet == W53 && k.dtype == F16S) return fused_dir<SCHEME, W53, __half, true>(inv, ns, info, call, err);
      if (k.wavelet == W97 && k.dtype == F16S) return fused_dir<SCHEME, W97, __half, true>(inv, ns, info, call, err);
    }
  }
  if (k.wavelet == W53 && k.dtype == F32) return fused_dir<SCHEME, W53, float, false>(inv, ns, info, call, err);
  if (k.wavelet == W97 && k.dtype == F32) return fused_dir<SCHEME, W97, float, false>(inv, ns, info, call, err);
  if (k.wavelet == W53 && k.dtype == F16S) return fused_dir<SCHEME, W53, __half, false>(inv, ns, info, call, err);
  if (k.wavelet == W97 && k.dtype == F16S) return fused_dir<SCHEME, W97, __half, false>(inv, ns, info, call, err);
  return false;
}

}  // namespace dev
}  // namespace dwt
