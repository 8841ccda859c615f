// Instantiation helpers shared by the kernel translation units.  Each unit
// owns a group of schemes and answers "kernel info" and "launch" requests
// for the (wavelet, dtype, direction) combinations of its group.
#pragma once

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

template <int SCHEME, int WL, typename ST, bool INV>
using FusedCfg = Cfg<ST, float, typename FusedProgram<SCHEME, WL, INV>::type, INV ? SUBBANDS : SAMPLES,
                     INV ? SAMPLES : SUBBANDS, kQuadsPerLane<SCHEME, WL>, 8 / kQuadsPerLane<SCHEME, WL>,
                     SCHEME == CONVOLUTION ? 8 : 16>;

// The eight float combinations of one fused scheme.
template <int SCHEME>
inline bool fused_float(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call,
                        cudaError_t* err) {
  if (k.pass != PASS_FUSED || k.scheme != SCHEME) return false;
  const bool inv = k.inverse != 0;
  if (k.wavelet == W53 && k.dtype == F32)
    return inv ? run<FusedCfg<SCHEME, W53, float, true>>(ns, info, call, err)
               : run<FusedCfg<SCHEME, W53, float, false>>(ns, info, call, err);
  if (k.wavelet == W97 && k.dtype == F32)
    return inv ? run<FusedCfg<SCHEME, W97, float, true>>(ns, info, call, err)
               : run<FusedCfg<SCHEME, W97, float, false>>(ns, info, call, err);
  if (k.wavelet == W53 && k.dtype == F16S)
    return inv ? run<FusedCfg<SCHEME, W53, __half, true>>(ns, info, call, err)
               : run<FusedCfg<SCHEME, W53, __half, false>>(ns, info, call, err);
  if (k.wavelet == W97 && k.dtype == F16S)
    return inv ? run<FusedCfg<SCHEME, W97, __half, true>>(ns, info, call, err)
               : run<FusedCfg<SCHEME, W97, __half, false>>(ns, info, call, err);
  return false;
}

}  // namespace dev
}  // namespace dwt
