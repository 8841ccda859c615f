// Kernels of the row-column baseline: the vertical 1-D transform and the
// horizontal 1-D transform as two launches with the intermediate plane in
// global memory (the separable strategy of Sec. 2.5 that the paper's
// block-based schemes replace).  Forward: vertical (samples -> samples),
// then horizontal (samples -> subbands).  Inverse: horizontal (subbands ->
// samples), then vertical (samples -> samples).
#include "dispatch.cuh"

namespace dwt {
namespace {

template <int PASS, int WL, typename ST, bool INV>
using FloatPass =
    dev::Cfg<ST, float, typename dev::PassProgram<PASS, WL, INV>::type,
             (PASS == PASS_HORZ && INV) ? SUBBANDS : SAMPLES,
             (PASS == PASS_HORZ && !INV) ? SUBBANDS : SAMPLES>;

template <int PASS, bool INV>
using IntPassCfg = dev::Cfg<int, int, typename dev::IntPass<PASS, INV>::type,
                            (PASS == PASS_HORZ && INV) ? SUBBANDS : SAMPLES,
                            (PASS == PASS_HORZ && !INV) ? SUBBANDS : SAMPLES>;

template <int PASS>
bool pass_switch(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call,
                 cudaError_t* err) {
  const bool inv = k.inverse != 0;
  if (k.dtype == I32) {
    if (k.wavelet != W53) return false;
    return inv ? dev::run<IntPassCfg<PASS, true>>(ns, info, call, err)
               : dev::run<IntPassCfg<PASS, false>>(ns, info, call, err);
  }
  if (k.wavelet == W53 && k.dtype == F32)
    return inv ? dev::run<FloatPass<PASS, W53, float, true>>(ns, info, call, err)
               : dev::run<FloatPass<PASS, W53, float, false>>(ns, info, call, err);
  if (k.wavelet == W97 && k.dtype == F32)
    return inv ? dev::run<FloatPass<PASS, W97, float, true>>(ns, info, call, err)
               : dev::run<FloatPass<PASS, W97, float, false>>(ns, info, call, err);
  if (k.wavelet == WDD && k.dtype == F32)
    return inv ? dev::run<FloatPass<PASS, WDD, float, true>>(ns, info, call, err)
               : dev::run<FloatPass<PASS, WDD, float, false>>(ns, info, call, err);
  if (k.wavelet == W53 && k.dtype == F16S)
    return inv ? dev::run<FloatPass<PASS, W53, __half, true>>(ns, info, call, err)
               : dev::run<FloatPass<PASS, W53, __half, false>>(ns, info, call, err);
  if (k.wavelet == W97 && k.dtype == F16S)
    return inv ? dev::run<FloatPass<PASS, W97, __half, true>>(ns, info, call, err)
               : dev::run<FloatPass<PASS, W97, __half, false>>(ns, info, call, err);
  return false;
}

}  // namespace

bool group_rowcol(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call,
                  cudaError_t* err) {
  if (k.pass == PASS_VERT) return pass_switch<PASS_VERT>(k, ns, info, call, err);
  if (k.pass == PASS_HORZ) return pass_switch<PASS_HORZ>(k, ns, info, call, err);
  return false;
}

}  // namespace dwt
