// Kernels of the SWELDENS scheme(s): forward and inverse, CDF 5/3 and 9/7,
// float32 and float16-storage.
#include "dispatch.cuh"

namespace dwt {

bool group_sweldens(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call,
                   cudaError_t* err) {
  if (k.pass == PASS_FUSED && k.scheme == SWELDENS && k.dtype == I32) {
    if (k.wavelet != W53) return false;
    // reversible 5/3: the separable single-loop order is the JPEG 2000 order
    return k.inverse
               ? dev::run<dev::Cfg<int, int, dev::IntFused<true>::type, SUBBANDS, SAMPLES>>(ns, info, call, err)
               : dev::run<dev::Cfg<int, int, dev::IntFused<false>::type, SAMPLES, SUBBANDS>>(ns, info, call, err);
  }
  if (dev::fused_float<SWELDENS, true>(k, ns, info, call, err)) return true;
  return false;
}

bool tail_sweldens(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err) {
  if (k.pass == PASS_FUSED && k.scheme == SWELDENS && k.dtype == I32) {
    if (k.wavelet != W53) return false;
    // reversible 5/3 in the JPEG 2000 order; a tail level has both sides >= 2
    return k.inverse ? dev::run_tail<dev::TailCfg<int, int, dev::IntFused<true>::type, SUBBANDS, SAMPLES,
                                                  dev::StCoefs<W53, true>>>(info, call, err)
                     : dev::run_tail<dev::TailCfg<int, int, dev::IntFused<false>::type, SAMPLES, SUBBANDS,
                                                  dev::StCoefs<W53, false>>>(info, call, err);
  }
  return dev::tail_float<SWELDENS>(k, info, call, err);
}

}  // namespace dwt
