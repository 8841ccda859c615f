// Kernels of the Iwahashi (Sec. 2.6) scheme: forward and inverse, every wavelet and
// storage type the scheme supports, and the reversible integer Iwahashi
// lifting of CDF 5/3 (each step rounded once; a transform of its own).
#include "dispatch.cuh"

namespace dwt {

bool group_iwahashi(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  if (k.pass == PASS_FUSED && k.scheme == IWAHASHI && k.dtype == I32) {
    if (k.wavelet != W53) return false;
    return k.inverse
               ? dev::run<dev::Cfg<int, int, dev::IntIwFused<true>::type, SUBBANDS, SAMPLES>>(ns, info, call, err)
               : dev::run<dev::Cfg<int, int, dev::IntIwFused<false>::type, SAMPLES, SUBBANDS>>(ns, info, call, err);
  }
  return dev::fused_float<IWAHASHI, true>(k, ns, info, call, err);
}

bool tail_iwahashi(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err) {
  if (k.pass == PASS_FUSED && k.scheme == IWAHASHI && k.dtype == I32) {
    if (k.wavelet != W53) return false;
    // a tail level has both sides >= 2: every subband exists
    return k.inverse ? dev::run_tail<dev::TailCfg<int, int, dev::IntIwFused<true>::type, SUBBANDS, SAMPLES,
                                                  dev::StCoefs<W53, true>>>(info, call, err)
                     : dev::run_tail<dev::TailCfg<int, int, dev::IntIwFused<false>::type, SAMPLES, SUBBANDS,
                                                  dev::StCoefs<W53, false>>>(info, call, err);
  }
  return dev::tail_float<IWAHASHI>(k, info, call, err);
}

}  // namespace dwt
