// Kernels of the Iwahashi (Sec. 2.6) scheme: forward and inverse, every wavelet and
// storage type the scheme supports.
#include "dispatch.cuh"

namespace dwt {

bool group_iwahashi(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  return dev::fused_float<IWAHASHI, true>(k, ns, info, call, err);
}

bool tail_iwahashi(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err) {
  return dev::tail_float<IWAHASHI>(k, info, call, err);
}

}  // namespace dwt
