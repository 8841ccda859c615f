// Kernels of the Monolithic (Sec. 3.2) scheme: forward and inverse, every wavelet and
// storage type the scheme supports.
#include "dispatch.cuh"

namespace dwt {

bool group_monolithic(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  return dev::fused_float<MONOLITHIC, true>(k, ns, info, call, err);
}

bool tail_monolithic(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err) {
  return dev::tail_float<MONOLITHIC>(k, info, call, err);
}

}  // namespace dwt
