// Kernels of the Explosive (Sec. 3.1) scheme: forward and inverse, every wavelet and
// storage type the scheme supports.
#include "dispatch.cuh"

namespace dwt {

bool group_explosive(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  return dev::fused_float<EXPLOSIVE, true>(k, ns, info, call, err);
}

bool tail_explosive(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err) {
  return dev::tail_float<EXPLOSIVE>(k, info, call, err);
}

}  // namespace dwt
