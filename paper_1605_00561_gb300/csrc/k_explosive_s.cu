// Kernels of the Explosive* (Sec. 3.1 with the split of Sec. 4) scheme: forward and
// inverse, every wavelet and storage type the scheme supports.
#include "dispatch.cuh"

namespace dwt {

bool group_explosive_s(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  return dev::fused_float<EXPLOSIVE_S, true>(k, ns, info, call, err);
}

bool tail_explosive_s(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err) {
  return dev::tail_float<EXPLOSIVE_S>(k, info, call, err);
}

}  // namespace dwt
