// Kernels of the Polyphase (Sec. 2.3) scheme: forward and inverse, every wavelet and
// storage type the scheme supports.
#include "dispatch.cuh"

namespace dwt {

bool group_polyphase(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  return dev::fused_float<POLYPHASE, true>(k, ns, info, call, err);
}

bool tail_polyphase(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err) {
  return dev::tail_float<POLYPHASE>(k, info, call, err);
}

}  // namespace dwt
