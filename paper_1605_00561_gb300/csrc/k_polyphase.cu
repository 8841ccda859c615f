// Kernels of the POLYPHASE and POLYPHASE_S scheme(s): forward and inverse, CDF 5/3 and 9/7,
// float32 and float16-storage.
#include "dispatch.cuh"

namespace dwt {

bool group_polyphase(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call,
                   cudaError_t* err) {
  if (dev::fused_float<POLYPHASE>(k, ns, info, call, err)) return true;
  if (dev::fused_float<POLYPHASE_S, true>(k, ns, info, call, err)) return true;
  return false;
}

}  // namespace dwt
