// Kernels of the CONVOLUTION scheme(s): forward and inverse, CDF 5/3 and 9/7,
// float32 and float16-storage.
#include "dispatch.cuh"

namespace dwt {

bool group_convolution(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call,
                   cudaError_t* err) {
  if (dev::fused_float<CONVOLUTION, true>(k, ns, info, call, err)) return true;
  return false;
}

}  // namespace dwt
