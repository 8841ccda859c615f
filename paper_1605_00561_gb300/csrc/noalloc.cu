// dwt2_forward_noalloc: the forward transform for callers that cannot
// allocate device memory -- for example code running inside a CUDA graph
// that is being captured, a real-time or embedded loop that must not call
// cudaMalloc (it can synchronise the device and take an unbounded time), or
// a host framework that owns every allocation itself.  The LL scratch of
// the multi-level pyramid and the device status word live in one
// file-scope device array of this library instead of a plan.
#include "dwt.h"

#include <mutex>

#include "dwt_internal.h"

namespace dwt {
dwt_status forward_on_scratch(int w, int h, int wavelet, int levels, int dtype, const void* src,
                              size_t src_pitch, void* dst, size_t dst_pitch, void* scratch,
                              size_t scratch_bytes, int* d_status, cudaStream_t s);
}

namespace {

// Bytes of LL scratch available to dwt2_forward_noalloc: enough for a
// 4096 x 4096 float32 image (24 MiB).  The status word sits after it.
constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr size_t kStatusOffset = kScratchBytes;

// Every device that loads this library holds this array until the process
// exits.  All calls share it: overlapping calls race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes + 256];

std::mutex g_mu;
void* g_addr[64];  // device address of the array, per device (set once)

}  // namespace

extern "C" dwt_status dwt2_forward_noalloc(int w, int h, dwt_wavelet wavelet, int levels,
                                           dwt_dtype dtype, const void* d_in, size_t in_pitch_bytes,
                                           void* d_out, size_t out_pitch_bytes, dwt_stream stream) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DWT_ECUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      // in host code the array's name only stands for the symbol: the
      // device address comes from the runtime, once per device
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DWT_ECUDA;
      }
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* d_status = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kStatusOffset);
  // the array keeps the previous call's contents: the status word starts at zero
  if (cudaMemsetAsync(d_status, 0, sizeof(int), s) != cudaSuccess) return DWT_ECUDA;
  return dwt::forward_on_scratch(w, h, (int)wavelet, levels, (int)dtype, d_in, in_pitch_bytes, d_out,
                                 out_pitch_bytes, base, kScratchBytes, d_status, s);
}
