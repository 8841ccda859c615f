// dwt2_forward_noalloc: the forward transform for callers that cannot
// allocate device memory -- a real-time loop that must not call cudaMalloc
// (it can synchronise the device and take an unbounded time), an embedded or
// plug-in caller whose host application owns every device allocation, or a
// process that has spent its memory budget.  The LL scratch of the
// multi-level pyramid and the device status word live in one file-scope
// device array of this library instead of a plan.
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
// 4096 x 4096 float32 image (24 MiB).  Two words follow it: the status word
// (raised by a bounded wait that ran out, cleared by the status query) and
// a flag that nothing ever writes (the injected hold of dwt_debug_inject
// waits on it).  Device arrays start zeroed when the module loads.
constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr size_t kStatusOffset = kScratchBytes;

// Every device that loads this library holds this array until the process
// exits.  All calls share it: overlapping calls race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes + 256];

std::mutex g_mu;
void* g_addr[64];  // device address of the array, per device (set once)

// The array's device address on the current device, looked up on first use
// (in host code the array's name only stands for the symbol).  With
// `lookup` false, a device that never made a call gives nullptr.
dwt_status array_address(bool lookup, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DWT_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev] && lookup) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return DWT_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DWT_OK;
}

}  // namespace

extern "C" dwt_status dwt2_forward_noalloc(int w, int h, dwt_wavelet wavelet, int levels,
                                           dwt_dtype dtype, const void* d_in, size_t in_pitch_bytes,
                                           void* d_out, size_t out_pitch_bytes, dwt_stream stream) {
  void* base = nullptr;
  const dwt_status st = array_address(true, &base);
  if (st != DWT_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* d_status = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kStatusOffset);
  return dwt::forward_on_scratch(w, h, (int)wavelet, levels, (int)dtype, d_in, in_pitch_bytes, d_out,
                                 out_pitch_bytes, base, kScratchBytes, d_status, s);
}

extern "C" dwt_status dwt_noalloc_device_status(dwt_stream stream) {
  void* base = nullptr;
  const dwt_status st = array_address(false, &base);
  if (st != DWT_OK) return st;
  if (!base) return DWT_OK;  // no call on this device yet
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* d_status = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kStatusOffset);
  int v = 0;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&v, d_status, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(d_status, 0, sizeof(int));
  if (e != cudaSuccess) return DWT_ECUDA;
  return v ? DWT_ETIMEOUT : DWT_OK;
}
