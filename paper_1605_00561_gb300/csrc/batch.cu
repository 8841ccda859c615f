// The persistent batch kernel behind dwt_batch_submit: every level of many
// transforms of mixed sizes, level counts, wavelets, storage types and
// directions in one launch.
//
// Work items are strips of (request, level); the host orders them so that
// every strip comes after the strips it reads (see batch_submit).
// Persistent one-warp blocks pop items from a global counter.  Before a
// strip of level k starts, the warp waits until the strip rows of the
// level it reads that cover its input rows (with the halo, mirrored) are
// complete: levels overlap as a wavefront instead of waiting for each
// other as a whole.  Items are popped in queue order, so everything a
// strip waits for was taken earlier by a running warp and the wait ends;
// it is bounded all the same, and a wait that runs out sets the request's
// status to DWT_ETIMEOUT instead of hanging.  Each kind of request runs the
// same strip code as the per-level kernels (run_strip), with a fixed
// scheme: Monolithic* for the float wavelets, the separable JPEG 2000
// order for reversible 5/3.
#include "batch.h"
#include "dispatch.cuh"

namespace dwt {
namespace dev {
namespace {

template <int WL, typename ST, bool INV, bool STATIC>
using FloatKind = FusedCfg<MONOLITHIC_S, WL, ST, INV, STATIC>;
template <bool INV>
using IntKind = Cfg<int, int, typename IntFused<INV>::type, INV ? SUBBANDS : SAMPLES, INV ? SAMPLES : SUBBANDS>;

// The kinds a batch can hold, in BatchKind order.
using K0 = FloatKind<W97, float, false, true>;
using K1 = FloatKind<W97, float, true, true>;
using K2 = FloatKind<W53, float, false, true>;
using K3 = FloatKind<W53, float, true, true>;
using K4 = IntKind<false>;
using K5 = IntKind<true>;
using K6 = FloatKind<W97, __half, false, true>;
using K7 = FloatKind<W97, __half, true, true>;
using K8 = FloatKind<W53, __half, false, true>;
using K9 = FloatKind<W53, __half, true, true>;
using R0 = FloatKind<W97, float, false, false>;
using R1 = FloatKind<W97, float, true, false>;
using R2 = FloatKind<W53, float, false, false>;
using R3 = FloatKind<W53, float, true, false>;
using R6 = FloatKind<W97, __half, false, false>;
using R7 = FloatKind<W97, __half, true, false>;
using R8 = FloatKind<W53, __half, false, false>;
using R9 = FloatKind<W53, __half, true, false>;
using D0 = FloatKind<WDD, float, false, true>;
using D1 = FloatKind<WDD, float, true, true>;
using D2 = FloatKind<WDD, float, false, false>;
using D3 = FloatKind<WDD, float, true, false>;

constexpr int cmax_bytes(int a, int b) { return a > b ? a : b; }
// runtime kinds share their geometry with the static ones
constexpr int kStageStride =
    cmax_bytes(cmax_bytes(cmax_bytes(K0::STAGE_BYTES, K1::STAGE_BYTES), cmax_bytes(K2::STAGE_BYTES, K3::STAGE_BYTES)),
               cmax_bytes(cmax_bytes(K4::STAGE_BYTES, K5::STAGE_BYTES),
                          cmax_bytes(cmax_bytes(K6::STAGE_BYTES, K7::STAGE_BYTES),
                                     cmax_bytes(cmax_bytes(K8::STAGE_BYTES, K9::STAGE_BYTES),
                                                cmax_bytes(D0::STAGE_BYTES, D1::STAGE_BYTES)))));

__constant__ ConvTaps kNoTaps;  // none of the batch kinds reads taps

// One strip of one level.  Not inlined: each kind gets its own register
// allocation instead of the union of all of them.
template <class C>
__device__ __noinline__ bool go(const BatchLevel& L, int cs, int rs, bool new_level, unsigned char* ring,
                                uint64_t* bars, uint32_t& ctr) {
  if (new_level && L.a.src_tma) {
    // the maps were uploaded by a copy, and an earlier batch may have left
    // another map at the same address in the tensor-map cache
    constexpr int nmaps = C::LOAD == SAMPLES ? 1 : 4;
    for (int i = 0; i < nmaps; ++i)
      if ((L.a.src_tma >> i) & 1) ptx::fence_tensormap_acquire(&L.maps.m[i]);
  }
  return run_strip<C>(L.a, L.maps, L.cf, kNoTaps, cs, rs, ring, kStageStride, bars, ctr);
}

// WITH_DD: the DD 13/7 kinds are dispatched too.  Batches without such a
// request run the kernel without them: its smaller switch and call frame
// keep the other kinds 1-2 % faster.
template <bool WITH_DD>
__device__ __forceinline__ bool dispatch(const BatchLevel& L, int cs, int rs, bool nl, unsigned char* ring,
                                         uint64_t* bars, uint32_t& ctr) {
  if constexpr (WITH_DD) {
    switch (L.kind) {
      case BK_DD_F32_FWD: return go<D0>(L, cs, rs, nl, ring, bars, ctr);
      case BK_DD_F32_INV: return go<D1>(L, cs, rs, nl, ring, bars, ctr);
      case BK_DD_F32_FWD_RT: return go<D2>(L, cs, rs, nl, ring, bars, ctr);
      case BK_DD_F32_INV_RT: return go<D3>(L, cs, rs, nl, ring, bars, ctr);
      default: break;
    }
  }
  switch (L.kind) {
    case BK_97_F32_FWD: return go<K0>(L, cs, rs, nl, ring, bars, ctr);
    case BK_97_F32_INV: return go<K1>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_F32_FWD: return go<K2>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_F32_INV: return go<K3>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_I32_FWD: return go<K4>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_I32_INV: return go<K5>(L, cs, rs, nl, ring, bars, ctr);
    case BK_97_F16_FWD: return go<K6>(L, cs, rs, nl, ring, bars, ctr);
    case BK_97_F16_INV: return go<K7>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_F16_FWD: return go<K8>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_F16_INV: return go<K9>(L, cs, rs, nl, ring, bars, ctr);
    case BK_97_F32_FWD_RT: return go<R0>(L, cs, rs, nl, ring, bars, ctr);
    case BK_97_F32_INV_RT: return go<R1>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_F32_FWD_RT: return go<R2>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_F32_INV_RT: return go<R3>(L, cs, rs, nl, ring, bars, ctr);
    case BK_97_F16_FWD_RT: return go<R6>(L, cs, rs, nl, ring, bars, ctr);
    case BK_97_F16_INV_RT: return go<R7>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_F16_FWD_RT: return go<R8>(L, cs, rs, nl, ring, bars, ctr);
    case BK_53_F16_INV_RT: return go<R9>(L, cs, rs, nl, ring, bars, ctr);
  }
  return false;
}

// 12 resident one-warp blocks per SM leave 168 registers a thread: the
// strip functions of the kinds (not inlined, each with its own allocation)
// fit with at most a few bytes of spill in the rarely used ones.
template <bool WITH_DD>
__global__ void __launch_bounds__(32, 12) batch_kernel(const __grid_constant__ BatchParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kMaxStages * kStageStride);
  if (lane == 0) {
    for (int s = 0; s < kMaxStages; ++s) ptx::mbar_init(&bars[s], 32);
    ptx::fence_barrier_init();
  }
  __syncwarp();
  uint32_t chunk_ctr = 0;
  int fenced = -1;  // level whose tensor maps this warp has acquired
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(P.head, 1);
    it = __shfl_sync(kFull, it, 0);
    if (it >= P.nitems) break;
    const BatchItem item = P.items[it];
    const BatchLevel& L = P.levels[item.level];
    const int rs = item.strip / L.a.ncs, cs = item.strip - rs * L.a.ncs;
    bool ok = true;
    if (L.dep_row_base >= 0) {
      const int2 d = P.row_deps[L.row_base + rs];
      ok = wait_rows(P.row_done + L.dep_row_base, d.x, d.y, L.dep_ncs, L.a.spins);
    }
    if (ok) ok = dispatch<WITH_DD>(L, cs, rs, item.level != fenced, smem_raw, bars, chunk_ctr);
    fenced = item.level;
    if (!ok && lane == 0) atomicExch(&P.req_status[L.request], 5 /* DWT_ETIMEOUT */);
    publish_row(P.row_done + L.row_base, rs);
  }
}

// Geometry of a kind for the host (the kernel pointer is the batch kernel's).
template <class C>
void kind_info(KernelInfo* k) {
  *k = KernelInfo{};
  k->hq = C::HQ;
  k->uq = C::UQ;
  k->up = C::Tot::UP;
  k->down = C::Tot::DOWN;
  k->load = (Layout)C::LOAD;
  k->store = (Layout)C::STORE;
  k->box_w = C::ROWE;
  k->box_h = C::ROWS;
  k->smem_bytes = batch_smem_bytes();
  k->fn = reinterpret_cast<const void*>(&batch_kernel<false>);
  k->supported = true;
  k->realign = C::REALIGN;
}

}  // namespace
}  // namespace dev

bool batch_kind_info(int kind, KernelInfo* k) {
  using namespace dev;
  switch (kind) {
    case BK_97_F32_FWD: kind_info<K0>(k); return true;
    case BK_97_F32_INV: kind_info<K1>(k); return true;
    case BK_53_F32_FWD: kind_info<K2>(k); return true;
    case BK_53_F32_INV: kind_info<K3>(k); return true;
    case BK_53_I32_FWD: kind_info<K4>(k); return true;
    case BK_53_I32_INV: kind_info<K5>(k); return true;
    case BK_97_F16_FWD: kind_info<K6>(k); return true;
    case BK_97_F16_INV: kind_info<K7>(k); return true;
    case BK_53_F16_FWD: kind_info<K8>(k); return true;
    case BK_53_F16_INV: kind_info<K9>(k); return true;
    case BK_97_F32_FWD_RT: kind_info<R0>(k); return true;
    case BK_97_F32_INV_RT: kind_info<R1>(k); return true;
    case BK_53_F32_FWD_RT: kind_info<R2>(k); return true;
    case BK_53_F32_INV_RT: kind_info<R3>(k); return true;
    case BK_97_F16_FWD_RT: kind_info<R6>(k); return true;
    case BK_97_F16_INV_RT: kind_info<R7>(k); return true;
    case BK_53_F16_FWD_RT: kind_info<R8>(k); return true;
    case BK_53_F16_INV_RT: kind_info<R9>(k); return true;
    case BK_DD_F32_FWD: kind_info<D0>(k); return true;
    case BK_DD_F32_INV: kind_info<D1>(k); return true;
    case BK_DD_F32_FWD_RT: kind_info<D2>(k); return true;
    case BK_DD_F32_INV_RT: kind_info<D3>(k); return true;
  }
  return false;
}

size_t batch_smem_bytes() {
  return (size_t)kMaxStages * dev::kStageStride + (size_t)kMaxStages * 8;
}

const void* batch_kernel_fn() { return reinterpret_cast<const void*>(&dev::batch_kernel<false>); }

cudaError_t launch_batch(const BatchParams& p, int blocks, bool with_dd, cudaStream_t s) {
  static int configured[64][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const void* fn = with_dd ? reinterpret_cast<const void*>(&dev::batch_kernel<true>)
                           : reinterpret_cast<const void*>(&dev::batch_kernel<false>);
  if (dev >= 0 && dev < 64 && !configured[dev][with_dd]) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes());
    if (e != cudaSuccess) return e;
    configured[dev][with_dd] = 1;
  }
  if (with_dd)
    dev::batch_kernel<true><<<blocks, 32, batch_smem_bytes(), s>>>(p);
  else
    dev::batch_kernel<false><<<blocks, 32, batch_smem_bytes(), s>>>(p);
  return cudaGetLastError();
}

}  // namespace dwt
