// The C ABI of libdwt (include/dwt.h): plans, argument validation, the
// per-level launch sequence, TMA descriptors, lifting coefficients,
// Convolution taps, profiling, host-buffer entry points, batches and the
// autotuner.  Every step of the transform runs in the CUDA kernels of this
// library; this file only prepares and orders launches.
#include "dwt.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "batch.h"
#include "dwt_internal.h"

using namespace dwt;

namespace {

// ---------------------------------------------------------------------------
// Wavelets (Sec. 5)
// ---------------------------------------------------------------------------


struct Lifting {
  int npairs;
  double p1[2], p3[2], u1[2], u3[2];  // taps at sample distance 1 and 3
  double dc;                          // DC gain of the unscaled analysis low-pass
};

Lifting lifting_of(int wl) {
  Lifting L{};
  if (wl == DWT_CDF53) {  // P = -1/2 (1 + z^-1), U = 1/4 (1 + z)
    L.npairs = 1;
    L.p1[0] = -0.5;
    L.u1[0] = 0.25;
    L.dc = 1.0;
  } else if (wl == DWT_CDF97) {
    L.npairs = 2;
    L.p1[0] = kAlpha;
    L.u1[0] = kBeta;
    L.p1[1] = kGamma;
    L.u1[1] = kDelta;
    L.dc = kK97;
  } else {  // DD 13/7: P = 1/16 (z + z^-2) - 9/16 (1 + z^-1), U = 9/32 (1 + z) - 1/32 (z^-1 + z^2)
    L.npairs = 1;
    L.p1[0] = -9.0 / 16.0;
    L.p3[0] = 1.0 / 16.0;
    L.u1[0] = 9.0 / 32.0;
    L.u3[0] = -1.0 / 32.0;
    L.dc = 1.0;
  }
  return L;
}

// Band scaling: JPEG 2000 (low DC gain 1, high Nyquist gain 2) or the
// paper's zeta (low x zeta, high x 1/zeta, zeta = sqrt(2)/K; sqrt(2) for 5/3).
void band_scales(const Lifting& L, int norm, double* lo, double* hi) {
  if (norm == DWT_NORM_ZETA) {
    *lo = std::sqrt(2.0) / L.dc;
    *hi = L.dc / std::sqrt(2.0);
  } else {
    *lo = 1.0 / L.dc;
    *hi = L.dc;
  }
}

// Coefficients of one launch.  A length-1 axis gets zero lifting
// coefficients and unit scaling: the line is left as it is.
Coefs make_coefs(const Lifting& L, int norm, int Wk, int Hk, int pass, bool inverse) {
  Coefs c{};
  const bool h_on = Wk > 1, v_on = Hk > 1;
  for (int k = 0; k < L.npairs; ++k) {
    c.ph1[k] = h_on ? (float)L.p1[k] : 0.f;
    c.ph3[k] = h_on ? (float)L.p3[k] : 0.f;
    c.uh1[k] = h_on ? (float)L.u1[k] : 0.f;
    c.uh3[k] = h_on ? (float)L.u3[k] : 0.f;
    c.pv1[k] = v_on ? (float)L.p1[k] : 0.f;
    c.pv3[k] = v_on ? (float)L.p3[k] : 0.f;
    c.uv1[k] = v_on ? (float)L.u1[k] : 0.f;
    c.uv3[k] = v_on ? (float)L.u3[k] : 0.f;
  }
  double lo, hi;
  band_scales(L, norm, &lo, &hi);
  const double lo_h = h_on ? lo : 1.0, hi_h = h_on ? hi : 1.0;
  const double lo_v = v_on ? lo : 1.0, hi_v = v_on ? hi : 1.0;
  double s[4];
  if (pass == PASS_VERT) {
    s[0] = s[1] = lo_v;
    s[2] = s[3] = hi_v;
  } else if (pass == PASS_HORZ) {
    s[0] = s[2] = lo_h;
    s[1] = s[3] = hi_h;
  } else {
    s[0] = lo_v * lo_h;
    s[1] = lo_v * hi_h;
    s[2] = hi_v * lo_h;
    s[3] = hi_v * hi_h;
  }
  for (int i = 0; i < 4; ++i) c.scale[i] = (float)(inverse ? 1.0 / s[i] : s[i]);
  c.h_on = h_on;
  c.v_on = v_on;
  return c;
}

// 1-D polyphase matrix of the whole factorisation, as Laurent polynomials in
// the quad offset (index + 4 covers offsets -4..4).
struct Poly {
  double c[9] = {0};
};
Poly pmul(const Poly& a, const Poly& b) {
  Poly r;
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) {
      const int k = i + j - 4;
      if (a.c[i] != 0 && b.c[j] != 0 && k >= 0 && k < 9) r.c[k] += a.c[i] * b.c[j];
    }
  return r;
}
void padd(Poly& a, const Poly& b, double s) {
  for (int i = 0; i < 9; ++i) a.c[i] += s * b.c[i];
}

// Predict P (reads even quads at offsets 0, +1 and, degree 3, -1, +2) and
// update U (odd quads at -1, 0 and -2, +1).
Poly pred_poly(const Lifting& L, int k) {
  Poly p;
  p.c[4] = p.c[5] = L.p1[k];
  p.c[3] = p.c[6] = L.p3[k];
  return p;
}
Poly upd_poly(const Lifting& L, int k) {
  Poly u;
  u.c[3] = u.c[4] = L.u1[k];
  u.c[2] = u.c[5] = L.u3[k];
  return u;
}

// m[out][in]: forward (L,H) <- (even,odd); inverse (even,odd) <- (L,H).
void polyphase_1d(const Lifting& L, int norm, bool on, bool inverse, Poly m[2][2]) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) m[i][j] = Poly();
  double lo, hi;
  band_scales(L, norm, &lo, &hi);
  if (!on) {
    m[0][0].c[4] = m[1][1].c[4] = 1.0;
    return;
  }
  if (!inverse) {
    m[0][0].c[4] = m[1][1].c[4] = 1.0;
    for (int k = 0; k < L.npairs; ++k) {
      const Poly P = pred_poly(L, k), U = upd_poly(L, k);
      for (int j = 0; j < 2; ++j) padd(m[1][j], pmul(P, m[0][j]), 1.0);  // H += P L
      for (int j = 0; j < 2; ++j) padd(m[0][j], pmul(U, m[1][j]), 1.0);  // L += U H
    }
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 9; ++i) {
        m[0][j].c[i] *= lo;
        m[1][j].c[i] *= hi;
      }
  } else {
    m[0][0].c[4] = 1.0 / lo;
    m[1][1].c[4] = 1.0 / hi;
    for (int k = L.npairs - 1; k >= 0; --k) {
      const Poly P = pred_poly(L, k), U = upd_poly(L, k);
      for (int j = 0; j < 2; ++j) padd(m[0][j], pmul(U, m[1][j]), -1.0);  // even -= U odd
      for (int j = 0; j < 2; ++j) padd(m[1][j], pmul(P, m[0][j]), -1.0);  // odd -= P even
    }
  }
}

bool conv_taps(const Lifting& L, int norm, int Wk, int Hk, bool inverse, ConvTaps* t) {
  Poly v[2][2], h[2][2];
  polyphase_1d(L, norm, Hk > 1, inverse, v);
  polyphase_1d(L, norm, Wk > 1, inverse, h);
  constexpr int R = kConvReach, N = 2 * kConvReach + 1;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int i = 0; i < 9; ++i)
        if ((i < 4 - R || i > 4 + R) && (std::fabs(v[a][b].c[i]) > 1e-12 || std::fabs(h[a][b].c[i]) > 1e-12))
          return false;  // reach beyond the kernel's tap table
  for (int so = 0; so < 2; ++so)
    for (int sx = 0; sx < 2; ++sx)
      for (int ti = 0; ti < 2; ++ti)
        for (int tx = 0; tx < 2; ++tx)
          for (int dy = 0; dy < N; ++dy)
            for (int dx = 0; dx < N; ++dx)
              t->t[so][sx][ti][tx][dy][dx] = (float)(v[so][ti].c[dy + 4 - R] * h[sx][tx].c[dx + 4 - R]);
  return true;
}

// ---------------------------------------------------------------------------
// Kernel lookup, geometry, TMA
// ---------------------------------------------------------------------------
const GroupFn kGroups[] = {group_sweldens,   group_iwahashi,   group_iwahashi_s,  group_explosive,
                           group_explosive_s, group_monolithic, group_monolithic_s, group_polyphase,
                           group_polyphase_s, group_convolution, group_rowcol};

bool find_kernel(const LaunchKey& k, int ns, KernelInfo* info) {
  for (GroupFn g : kGroups) {
    cudaError_t e = cudaSuccess;
    if (g(k, ns, info, nullptr, &e)) return true;
  }
  return false;
}

cudaError_t call_kernel(const LaunchKey& k, int ns, const LaunchCall& call) {
  for (GroupFn g : kGroups) {
    cudaError_t e = cudaSuccess;
    if (g(k, ns, nullptr, &call, &e)) return e;
  }
  return cudaErrorInvalidDeviceFunction;
}

const TailFn kTails[] = {tail_sweldens,   tail_iwahashi,    tail_iwahashi_s, tail_explosive, tail_explosive_s,
                         tail_monolithic, tail_monolithic_s, tail_polyphase, tail_polyphase_s};

bool find_tail(const LaunchKey& k, TailInfo* info) {
  for (TailFn g : kTails) {
    cudaError_t e = cudaSuccess;
    if (g(k, info, nullptr, &e)) return true;
  }
  return false;
}

cudaError_t call_tail(const LaunchKey& k, const TailCall& call) {
  for (TailFn g : kTails) {
    cudaError_t e = cudaSuccess;
    if (g(k, nullptr, &call, &e)) return e;
  }
  return cudaErrorInvalidDeviceFunction;
}

struct Occ {
  int sms = 0;
  int per_sm = 0;
};

// Occupancy cache: a fixed open-addressing table (no heap allocation, so
// the entry point that allocates nothing can use it too).  When it is full,
// further keys are computed on every call instead of cached.
struct OccEntry {
  const void* fn;
  int device;
  size_t smem;
  Occ occ;
};
constexpr int kOccSlots = 1024;
std::mutex g_occ_mu;
OccEntry g_occ[kOccSlots];

// Resident blocks of `threads` threads (one warp by default) for kernel
// `fn` with `smem` bytes of dynamic shared memory per block.  A kernel is
// always queried with the same block size, so `fn` identifies it.
Occ occupancy(const void* fn, size_t smem, int device, int threads = kWarpsPerCta * 32) {
  std::lock_guard<std::mutex> lk(g_occ_mu);
  const size_t hsh = (reinterpret_cast<uintptr_t>(fn) >> 4) * 31u + (size_t)device * 131u + smem;
  int free_slot = -1;
  for (int i = 0; i < 16; ++i) {
    OccEntry& e = g_occ[(hsh + i) % kOccSlots];
    if (e.fn == fn && e.device == device && e.smem == smem) return e.occ;
    if (!e.fn) {
      free_slot = (int)((hsh + i) % kOccSlots);
      break;
    }
  }
  Occ o;
  cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  // the largest dynamic allocation the kernel can take: the opt-in limit
  // less its static shared memory.  A failed call is cleared here, so that
  // it cannot surface later as another call's error.
  cudaFuncAttributes fa{};
  const int stat = cudaFuncGetAttributes(&fa, fn) == cudaSuccess ? (int)fa.sharedSizeBytes : 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin > stat ? optin - stat : (int)smem) != cudaSuccess)
    cudaGetLastError();
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, fn, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    o.per_sm = 1;
  }
  o.sms = std::max(o.sms, 1);
  o.per_sm = std::max(o.per_sm, 1);
  if (free_slot >= 0) g_occ[free_slot] = OccEntry{fn, device, smem, o};
  return o;
}

// ---------------------------------------------------------------------------
// Wait limits and failure injection
// ---------------------------------------------------------------------------
std::atomic<uint32_t> g_ring_probes{kDefaultRingProbes};
std::atomic<uint32_t> g_dep_spins{kDefaultDepSpins};

// Host-side failure injection for tests of the error paths (dwt_debug_inject):
// each kind lets `skip` events pass, then acts on the next `count`.
struct Injection {
  int skip = 0, count = 0;
};
std::mutex g_inject_mu;
Injection g_inject[4];

bool injected(int what) {
  std::lock_guard<std::mutex> lk(g_inject_mu);
  Injection& j = g_inject[what];
  if (j.count <= 0) return false;
  if (j.skip > 0) {
    --j.skip;
    return false;
  }
  --j.count;
  return true;
}

// Every device or page-locked allocation of the library goes through these,
// so that an injected allocation failure reaches each of them.
cudaError_t dev_malloc(void** p, size_t n) {
  if (injected(DWT_INJECT_ENOMEM)) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, n);
}
cudaError_t host_malloc(void** p, size_t n) {
  if (injected(DWT_INJECT_ENOMEM)) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, n);
}
cudaError_t pool_malloc(void** p, size_t n, cudaMemPool_t pool, cudaStream_t s) {
  if (injected(DWT_INJECT_ENOMEM)) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(p, n, pool, s);
}

// The wait limits and the injected hold of a single-image launch; `flag` is
// a device word that nothing sets.
void set_waits(LevelArgs& a, const int* flag) {
  a.probes = g_ring_probes.load();
  a.spins = g_dep_spins.load();
  a.hold = injected(DWT_INJECT_HOLD) ? flag : nullptr;
}
Occ occupancy(const KernelInfo& ki, int device) { return occupancy(ki.fn, ki.smem_bytes, device); }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
typedef CUresult (*AddrRangeFn)(CUdeviceptr*, size_t*, CUdeviceptr);

template <class F>
F driver_fn(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(p);
}

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = driver_fn<EncodeTiledFn>("cuTensorMapEncodeTiled");
  return fn;
}
AddrRangeFn addr_range_fn() {
  static AddrRangeFn fn = driver_fn<AddrRangeFn>("cuMemGetAddressRange");
  return fn;
}

bool encode_2d(CUtensorMap* m, int dtype, const void* base, int w, int h, size_t pitch_bytes,
               int boxw, int boxh) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || w < 1 || h < 1 || (reinterpret_cast<uintptr_t>(base) & 15) || (pitch_bytes & 15))
    return false;
  const CUtensorMapDataType dt = dtype == F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : dtype == F16S ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                 : CU_TENSOR_MAP_DATA_TYPE_INT32;
  cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
  cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
  cuuint32_t box[2] = {(cuuint32_t)boxw, (cuuint32_t)boxh};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of a level's source planes.  Returns the planes whose map is
// valid (bit p for plane p): the kernels load those by TMA and copy the
// others (a plane whose base or row pitch is not 16-byte aligned, as the HL
// and HH bands at column ceil(w/2) of most odd-width coefficient planes).
//
// A subband plane whose rows are 16-byte multiples but whose first element
// is not 16-byte aligned (HL and HH at column ceil(w/2) of padded rows)
// gets a map anchored at the aligned column before it, `off` elements
// earlier and `off` columns wider, when the kernel takes such planes
// (ki.realign); a.src_off records the offset.  Only HL and HH (the odd
// column parity) are realigned, and both must share the offset (one box
// geometry in the kernel); LL and LH start at column 0 of their rows.
int encode_level_maps(TmaMaps* maps, int dtype, LevelArgs& a, const KernelInfo& ki, size_t es) {
  std::memset(maps, 0, sizeof *maps);
  for (int i = 0; i < 4; ++i) a.src_off[i] = 0;
  if (a.W < 2 || a.H < 2) return 0;
  if (ki.load == SAMPLES)
    return encode_2d(&maps->m[0], dtype, a.src[0], a.W, a.H, (size_t)a.src_pitch[0] * es, ki.box_w, ki.box_h)
               ? 1
               : 0;
  const int pw[4] = {a.cw, a.fw, a.cw, a.fw}, ph[4] = {a.ch, a.ch, a.fh, a.fh};
  // only the odd-parity planes (HL, HH) are realigned: the even ones start
  // at column 0 of their rows
  int off[4] = {0, 0, 0, 0};
  if (ki.realign)
    for (int i = 1; i < 4; i += 2) {
      const uintptr_t b = reinterpret_cast<uintptr_t>(a.src[i]);
      if ((((size_t)a.src_pitch[i] * es) & 15) == 0 && b % es == 0) off[i] = (int)((b & 15) / es);
    }
  if (off[1] != off[3]) off[1] = off[3] = 0;
  int mask = 0;
  for (int i = 0; i < 4; ++i) {
    const void* base = static_cast<const char*>(a.src[i]) - (size_t)off[i] * es;
    if (encode_2d(&maps->m[i], dtype, base, pw[i] + off[i], ph[i], (size_t)a.src_pitch[i] * es, ki.box_w, ki.box_h)) {
      mask |= 1 << i;
      a.src_off[i] = off[i];
    }
  }
  // realigned only if both odd-parity planes got their maps
  if (a.src_off[1] != a.src_off[3]) a.src_off[1] = a.src_off[3] = 0;
  return mask;
}

size_t elem_size(int dtype) { return dtype == F16S ? 2 : 4; }

// Strip height of batched requests whose plan has no tile set by the caller.
// The persistent kernel pays per strip (a dependency poll, a descriptor
// read, the halo), so it favours taller strips than the per-level kernels:
// on 256 images of 256-4096 per side, 48-row strips with the full ring
// match the best tile found per size class (4.39 against 4.39 ms), where
// the per-level default (10 rows, 2 stages) takes 7.79 ms.
constexpr int kBatchStripRows = 48;

// Largest side a plan accepts: quad, strip and row counts and the halvings
// of a side stay far from int overflow.
constexpr int kMaxSide = 1 << 28;

// Levels whose input has at most this many samples run in the fused tail
// (tile_kernel.cuh) by default: one launch for all of them.  Measured on
// one 9/7 level alone, the tile kernel beats the streaming kernel up to
// 512 x 512 (5.7 against 6.2 us forward, 6.2 against 7.9 inverse) and loses
// from 1024 x 1024 (forward 8.2 against 7.4 us) and 2048 x 2048 (18.5
// against 10.8 us), where it is bound by instruction issue with a tile's
// halo recomputed; each fused level costs about 4.6 us (a grid barrier
// and one tile's chain of steps) against 6-8 us per streaming launch.
constexpr long long kDefaultFusePx = 512LL * 512LL;

// Quad rows per strip.  Strips of about ten rows keep several waves of
// one-warp blocks in flight, so the block scheduler balances SMs that
// progress at different rates, while the vertical halo re-reads hit L2
// (vertically adjacent strips run at the same time).  A level that fills
// the GPU fewer than four times at that height is governed by its last
// wave: it takes the height (2..32 rows) that minimises the number of waves
// times the rows each strip streams (its own, the halo `halo` and the
// padding to whole chunks of `chunk` rows).
int strip_height(int target, int ch, int ncs, int cap_warps, int halo, int chunk) {
  auto strips = [&](int T) { return (long long)ncs * ((ch + T - 1) / T); };
  if (strips(target) >= 4LL * cap_warps) return target;
  int best = 2;
  long long best_cost = -1;
  for (int T = 2; T <= 32; ++T) {
    const long long waves = (strips(T) + cap_warps - 1) / cap_warps;
    const long long rows = ((std::min(T, ch) + halo + chunk - 1) / chunk) * chunk;
    const long long cost = waves * rows;
    if (best_cost < 0 || cost < best_cost) {
      best = T;
      best_cost = cost;
    }
  }
  return best;
}

// Default strip height of a scheme.  Ten quadruple rows in general.  Every
// strip also recomputes the rows of its vertical halo, so schemes that
// spend many instructions per row take taller strips: the three-step
// schemes (Iwahashi, Explosive and their starred forms) with two lifting
// pairs or degree-3 steps (8-10 halo rows) and the unstarred Polyphase take
// 32, Convolution 32 (5/3) or 48 (9/7), and Monolithic, Monolithic* and
// Polyphase* with DD 13/7 (a 6-row halo of merged degree-3 stencils) 24.
// Measured on 8192^2 and 16384^2 at 10-48 rows: Polyphase 9/7 at 8192^2
// one level takes 164 us at 10 rows and 144 us at 32, Convolution 9/7 492
// us at 10 and 356 us at 48; the schemes left at 10 are fastest there.
int default_strip_rows(int scheme, int wavelet) {
  const bool three_step = scheme == DWT_IWAHASHI || scheme == DWT_IWAHASHI_S || scheme == DWT_EXPLOSIVE ||
                          scheme == DWT_EXPLOSIVE_S;
  if (three_step && wavelet != DWT_CDF53) return 32;
  if (scheme == DWT_POLYPHASE) return 32;
  if (scheme == DWT_CONVOLUTION) return wavelet == DWT_CDF53 ? 32 : 48;
  if (wavelet == DWT_DD137 && (scheme == DWT_MONOLITHIC || scheme == DWT_MONOLITHIC_S || scheme == DWT_POLYPHASE_S))
    return 24;
  return kDefaultStripRows;
}

// Rows of strips one resident wave holds, for the kernels' dealt strip-row
// order (strip_coords): vertically adjacent strips then run in consecutive
// waves and the rows they share come from L2.  Only tall strips (24 rows or
// more) use it: their neighbours, run in the same wave, read the shared
// rows a long strip apart and miss L2 (8192^2 Iwahashi 9/7 at 32 rows: 358
// MB of DRAM reads against 312 MB dealt, and 3-7 % faster at 16384^2).
// Short strips share rows a few row steps apart in the same wave, which
// already hits L2; dealt, they read 2 % more from DRAM.  0: row by row.
int wave_rows(const LevelArgs& a, int cap) {
  if (a.T < 24) return 0;
  return std::max(1, cap / std::max(1, a.ncs > 2 ? a.ncs - 2 : a.ncs));
}

// Chunk rows (quad rows per ring stage) of a kernel.
int chunk_rows(const KernelInfo& ki) { return ki.load == SAMPLES ? ki.box_h / 2 : ki.box_h; }

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Whole-sample symmetric extension of index i on a line of n >= 2 samples
// (period 2(n - 1)), as the kernels apply it.
int host_mirror(int i, int n) {
  const int period = 2 * (n - 1);
  i %= period;
  if (i < 0) i += period;
  return i >= n ? period - i : i;
}

}  // namespace

// ---------------------------------------------------------------------------
// Plans
// ---------------------------------------------------------------------------
struct ProfSlot {
  std::string name;
  int launches = 0;
  double ms = 0, bytes = 0;
};
struct ProfRec {
  int slot;
  cudaEvent_t a, b;
  double bytes;
};

struct dwt_plan_s {
  int w = 0, h = 0, levels = 0, wavelet = 0, dtype = 0;
  int scheme = DWT_AUTO, auto_scheme = -1, norm = DWT_NORM_JPEG2000;
  int device = 0;
  size_t es = 4;
  std::vector<int> W, H;
  // LL_k of every level but the last, each in its own buffer
  std::vector<void*> ll;
  std::vector<size_t> ll_pitch;

  void* tmp = nullptr;
  size_t tmp_pitch = 0;
  void* stage_in = nullptr;
  void* stage_out = nullptr;
  size_t stage_pitch = 0;
  int* d_status = nullptr;
  cudaStream_t last_stream = nullptr;
  bool profiling = false;
  std::vector<ProfSlot> slots;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  int nstages = kDefaultStages;
  int strip_rows = 0;  // 0: the default of the scheme a call runs (default_strip_rows)
  long long fuse_px = -1;  // fused-tail threshold (samples per level input); -1 default, 0 off
  bool tile_set = false;  // the caller chose the tile: the autotuner's choice does not apply
  bool tuned = false;     // the autotuner cache was consulted
  std::mutex mu;
};

namespace {

dwt_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return DWT_OK;
  if (e == cudaErrorMemoryAllocation) return DWT_ENOMEM;
  return DWT_ECUDA;
}

// ---- autotune cache (text lines "key scheme") ----------------------------
std::mutex g_cache_mu;

std::string gpu_name(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
  std::string s = prop.name;
  for (char& c : s)
    if (c == ' ') c = '_';
  return s;
}

std::string cache_key(const dwt_plan_s* p) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s|wl%d|dt%d|%dx%d|L%d", gpu_name(p->device).c_str(), p->wavelet,
                p->dtype, p->w, p->h, p->levels);
  return buf;
}

// One autotuner choice: scheme and tile (strip rows, ring stages).
struct Tuned {
  int scheme = -1, rows = 0, stages = 0;
};

Tuned cache_lookup(const std::string& key) {
  Tuned t;
  const char* path = std::getenv("DWT_AUTOTUNE_CACHE");
  if (!path) return t;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  FILE* f = std::fopen(path, "r");
  if (!f) return t;
  char line[512], k[256];
  while (std::fgets(line, sizeof line, f)) {
    Tuned v;
    if (std::sscanf(line, "%255s %d %d %d", k, &v.scheme, &v.rows, &v.stages) >= 2 && key == k) t = v;
  }
  std::fclose(f);
  return t;
}

void cache_store(const std::string& key, const Tuned& t) {
  const char* path = std::getenv("DWT_AUTOTUNE_CACHE");
  if (!path) return;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d\n", key.c_str(), t.scheme, t.rows, t.stages);
  std::fclose(f);
}

int default_scheme(const dwt_plan_s* p) {
  return p->dtype == DWT_I32 ? DWT_SWELDENS : DWT_MONOLITHIC_S;
}

bool scheme_supported(int wavelet, int dtype, int scheme) {
  if (scheme <= DWT_AUTO || scheme >= NUM_SCHEMES) return false;
  // int32: the JPEG 2000 reversible 5/3 (row-column or single-loop), or the
  // reversible integer Iwahashi lifting, a transform of its own
  if (dtype == DWT_I32)
    return wavelet == DWT_CDF53 && (scheme == DWT_ROWCOL || scheme == DWT_SWELDENS || scheme == DWT_IWAHASHI);
  // DD 13/7 (degree-3 pairs): float32, every scheme
  if (wavelet == DWT_DD137) return dtype == DWT_F32;
  return true;
}

// Schemes the autotuner may choose among: every scheme of the plan's
// wavelet and storage type, except that int32 stays with the JPEG 2000
// transform (the integer Iwahashi lifting gives other coefficients and is
// only run when a caller selects it).
bool tunable(int wavelet, int dtype, int scheme) {
  return scheme_supported(wavelet, dtype, scheme) && !(dtype == DWT_I32 && scheme == DWT_IWAHASHI);
}

// Applies a cached autotuner choice once per plan: the scheme when the
// caller left it to DWT_AUTO, the tile when the caller did not set one.
void apply_cache(dwt_plan_s* p) {
  if (p->tuned) return;
  p->tuned = true;
  const Tuned t = cache_lookup(cache_key(p));
  if (p->auto_scheme < 0)
    p->auto_scheme = tunable(p->wavelet, p->dtype, t.scheme) ? t.scheme : default_scheme(p);
  if (!p->tile_set && t.rows > 0 && t.stages >= 1 && t.stages <= kMaxStages) {
    p->strip_rows = t.rows;
    p->nstages = t.stages;
  }
}

int resolve_scheme(dwt_plan_s* p) {
  apply_cache(p);
  return p->scheme != DWT_AUTO ? p->scheme : p->auto_scheme;
}

bool device_pointer_ok(const void* ptr, size_t extent, int device) {
  if (!ptr) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type == cudaMemoryTypeDevice) {
    if (attr.device != device) return false;
  } else if (attr.type != cudaMemoryTypeManaged) {
    return false;
  }
  if (AddrRangeFn fn = addr_range_fn()) {
    CUdeviceptr base = 0;
    size_t size = 0;
    if (fn(&base, &size, reinterpret_cast<CUdeviceptr>(ptr)) == CUDA_SUCCESS) {
      const uintptr_t lo = reinterpret_cast<uintptr_t>(ptr);
      if (lo + extent > (uintptr_t)base + size) return false;
    }
  }
  return true;
}

size_t plane_extent(int w, int h, size_t pitch, size_t es) {
  return (size_t)(h - 1) * pitch + (size_t)w * es;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

cudaEvent_t take_event(dwt_plan_s* p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int slot_of(dwt_plan_s* p, const std::string& name) {
  for (size_t i = 0; i < p->slots.size(); ++i)
    if (p->slots[i].name == name) return (int)i;
  p->slots.push_back(ProfSlot{name});
  return (int)p->slots.size() - 1;
}

// Dynamic shared memory of a level kernel with `nstages` ring stages, from
// its info for `info_stages` stages.
size_t smem_with_stages(const KernelInfo& ki, int info_stages, int nstages) {
  const size_t bars = (size_t)kWarpsPerCta * kMaxStages * 8;
  return (ki.smem_bytes - bars) / info_stages * nstages + bars;
}

// The tile a single-image launch uses: device, ring depth and strip height
// (0: the default of the scheme).
struct Tile {
  int device, nstages, strip_rows;
};

// Strips of one level: column strips, strip height, strip rows and ring
// depth, for the kernel of `key`.
dwt_status level_geometry(const Tile& t, const LaunchKey& key, LevelArgs& a, KernelInfo& ki) {
  if (!find_kernel(key, t.nstages, &ki)) return DWT_EUNSUPPORTED;
  const Occ oc = occupancy(ki, t.device);
  const int cap = oc.sms * oc.per_sm * kWarpsPerCta;  // resident warps (strips)
  // one strip per resident warp when the level is large enough: a single
  // wave, with strips as tall as that allows (less vertical halo)
  a.ncs = (a.cw + ki.uq - 1) / ki.uq;
  const int target = t.strip_rows > 0 ? t.strip_rows : default_strip_rows(key.scheme, key.wavelet);
  a.T = strip_height(target, a.ch, a.ncs, cap, ki.up + ki.down, chunk_rows(ki));
  a.nrs = (a.ch + a.T - 1) / a.T;
  a.wave_rows = wave_rows(a, cap);
  // a level that does not fill the GPU once is latency-bound: a deeper
  // ring lets each (short) strip issue all its chunk loads at once, as long
  // as the level still fits one wave with the larger shared-memory ring
  a.nstages = t.nstages;
  if (t.nstages < kMaxStages && (long long)a.ncs * a.nrs < cap) {
    const Occ deep = occupancy(ki.fn, smem_with_stages(ki, t.nstages, kMaxStages), t.device);
    if ((long long)a.ncs * a.nrs <= (long long)deep.sms * deep.per_sm * kWarpsPerCta) a.nstages = kMaxStages;
  }
  return DWT_OK;
}

// One launch: geometry, descriptors, optional timing events.
dwt_status launch(dwt_plan_s* p, const LaunchKey& key, LevelArgs& a, const Coefs& cf,
                  const ConvTaps& ct, cudaStream_t s, const char* slot) {
  KernelInfo ki{};
  const dwt_status g = level_geometry(Tile{p->device, p->nstages, p->strip_rows}, key, a, ki);
  if (g != DWT_OK) return g;
  a.status = p->d_status;
  set_waits(a, p->d_status + 1);

  TmaMaps maps;
  a.src_tma = encode_level_maps(&maps, p->dtype, a, ki, p->es);

  ProfRec rec{-1, nullptr, nullptr, 0.0};
  if (p->profiling) {
    rec.slot = slot_of(p, slot);
    rec.a = take_event(p);
    rec.b = take_event(p);
    rec.bytes = 2.0 * a.W * (double)a.H * p->es;
    cudaEventRecord(rec.a, s);
  }
  LaunchCall call{&a, &maps, &cf, &ct, s};
  cudaError_t e = call_kernel(key, p->nstages, call);
  if (p->profiling) {
    cudaEventRecord(rec.b, s);
    p->pending.push_back(rec);
  }
  return from_cuda(e);
}

void level_dims(const dwt_plan_s* p, int k, LevelArgs& a) {
  a.W = p->W[k];
  a.H = p->H[k];
  a.cw = (a.W + 1) / 2;
  a.ch = (a.H + 1) / 2;
  a.fw = a.W / 2;
  a.fh = a.H / 2;
}

dwt_status ensure_tmp(dwt_plan_s* p) {
  if (p->tmp) return DWT_OK;
  p->tmp_pitch = round_up((size_t)p->w * p->es, 128);
  return from_cuda(dev_malloc(&p->tmp, p->tmp_pitch * p->h));
}

// Which strip rows of level d (the level whose output level a reads) each
// strip row of level a needs: the rows its chunks load (the strip plus
// halo, padded to whole chunks), mirrored the way the kernel mirrors them,
// mapped to the strip rows of d that write them.  In-range rows map
// monotonically (their span is exact); only the few halo rows beyond an
// edge are mirrored one by one.  out[rs] = (first, last) for every rs < a.nrs.
void row_dependencies(const LevelArgs& a, const LevelArgs& d, const KernelInfo& ki, bool inverse, int2* out) {
  const int CH = chunk_rows(ki);
  // forward: sample rows of the level = LL quad rows of the level before,
  // written by its strip row y / T; inverse: LL plane rows = sample rows
  // of the coarser level's output, written by its strip row y / (2 T)
  const int n = inverse ? a.ch : a.H;
  const int per = inverse ? 2 * d.T : d.T;
  auto row_of = [&](int y) {
    int ym;
    if (inverse) ym = a.H == 1 ? 0 : (y >= 0 && y < a.ch) ? y : (host_mirror(2 * y, a.H) >> 1);
    else ym = a.H == 1 ? 0 : host_mirror(y, a.H);
    return ym / per;
  };
  for (int rs = 0; rs < a.nrs; ++rs) {
    const int q0 = rs * a.T;
    const int rows_out = std::min(a.T, a.ch - q0);
    const int nchunks = (rows_out + ki.up + ki.down + CH - 1) / CH;
    const int y0 = q0 - ki.up, y1 = y0 + nchunks * CH;                 // quad rows loaded
    const int r0 = inverse ? y0 : 2 * y0, r1 = inverse ? y1 : 2 * y1;  // rows of the read plane
    int lo = INT32_MAX, hi = -1;
    const int in0 = std::max(r0, 0), in1 = std::min(r1, n);
    if (in0 < in1) {
      lo = in0 / per;
      hi = (in1 - 1) / per;
    }
    for (int y = r0; y < std::min(r1, 0); ++y) {
      lo = std::min(lo, row_of(y));
      hi = std::max(hi, row_of(y));
    }
    for (int y = std::max(r0, n); y < r1; ++y) {
      lo = std::min(lo, row_of(y));
      hi = std::max(hi, row_of(y));
    }
    out[rs] = make_int2(std::max(lo, 0), std::min(hi, d.nrs - 1));
  }
}

// Where level k of a transform reads and writes (Mallat layout): the four
// subband planes inside the coefficient buffer, with LL_k in the buffer
// ll[k] (pitch llp[k] bytes) except at the coarsest level, and the level's
// sample plane (the image at level 0, LL_{k-1} above).  Every level has its
// own LL buffer (about w*h/3 elements in all): in batches the levels of an
// image overlap, so no level may overwrite data another level still reads.
struct LevelIO {
  const void* band[4];
  long long bpitch[4];
  const void* samples;
  long long spitch;
};

LevelIO level_io(const dwt_plan_s* p, bool inverse, int k, const LevelArgs& a, const void* src,
                 size_t src_pitch, const void* dst, size_t dst_pitch, void* const* ll, const size_t* llp) {
  const size_t es = p->es;
  LevelIO io;
  const void* coef = inverse ? src : dst;
  const size_t cp = inverse ? src_pitch : dst_pitch;
  const char* cb = static_cast<const char*>(coef);
  io.band[1] = cb + a.cw * es;
  io.band[2] = cb + a.ch * cp;
  io.band[3] = cb + a.ch * cp + a.cw * es;
  for (int i = 1; i < 4; ++i) io.bpitch[i] = (long long)(cp / es);
  if (k == p->levels - 1) {
    io.band[0] = coef;
    io.bpitch[0] = (long long)(cp / es);
  } else {
    io.band[0] = ll[k];
    io.bpitch[0] = (long long)(llp[k] / es);
  }
  if (k == 0) {
    io.samples = inverse ? dst : src;
    io.spitch = (long long)((inverse ? dst_pitch : src_pitch) / es);
  } else {
    io.samples = ll[k - 1];
    io.spitch = (long long)(llp[k - 1] / es);
  }
  return io;
}

// Sources and destinations of one fused (single-launch) level.
void fused_io(const LevelIO& io, bool inverse, LevelArgs& a) {
  if (!inverse) {
    a.src[0] = io.samples;
    a.src_pitch[0] = io.spitch;
    for (int i = 0; i < 4; ++i) {
      a.dst[i] = const_cast<void*>(io.band[i]);
      a.dst_pitch[i] = io.bpitch[i];
    }
  } else {
    for (int i = 0; i < 4; ++i) {
      a.src[i] = io.band[i];
      a.src_pitch[i] = io.bpitch[i];
    }
    a.dst[0] = const_cast<void*>(io.samples);
    a.dst_pitch[0] = io.spitch;
  }
}

// A plan's own device memory (status word, one LL buffer per level), made on
// its first single-image call: plans used only in batches never allocate.
// The status allocation holds four words: the status, a flag that nothing
// sets (the injected hold of dwt_debug_inject waits on it), the fused
// tail's grid-barrier counter and a spare.
dwt_status ensure_device(dwt_plan_s* p) {
  cudaError_t e = cudaSuccess;
  if (!p->d_status) {
    e = dev_malloc(reinterpret_cast<void**>(&p->d_status), 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, 4 * sizeof(int));
    if (e != cudaSuccess) {
      cudaFree(p->d_status);
      p->d_status = nullptr;
      return from_cuda(e);
    }
  }
  if (p->levels >= 2 && p->ll.empty()) {
    for (int k = 0; k + 1 < p->levels; ++k) {
      const size_t pitch = round_up((size_t)p->W[k + 1] * p->es, 128);
      void* q = nullptr;
      e = dev_malloc(&q, pitch * p->H[k + 1]);
      if (e != cudaSuccess) {
        for (void* r : p->ll) cudaFree(r);
        p->ll.clear();
        p->ll_pitch.clear();
        return from_cuda(e);
      }
      p->ll.push_back(q);
      p->ll_pitch.push_back(pitch);
    }
  }
  return DWT_OK;
}

// Checks shared by every call that transforms one image with a plan.
dwt_status check_buffers(const dwt_plan_s* p, const void* src, size_t src_pitch, const void* dst,
                         size_t dst_pitch) {
  const size_t es = p->es;
  if (src_pitch < (size_t)p->w * es || dst_pitch < (size_t)p->w * es || src_pitch % es ||
      dst_pitch % es)
    return DWT_EINVAL;
  // samples are accessed whole: the planes must start on an element boundary
  if (reinterpret_cast<uintptr_t>(src) % es || reinterpret_cast<uintptr_t>(dst) % es) return DWT_EINVAL;
  const size_t nsrc = plane_extent(p->w, p->h, src_pitch, es);
  const size_t ndst = plane_extent(p->w, p->h, dst_pitch, es);
  if (!device_pointer_ok(src, nsrc, p->device) || !device_pointer_ok(dst, ndst, p->device))
    return DWT_EINVAL;
  if (overlaps(src, nsrc, dst, ndst)) return DWT_EINVAL;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device) return DWT_EINVAL;
  return DWT_OK;
}

// One level of a single-image call with the streaming kernels: the fused
// scheme in one launch, or the row-column baseline's two passes.
dwt_status run_level(dwt_plan_s* p, bool inverse, int k, int scheme, const Lifting& L, const void* src,
                     size_t src_pitch, void* dst, size_t dst_pitch, void* const* ll, const size_t* llp,
                     cudaStream_t s) {
  const size_t es = p->es;
  char slot[32];
  LevelArgs a{};
  level_dims(p, k, a);
  const LevelIO io = level_io(p, inverse, k, a, src, src_pitch, dst, dst_pitch, ll, llp);
  const void* const* band = io.band;
  const long long* bpitch = io.bpitch;
  const void* samples = io.samples;
  const long long spitch = io.spitch;
  const Coefs cf = make_coefs(L, p->norm, a.W, a.H, PASS_FUSED, inverse);
  ConvTaps ct;
  std::memset(&ct, 0, sizeof ct);
  if (scheme == DWT_CONVOLUTION && !conv_taps(L, p->norm, a.W, a.H, inverse, &ct)) return DWT_EUNSUPPORTED;
  if (scheme != DWT_ROWCOL) {
    LaunchKey key{p->wavelet, p->dtype, scheme, PASS_FUSED, inverse ? 1 : 0,
                  p->norm == DWT_NORM_JPEG2000 && a.W >= 2 && a.H >= 2 ? 1 : 0};
    fused_io(io, inverse, a);
    std::snprintf(slot, sizeof slot, "%s/L%d", inverse ? "inv" : "fwd", k);
    return launch(p, key, a, cf, ct, s, slot);
  }
  // row-column: vertical pass and horizontal pass through p->tmp
  const long long tp = (long long)(p->tmp_pitch / es);
  LevelArgs v = a, hz = a;
  const Coefs cv = make_coefs(L, p->norm, a.W, a.H, PASS_VERT, inverse);
  const Coefs chz = make_coefs(L, p->norm, a.W, a.H, PASS_HORZ, inverse);
  LaunchKey kv{p->wavelet, p->dtype, DWT_ROWCOL, PASS_VERT, inverse ? 1 : 0, 0};
  LaunchKey kh{p->wavelet, p->dtype, DWT_ROWCOL, PASS_HORZ, inverse ? 1 : 0, 0};
  dwt_status st;
  if (!inverse) {
    v.src[0] = samples;
    v.src_pitch[0] = spitch;
    v.dst[0] = p->tmp;
    v.dst_pitch[0] = tp;
    hz.src[0] = p->tmp;
    hz.src_pitch[0] = tp;
    for (int i = 0; i < 4; ++i) {
      hz.dst[i] = const_cast<void*>(band[i]);
      hz.dst_pitch[i] = bpitch[i];
    }
    std::snprintf(slot, sizeof slot, "fwd-v/L%d", k);
    st = launch(p, kv, v, cv, ct, s, slot);
    if (st != DWT_OK) return st;
    std::snprintf(slot, sizeof slot, "fwd-h/L%d", k);
    return launch(p, kh, hz, chz, ct, s, slot);
  }
  for (int i = 0; i < 4; ++i) {
    hz.src[i] = band[i];
    hz.src_pitch[i] = bpitch[i];
  }
  hz.dst[0] = p->tmp;
  hz.dst_pitch[0] = tp;
  v.src[0] = p->tmp;
  v.src_pitch[0] = tp;
  v.dst[0] = const_cast<void*>(samples);
  v.dst_pitch[0] = spitch;
  std::snprintf(slot, sizeof slot, "inv-h/L%d", k);
  st = launch(p, kh, hz, chz, ct, s, slot);
  if (st != DWT_OK) return st;
  std::snprintf(slot, sizeof slot, "inv-v/L%d", k);
  return launch(p, kv, v, cv, ct, s, slot);
}

// The levels [k0, k1) a call runs in the fused tail (k0 == k1: none): from
// the first level whose input has at most the plan's threshold of samples,
// while both sides stay >= 2, at most kMaxTailLevels, for every scheme with
// a tile program (not row-column or Convolution).
void tail_range(const dwt_plan_s* p, int scheme, bool inverse, int* k0, int* k1) {
  *k0 = *k1 = p->levels;
  const long long fp = p->fuse_px < 0 ? kDefaultFusePx : p->fuse_px;
  if (fp == 0 || scheme == DWT_ROWCOL || scheme == DWT_CONVOLUTION) return;
  int a = 0;
  while (a < p->levels && (long long)p->W[a] * p->H[a] > fp) ++a;
  int b = a;
  while (b < p->levels && b - a < kMaxTailLevels && p->W[b] >= 2 && p->H[b] >= 2) ++b;
  if (b == a) return;
  TailInfo ti{};
  const LaunchKey key{p->wavelet, p->dtype, scheme, PASS_FUSED, inverse ? 1 : 0,
                      p->norm == DWT_NORM_JPEG2000 ? 1 : 0};
  if (!find_tail(key, &ti)) return;
  *k0 = a;
  *k1 = b;
}

// Levels [k0, k1) of a call in one launch of the fused-tail kernel, in
// processing order (finest first forward, coarsest first inverse).
dwt_status run_tail(dwt_plan_s* p, bool inverse, int k0, int k1, int scheme, const Lifting& L, const void* src,
                    size_t src_pitch, void* dst, size_t dst_pitch, void* const* ll, const size_t* llp,
                    cudaStream_t s) {
  const LaunchKey key{p->wavelet, p->dtype, scheme, PASS_FUSED, inverse ? 1 : 0,
                      p->norm == DWT_NORM_JPEG2000 ? 1 : 0};
  TailInfo ti{};
  if (!find_tail(key, &ti)) return DWT_EUNSUPPORTED;
  TailParams tp;
  std::memset(&tp, 0, sizeof tp);
  long long max_tiles = 0;
  double bytes = 0.0;
  for (int i = 0; i < k1 - k0; ++i) {
    const int k = inverse ? k1 - 1 - i : k0 + i;
    TileLevel& tl = tp.lv[i];
    level_dims(p, k, tl.a);
    const LevelIO io = level_io(p, inverse, k, tl.a, src, src_pitch, dst, dst_pitch, ll, llp);
    fused_io(io, inverse, tl.a);
    tl.a.status = p->d_status;
    if (i == 0) {
      set_waits(tl.a, p->d_status + 1);  // one injected hold per launch at most
    } else {
      tl.a.probes = tp.lv[0].a.probes;
      tl.a.spins = tp.lv[0].a.spins;
      tl.a.hold = nullptr;
    }
    tl.cf = make_coefs(L, p->norm, tl.a.W, tl.a.H, PASS_FUSED, inverse);
    tl.ntx = (tl.a.cw + ti.inner_cols - 1) / ti.inner_cols;
    tl.nty = (tl.a.ch + ti.inner_rows - 1) / ti.inner_rows;
    max_tiles = std::max(max_tiles, (long long)tl.ntx * tl.nty);
    bytes += 2.0 * tl.a.W * (double)tl.a.H * p->es;
  }
  tp.nlevels = k1 - k0;
  tp.barrier = reinterpret_cast<unsigned*>(p->d_status + 2);
  const Occ oc = occupancy(ti.fn, ti.smem_bytes, p->device, kTileThreads);
  const int blocks = (int)std::max<long long>(1, std::min<long long>(max_tiles, (long long)oc.sms * oc.per_sm));

  ProfRec rec{-1, nullptr, nullptr, 0.0};
  if (p->profiling) {
    char slot[32];
    std::snprintf(slot, sizeof slot, "%s/L%d-%d", inverse ? "inv" : "fwd", k0, k1 - 1);
    rec.slot = slot_of(p, slot);
    rec.a = take_event(p);
    rec.b = take_event(p);
    rec.bytes = bytes;
    cudaEventRecord(rec.a, s);
  }
  const cudaError_t e = call_tail(key, TailCall{&tp, blocks, s});
  if (p->profiling) {
    cudaEventRecord(rec.b, s);
    p->pending.push_back(rec);
  }
  return from_cuda(e);
}

// The transform proper: levels in order (forward) or reverse (inverse), the
// small ones in one fused-tail launch.
dwt_status run(dwt_plan_s* p, bool inverse, const void* src, size_t src_pitch, void* dst,
               size_t dst_pitch, cudaStream_t s) {
  const size_t es = p->es;
  const dwt_status chk = check_buffers(p, src, src_pitch, dst, dst_pitch);
  if (chk != DWT_OK) return chk;
  const dwt_status dev = ensure_device(p);
  if (dev != DWT_OK) return dev;
  p->last_stream = s;
  if (p->levels == 0)
    return from_cuda(cudaMemcpy2DAsync(dst, dst_pitch, src, src_pitch, (size_t)p->w * es, p->h,
                                       cudaMemcpyDeviceToDevice, s));
  const int scheme = resolve_scheme(p);
  if (!scheme_supported(p->wavelet, p->dtype, scheme)) return DWT_EUNSUPPORTED;
  if (scheme == DWT_ROWCOL) {
    dwt_status st = ensure_tmp(p);
    if (st != DWT_OK) return st;
  }
  const Lifting L = lifting_of(p->wavelet);
  const int Lv = p->levels;
  std::vector<void*> ll(p->ll);
  std::vector<size_t> llp(p->ll_pitch);
  ll.resize(Lv, nullptr);
  llp.resize(Lv, 0);
  int k0, k1;
  tail_range(p, scheme, inverse, &k0, &k1);

  if (!inverse) {
    for (int k = 0; k < Lv; ++k) {
      dwt_status st;
      if (k == k0) {
        st = run_tail(p, false, k0, k1, scheme, L, src, src_pitch, dst, dst_pitch, ll.data(), llp.data(), s);
        k = k1 - 1;
      } else {
        st = run_level(p, false, k, scheme, L, src, src_pitch, dst, dst_pitch, ll.data(), llp.data(), s);
      }
      if (st != DWT_OK) return st;
    }
  } else {
    for (int k = Lv - 1; k >= 0; --k) {
      dwt_status st;
      if (k0 < k1 && k == k1 - 1) {
        st = run_tail(p, true, k0, k1, scheme, L, src, src_pitch, dst, dst_pitch, ll.data(), llp.data(), s);
        k = k0;
      } else {
        st = run_level(p, true, k, scheme, L, src, src_pitch, dst, dst_pitch, ll.data(), llp.data(), s);
      }
      if (st != DWT_OK) return st;
    }
  }
  return DWT_OK;
}

// ---------------------------------------------------------------------------
// Batches: every level of every request in one persistent launch (batch.cu)
// ---------------------------------------------------------------------------
int batch_kind(int wavelet, int dtype, bool inverse) {
  const int inv = inverse ? 1 : 0;
  if (dtype == DWT_F32 && wavelet == DWT_CDF97) return BK_97_F32_FWD + inv;
  if (dtype == DWT_F32 && wavelet == DWT_CDF53) return BK_53_F32_FWD + inv;
  if (dtype == DWT_I32 && wavelet == DWT_CDF53) return BK_53_I32_FWD + inv;
  if (dtype == DWT_F16S && wavelet == DWT_CDF97) return BK_97_F16_FWD + inv;
  if (dtype == DWT_F16S && wavelet == DWT_CDF53) return BK_53_F16_FWD + inv;
  if (dtype == DWT_F32 && wavelet == DWT_DD137) return BK_DD_F32_FWD + inv;
  return -1;
}

// Page-locked upload buffers for the work lists: a ring of slots per
// device.  A slot is refilled only after its previous upload completed;
// with several slots a new batch rarely waits, even when the stream of the
// batch before it is still busy.
constexpr int kStagingSlots = 8;
struct StagingSlot {
  void* host = nullptr;
  size_t cap = 0;
  cudaEvent_t uploaded = nullptr;
};
struct BatchStaging {
  std::mutex mu;
  StagingSlot slot[kStagingSlots];
  int next = 0;
};
BatchStaging g_staging[64];

// Stream-ordered pool of the batches' work areas, one per device.  It keeps
// the memory it has handed out (no release threshold), so a steady stream of
// batches allocates from the driver only while its peak grows.
cudaError_t batch_pool(int device, cudaMemPool_t* out) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[device]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    pools[device] = pool;
  }
  *out = pools[device];
  return cudaSuccess;
}

dwt_status batch_submit(const dwt_request* reqs, int n, cudaStream_t s, int* d_status) {
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) return DWT_ECUDA;
  if (device < 0 || device >= 64) return DWT_EUNSUPPORTED;
  std::vector<int> kinds(n);
  int maxl = 0;
  bool with_dd = false;
  for (int i = 0; i < n; ++i) {
    const dwt_plan_s* p = reqs[i].plan;
    if (p->device != device) return DWT_EINVAL;
    const dwt_status chk = check_buffers(p, reqs[i].in, reqs[i].in_pitch, reqs[i].out, reqs[i].out_pitch);
    if (chk != DWT_OK) return chk;
    kinds[i] = batch_kind(p->wavelet, p->dtype, reqs[i].inverse != 0);
    if (kinds[i] < 0) return DWT_EUNSUPPORTED;
    // the batch's int32 kind is the JPEG 2000 transform
    if (p->dtype == DWT_I32 && p->scheme == DWT_IWAHASHI) return DWT_EUNSUPPORTED;
    with_dd = with_dd || p->wavelet == DWT_DD137;
    maxl = std::max(maxl, p->levels);
  }
  // images may not share memory with each other either: no output range
  // may meet another output or any input (sorted sweeps, O(n log n))
  {
    typedef std::pair<uintptr_t, uintptr_t> Range;  // [begin, end)
    std::vector<Range> outs(n), ins(n);
    for (int i = 0; i < n; ++i) {
      const dwt_plan_s* p = reqs[i].plan;
      const uintptr_t o = reinterpret_cast<uintptr_t>(reqs[i].out);
      const uintptr_t x = reinterpret_cast<uintptr_t>(reqs[i].in);
      outs[i] = Range(o, o + plane_extent(p->w, p->h, reqs[i].out_pitch, p->es));
      ins[i] = Range(x, x + plane_extent(p->w, p->h, reqs[i].in_pitch, p->es));
    }
    std::sort(outs.begin(), outs.end());
    for (int i = 1; i < n; ++i)
      if (outs[i].first < outs[i - 1].second) return DWT_EINVAL;
    // an input meets some output iff the output starting last before the
    // input's end reaches past the input's start (outputs are disjoint)
    for (const Range& r : ins) {
      auto it = std::lower_bound(outs.begin(), outs.end(), Range(r.second, 0));
      if (it != outs.begin() && std::prev(it)->second > r.first) return DWT_EINVAL;
    }
  }

  KernelInfo kinfo[BK_COUNT];
  for (int k = 0; k < BK_COUNT; ++k)
    if (!batch_kind_info(k, &kinfo[k])) return DWT_EUNSUPPORTED;
  const Occ oc = occupancy(kinfo[0].fn, kinfo[0].smem_bytes, device, 32);  // one-warp blocks
  const int resident = oc.sms * oc.per_sm;

  // ring depth: the deepest any plan whose tile the caller set asks for,
  // else the full ring (the batch kernel's shared memory is sized for
  // kMaxStages whatever the depth, so the deepest ring costs no occupancy)
  int nstages = 0;
  for (int i = 0; i < n; ++i)
    if (reqs[i].plan->tile_set) nstages = std::max(nstages, reqs[i].plan->nstages);
  if (nstages == 0) nstages = kMaxStages;

  // pass 1, geometry: every (request, level) in step order per request,
  // with its strip rows numbered consecutively
  std::vector<int> active(maxl + 1, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < reqs[i].plan->levels; ++j) ++active[j];
  std::vector<BatchLevel> levels;
  std::vector<int> level_of(0), step_of(0);
  int nrows = 0;
  for (int i = 0; i < n; ++i) {
    const dwt_plan_s* p = reqs[i].plan;
    const bool inverse = reqs[i].inverse != 0;
    const KernelInfo& ki = kinfo[kinds[i]];
    for (int step = 0; step < p->levels; ++step) {
      const int k = inverse ? p->levels - 1 - step : step;
      const int cap = std::max(1, resident / std::max(active[step], 1));
      BatchLevel b;
      std::memset(&b, 0, sizeof b);
      LevelArgs& a = b.a;
      level_dims(p, k, a);
      a.ncs = (a.cw + ki.uq - 1) / ki.uq;
      a.T = strip_height(p->tile_set && p->strip_rows > 0 ? p->strip_rows : kBatchStripRows, a.ch, a.ncs, cap,
                         ki.up + ki.down, chunk_rows(ki));
      a.nrs = (a.ch + a.T - 1) / a.T;
      a.nstages = nstages;
      b.cf = make_coefs(lifting_of(p->wavelet), p->norm, a.W, a.H, PASS_FUSED, inverse);
      const bool static_ok = p->norm == DWT_NORM_JPEG2000 && a.W >= 2 && a.H >= 2;
      b.kind = static_ok ? kinds[i] : batch_runtime_kind(kinds[i]);
      b.request = i;
      b.row_base = nrows;
      b.dep_row_base = step > 0 ? levels.back().row_base : -1;
      b.dep_ncs = step > 0 ? levels.back().a.ncs : 0;
      nrows += a.nrs;
      levels.push_back(b);
      level_of.push_back(k);
      step_of.push_back(step);
    }
  }
  const int nl = (int)levels.size();
  // injected failure: the second level of the first request waits for one
  // more strip per row than its rows have, a count nothing reaches
  if (injected(DWT_INJECT_BATCH_DEP))
    for (BatchLevel& bl : levels)
      if (bl.request == 0 && bl.dep_row_base >= 0) {
        ++bl.dep_ncs;
        break;
      }

  std::vector<int2> row_deps(nrows, make_int2(0, -1));
  for (int l = 0; l < nl; ++l) {
    const BatchLevel& bl = levels[l];
    if (bl.dep_row_base < 0) continue;
    row_dependencies(bl.a, levels[l - 1].a, kinfo[bl.kind], reqs[bl.request].inverse != 0,
                     row_deps.data() + bl.row_base);
  }

  // queue order: a wavefront.  The first level of each request enters in
  // request order; a strip row of a later level is placed three resident
  // waves of items after the last row it depends on: items popped that long
  // ago have almost always finished (a warp pops one item per strip time),
  // so the row rarely waits, and the levels of different requests overlap.
  // Every row comes strictly after its dependencies (keys grow by the lag),
  // which is what keeps the persistent kernel's waits finite.
  const long long lag = 3LL * resident;
  struct OrderedRow {
    long long key;
    int step, level, rs;
  };
  std::vector<OrderedRow> rows(nrows);
  {
    long long root = 0;
    for (int l = 0; l < nl; ++l) {
      const BatchLevel& bl = levels[l];
      for (int rs = 0; rs < bl.a.nrs; ++rs) {
        long long k;
        if (bl.dep_row_base < 0) {
          root += bl.a.ncs;
          k = root;
        } else {
          const int2 d = row_deps[bl.row_base + rs];
          long long m = 0;
          for (int r = d.x; r <= d.y; ++r) m = std::max(m, rows[bl.dep_row_base + r].key);
          k = m + lag;
        }
        rows[bl.row_base + rs] = OrderedRow{k, step_of[l], l, rs};
      }
    }
  }
  std::sort(rows.begin(), rows.end(), [](const OrderedRow& x, const OrderedRow& y) {
    if (x.key != y.key) return x.key < y.key;
    if (x.step != y.step) return x.step < y.step;
    if (x.level != y.level) return x.level < y.level;
    return x.rs < y.rs;
  });
  size_t nitems = 0;
  for (const BatchLevel& bl : levels) nitems += (size_t)bl.a.ncs * bl.a.nrs;
  if (nitems > (size_t)INT32_MAX) return DWT_EINVAL;

  // work area: levels | items | row deps (uploaded) | per-request LL
  // buffers | head, row_done[nrows], status[n]
  const size_t off_items = round_up(sizeof(BatchLevel) * nl, 256);
  const size_t off_deps = round_up(off_items + sizeof(BatchItem) * nitems, 256);
  const size_t upload = round_up(off_deps + sizeof(int2) * (size_t)nrows, 256);
  std::vector<std::vector<size_t>> ll_off(n), ll_pitch(n);
  size_t off = upload;
  for (int i = 0; i < n; ++i) {
    const dwt_plan_s* p = reqs[i].plan;
    for (int k = 0; k + 1 < p->levels; ++k) {
      const size_t pitch = round_up((size_t)p->W[k + 1] * p->es, 128);
      ll_off[i].push_back(off);
      ll_pitch[i].push_back(pitch);
      off = round_up(off + pitch * p->H[k + 1], 256);
    }
  }
  const size_t off_head = off;
  const size_t counters = sizeof(int) * (1 + (size_t)nrows + (size_t)n);

  BatchStaging& bs = g_staging[device];
  std::lock_guard<std::mutex> lk(bs.mu);
  StagingSlot& st = bs.slot[bs.next];
  bs.next = (bs.next + 1) % kStagingSlots;
  cudaError_t e = cudaSuccess;
  if (!st.uploaded) e = cudaEventCreateWithFlags(&st.uploaded, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventSynchronize(st.uploaded);
  if (e == cudaSuccess && st.cap < upload) {
    if (st.host) cudaFreeHost(st.host);
    st.host = nullptr;
    st.cap = 0;
    e = host_malloc(&st.host, upload * 2);
    if (e == cudaSuccess) st.cap = upload * 2;
  }
  if (e != cudaSuccess) return from_cuda(e);
  // requests without levels are copies
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const dwt_plan_s* p = reqs[i].plan;
    if (p->levels == 0)
      e = cudaMemcpy2DAsync(reqs[i].out, reqs[i].out_pitch, reqs[i].in, reqs[i].in_pitch,
                            (size_t)p->w * p->es, p->h, cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess && d_status && n) e = cudaMemsetAsync(d_status, 0, sizeof(int) * n, s);
  if (e != cudaSuccess || nitems == 0) return from_cuda(e);

  cudaMemPool_t pool = nullptr;
  e = batch_pool(device, &pool);
  if (e != cudaSuccess) return from_cuda(e);
  // tensor maps read from global memory must be 64-byte aligned
  unsigned char* block = nullptr;
  e = pool_malloc(reinterpret_cast<void**>(&block), off_head + counters + 128, pool, s);
  if (e != cudaSuccess) return from_cuda(e);
  unsigned char* d = block + ((128 - (reinterpret_cast<uintptr_t>(block) & 127)) & 127);
  int* head = reinterpret_cast<int*>(d + off_head);
  int* row_done = head + 1;
  // a strip that gives up on its ring raises its level's status word: the
  // caller's slot for the request, or a slot of this block
  int* status = d_status ? d_status : row_done + nrows;

  // pass 2, addresses: buffers, LL buffers, tensor maps
  for (int l = 0; l < nl; ++l) {
    BatchLevel& b = levels[l];
    const int i = b.request;
    const dwt_plan_s* p = reqs[i].plan;
    const bool inverse = reqs[i].inverse != 0;
    LevelArgs& a = b.a;
    std::vector<void*> ll(ll_off[i].size());
    for (size_t k = 0; k < ll.size(); ++k) ll[k] = d + ll_off[i][k];
    const LevelIO io = level_io(p, inverse, level_of[l], a, reqs[i].in, reqs[i].in_pitch, reqs[i].out,
                                reqs[i].out_pitch, ll.data(), ll_pitch[i].data());
    fused_io(io, inverse, a);
    a.status = status + i;
    a.probes = g_ring_probes.load();
    a.spins = g_dep_spins.load();
    a.hold = nullptr;
    a.src_tma = encode_level_maps(&b.maps, p->dtype, a, kinfo[b.kind], p->es);
  }
  unsigned char* h = static_cast<unsigned char*>(st.host);
  std::memcpy(h, levels.data(), sizeof(BatchLevel) * nl);
  BatchItem* items = reinterpret_cast<BatchItem*>(h + off_items);
  size_t it = 0;
  for (const OrderedRow& r : rows) {
    const int ncs = levels[r.level].a.ncs;
    for (int cs = 0; cs < ncs; ++cs) items[it++] = BatchItem{r.level, r.rs * ncs + cs};
  }
  std::memcpy(h + off_deps, row_deps.data(), sizeof(int2) * (size_t)nrows);
  e = cudaMemcpyAsync(d, h, upload, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(st.uploaded, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(head, 0, counters, s);
  if (e == cudaSuccess) {
    BatchParams bp;
    bp.levels = reinterpret_cast<const BatchLevel*>(d);
    bp.items = reinterpret_cast<const BatchItem*>(d + off_items);
    bp.row_deps = reinterpret_cast<const int2*>(d + off_deps);
    bp.nitems = (int)nitems;
    bp.head = head;
    bp.row_done = row_done;
    bp.req_status = status;
    e = launch_batch(bp, (int)std::min<size_t>((size_t)resident, nitems), with_dd, s);
  }
  const cudaError_t ef = cudaFreeAsync(block, s);
  if (e == cudaSuccess) e = ef;
  return from_cuda(e);
}

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess) ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// Forward transform on caller-provided scratch, for the entry point that
// allocates nothing (noalloc.cu).  It runs the plan path's forward level
// loop with the default scheme (Monolithic* for float, the separable JPEG
// 2000 order for int32) and the tile a fresh plan takes (the scheme's
// default strip height and ring depth, the same deeper ring for levels
// that fit one wave), keeps its state on the stack, and makes no device or
// host allocation.  d_status points at two device words: the status word
// and a flag that nothing sets (for the injected hold).
// ---------------------------------------------------------------------------
namespace dwt {

dwt_status forward_on_scratch(int w, int h, int wavelet, int levels, int dtype, const void* src,
                              size_t src_pitch, void* dst, size_t dst_pitch, void* scratch,
                              size_t scratch_bytes, int* d_status, cudaStream_t s) {
  if (w < 1 || h < 1 || w > kMaxSide || h > kMaxSide || levels < 0 || levels > 30) return DWT_EINVAL;
  if (wavelet < 0 || wavelet > 2 || dtype < 0 || dtype > 2) return DWT_EINVAL;
  int Wk[32], Hk[32];
  Wk[0] = w;
  Hk[0] = h;
  int maxl = 0;
  for (int a = w, b = h; a > 1 || b > 1; a = (a + 1) / 2, b = (b + 1) / 2) ++maxl;
  if (levels > maxl) return DWT_EINVAL;
  for (int k = 1; k <= levels + 1 && k < 32; ++k) {
    Wk[k] = (Wk[k - 1] + 1) / 2;
    Hk[k] = (Hk[k - 1] + 1) / 2;
  }
  const int scheme = dtype == DWT_I32 ? DWT_SWELDENS : DWT_MONOLITHIC_S;
  if (!scheme_supported(wavelet, dtype, scheme)) return DWT_EUNSUPPORTED;
  const size_t es = elem_size(dtype);
  if (src_pitch < (size_t)w * es || dst_pitch < (size_t)w * es || src_pitch % es || dst_pitch % es)
    return DWT_EINVAL;
  if (reinterpret_cast<uintptr_t>(src) % es || reinterpret_cast<uintptr_t>(dst) % es) return DWT_EINVAL;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) return DWT_ECUDA;
  const size_t nsrc = plane_extent(w, h, src_pitch, es), ndst = plane_extent(w, h, dst_pitch, es);
  if (!device_pointer_ok(src, nsrc, device) || !device_pointer_ok(dst, ndst, device)) return DWT_EINVAL;
  if (overlaps(src, nsrc, dst, ndst)) return DWT_EINVAL;
  // Two LL regions used in turn: LL_1, LL_3, ... in the first (ceil(h/2)
  // rows), LL_2, LL_4, ... in the second (ceil(h/4) rows), rows at a
  // 128-byte pitch of ceil(w/2) elements.  A level's kernel starts reading
  // only after the previous level's grid completed, so overwriting LL_k
  // with LL_{k+2} is safe.
  const size_t spitch = levels >= 2 ? round_up((size_t)Wk[1] * es, 128) : 0;
  const size_t need = levels >= 2 ? spitch * ((size_t)Hk[1] + Hk[2]) : 0;
  if (need > scratch_bytes) return DWT_EINVAL;
  if (levels == 0)
    return from_cuda(cudaMemcpy2DAsync(dst, dst_pitch, src, src_pitch, (size_t)w * es, h,
                                       cudaMemcpyDeviceToDevice, s));
  char* sbase = static_cast<char*>(scratch);
  void* sc[2] = {sbase, sbase + spitch * (size_t)Hk[1]};
  const Lifting L = lifting_of(wavelet);
  const Tile tile{device, kDefaultStages, 0};
  for (int k = 0; k < levels; ++k) {
    LevelArgs a{};
    a.W = Wk[k];
    a.H = Hk[k];
    a.cw = (a.W + 1) / 2;
    a.ch = (a.H + 1) / 2;
    a.fw = a.W / 2;
    a.fh = a.H / 2;
    char* ob = static_cast<char*>(dst);
    a.src[0] = k == 0 ? src : sc[(k - 1) & 1];
    a.src_pitch[0] = (long long)((k == 0 ? src_pitch : spitch) / es);
    a.dst[0] = k == levels - 1 ? dst : sc[k & 1];
    a.dst_pitch[0] = (long long)((k == levels - 1 ? dst_pitch : spitch) / es);
    a.dst[1] = ob + a.cw * es;
    a.dst[2] = ob + a.ch * dst_pitch;
    a.dst[3] = ob + a.ch * dst_pitch + a.cw * es;
    for (int i = 1; i < 4; ++i) a.dst_pitch[i] = (long long)(dst_pitch / es);
    const Coefs cf = make_coefs(L, DWT_NORM_JPEG2000, a.W, a.H, PASS_FUSED, false);
    ConvTaps ct;
    std::memset(&ct, 0, sizeof ct);
    const LaunchKey key{wavelet, dtype, scheme, PASS_FUSED, 0, a.W >= 2 && a.H >= 2 ? 1 : 0};
    KernelInfo ki{};
    const dwt_status g = level_geometry(tile, key, a, ki);
    if (g != DWT_OK) return g;
    a.status = d_status;
    set_waits(a, d_status + 1);
    TmaMaps maps;
    a.src_tma = encode_level_maps(&maps, dtype, a, ki, es);
    const LaunchCall call{&a, &maps, &cf, &ct, s};
    const cudaError_t e = call_kernel(key, kDefaultStages, call);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return DWT_OK;
}

}  // namespace dwt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* dwt_version(void) { return "0.1.0"; }

const char* dwt_status_string(dwt_status s) {
  switch (s) {
    case DWT_OK: return "ok";
    case DWT_EINVAL: return "invalid argument";
    case DWT_ENOMEM: return "out of memory";
    case DWT_EUNSUPPORTED: return "unsupported combination";
    case DWT_ECUDA: return "CUDA error";
    case DWT_ETIMEOUT: return "device-side wait timed out";
    case DWT_EBUSY: return "resource busy";
  }
  return "unknown status";
}

dwt_status dwt_plan_create(int w, int h, dwt_wavelet wavelet, int levels, dwt_dtype dtype,
                           dwt_plan* out) {
  if (!out) return DWT_EINVAL;
  *out = nullptr;
  if (w < 1 || h < 1 || w > kMaxSide || h > kMaxSide || levels < 0) return DWT_EINVAL;
  if ((int)wavelet < 0 || (int)wavelet > 2 || (int)dtype < 0 || (int)dtype > 2) return DWT_EINVAL;
  int maxl = 0;
  for (int a = w, b = h; a > 1 || b > 1; a = (a + 1) / 2, b = (b + 1) / 2) ++maxl;
  if (levels > maxl) return DWT_EINVAL;
  if (dtype == DWT_I32 && wavelet != DWT_CDF53) return DWT_EUNSUPPORTED;
  if (wavelet == DWT_DD137 && dtype != DWT_F32) return DWT_EUNSUPPORTED;
  dwt_plan_s* p = new (std::nothrow) dwt_plan_s();
  if (!p) return DWT_ENOMEM;
  p->w = w;
  p->h = h;
  p->levels = levels;
  p->wavelet = wavelet;
  p->dtype = dtype;
  p->es = elem_size(dtype);
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return DWT_ECUDA;
  }
  p->W.resize(levels + 2);
  p->H.resize(levels + 2);
  p->W[0] = w;
  p->H[0] = h;
  for (int k = 1; k <= levels + 1; ++k) {
    p->W[k] = (p->W[k - 1] + 1) / 2;
    p->H[k] = (p->H[k - 1] + 1) / 2;
  }
  *out = p;
  return DWT_OK;
}

dwt_status dwt_plan_set_scheme(dwt_plan p, dwt_scheme scheme) {
  if (!p) return DWT_EINVAL;
  if ((int)scheme < 0 || (int)scheme >= NUM_SCHEMES) return DWT_EINVAL;
  if (scheme != DWT_AUTO && !scheme_supported(p->wavelet, p->dtype, scheme)) return DWT_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(p->mu);
  p->scheme = scheme;
  if (scheme == DWT_ROWCOL && p->levels > 0) {
    DeviceGuard g(p->device);
    return ensure_tmp(p);
  }
  return DWT_OK;
}

dwt_status dwt_plan_set_tile(dwt_plan p, int strip_rows, int stages) {
  if (!p || strip_rows < 0 || strip_rows > 1 << 20 || stages < 0 || stages > kMaxStages)
    return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  p->strip_rows = strip_rows;
  p->nstages = stages ? stages : kDefaultStages;
  p->tile_set = strip_rows != 0 || stages != 0;
  return DWT_OK;
}

dwt_status dwt_plan_set_fusion(dwt_plan p, long long max_pixels) {
  if (!p || max_pixels < -1) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  p->fuse_px = max_pixels;
  return DWT_OK;
}

dwt_status dwt_plan_get_fusion(dwt_plan p, long long* max_pixels) {
  if (!p || !max_pixels) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  *max_pixels = p->fuse_px < 0 ? kDefaultFusePx : p->fuse_px;
  return DWT_OK;
}

dwt_status dwt_plan_get_tile(dwt_plan p, int* strip_rows, int* stages) {
  if (!p) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  const int scheme = resolve_scheme(p);
  if (strip_rows) *strip_rows = p->strip_rows > 0 ? p->strip_rows : default_strip_rows(scheme, p->wavelet);
  if (stages) *stages = p->nstages;
  return DWT_OK;
}

dwt_status dwt_plan_get_scheme(dwt_plan p, dwt_scheme* scheme) {
  if (!p || !scheme) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  *scheme = (dwt_scheme)resolve_scheme(p);
  return DWT_OK;
}

dwt_status dwt_plan_set_normalization(dwt_plan p, dwt_norm norm) {
  if (!p || ((int)norm != DWT_NORM_JPEG2000 && (int)norm != DWT_NORM_ZETA)) return DWT_EINVAL;
  if (p->dtype == DWT_I32 && norm != DWT_NORM_JPEG2000) return DWT_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(p->mu);
  p->norm = norm;
  return DWT_OK;
}

dwt_status dwt2_forward(dwt_plan p, const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch,
                        dwt_stream stream) {
  if (!p) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  return run(p, false, d_in, in_pitch, d_out, out_pitch, reinterpret_cast<cudaStream_t>(stream));
}

dwt_status dwt2_inverse(dwt_plan p, const void* d_coef, size_t coef_pitch, void* d_out,
                        size_t out_pitch, dwt_stream stream) {
  if (!p) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  return run(p, true, d_coef, coef_pitch, d_out, out_pitch, reinterpret_cast<cudaStream_t>(stream));
}

static dwt_status host_call(dwt_plan p, bool inverse, const void* h_in, size_t in_pitch, void* h_out,
                            size_t out_pitch, dwt_stream stream) {
  if (!p || !h_in || !h_out) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  const size_t row = (size_t)p->w * p->es;
  if (in_pitch < row || out_pitch < row) return DWT_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!p->stage_in || !p->stage_out) {
    // both staging planes or neither: a failure frees what was made
    const size_t pitch = round_up(row, 128);
    void *in = nullptr, *out = nullptr;
    cudaError_t e = dev_malloc(&in, pitch * p->h);
    if (e == cudaSuccess) e = dev_malloc(&out, pitch * p->h);
    if (e != cudaSuccess) {
      if (in) cudaFree(in);
      return from_cuda(e);
    }
    p->stage_pitch = pitch;
    p->stage_in = in;
    p->stage_out = out;
  }
  cudaError_t e = cudaMemcpy2DAsync(p->stage_in, p->stage_pitch, h_in, in_pitch, row, p->h,
                                    cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return from_cuda(e);
  dwt_status st = run(p, inverse, p->stage_in, p->stage_pitch, p->stage_out, p->stage_pitch, s);
  if (st != DWT_OK) return st;
  return from_cuda(cudaMemcpy2DAsync(h_out, out_pitch, p->stage_out, p->stage_pitch, row, p->h,
                                     cudaMemcpyDeviceToHost, s));
}

dwt_status dwt2_forward_host(dwt_plan p, const void* h_in, size_t in_pitch, void* h_out,
                             size_t out_pitch, dwt_stream stream) {
  return host_call(p, false, h_in, in_pitch, h_out, out_pitch, stream);
}

dwt_status dwt2_inverse_host(dwt_plan p, const void* h_coef, size_t coef_pitch, void* h_out,
                             size_t out_pitch, dwt_stream stream) {
  return host_call(p, true, h_coef, coef_pitch, h_out, out_pitch, stream);
}

dwt_status dwt_batch_submit(const dwt_request* reqs, int n, dwt_stream stream, int* d_status) {
  if (n < 0 || (n > 0 && !reqs)) return DWT_EINVAL;
  std::vector<dwt_plan_s*> plans(n);
  for (int i = 0; i < n; ++i) {
    if (!reqs[i].plan) return DWT_EINVAL;
    plans[i] = reqs[i].plan;
  }
  if (n == 0) return DWT_OK;
  // every plan of the call stays locked until the launch is queued; taking
  // the locks in address order keeps concurrent batches from deadlocking
  std::sort(plans.begin(), plans.end());
  plans.erase(std::unique(plans.begin(), plans.end()), plans.end());
  std::vector<std::unique_lock<std::mutex>> locks;
  locks.reserve(plans.size());
  for (dwt_plan_s* p : plans) locks.emplace_back(p->mu);
  return batch_submit(reqs, n, reinterpret_cast<cudaStream_t>(stream), d_status);
}

dwt_status dwt_set_wait_limits(unsigned int ring_probes, unsigned int dep_spins) {
  g_ring_probes.store(ring_probes ? ring_probes : kDefaultRingProbes);
  g_dep_spins.store(dep_spins ? dep_spins : kDefaultDepSpins);
  return DWT_OK;
}

dwt_status dwt_debug_inject(dwt_injection what, int skip, int count) {
  if ((int)what < DWT_INJECT_NONE || (int)what > DWT_INJECT_BATCH_DEP || skip < 0 || count < 0)
    return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(g_inject_mu);
  if (what == DWT_INJECT_NONE) {
    for (Injection& j : g_inject) j = Injection{};
  } else {
    g_inject[what] = Injection{skip, count};
  }
  return DWT_OK;
}

dwt_status dwt_plan_device_status(dwt_plan p) {
  if (!p) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  int v = 0;
  cudaError_t e = cudaStreamSynchronize(p->last_stream);
  if (e == cudaSuccess && !p->d_status) return DWT_OK;
  if (e == cudaSuccess) e = cudaMemcpy(&v, p->d_status, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return from_cuda(e);
  return v ? DWT_ETIMEOUT : DWT_OK;
}

dwt_status dwt_plan_set_profiling(dwt_plan p, int enable) {
  if (!p) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  p->profiling = enable != 0;
  return DWT_OK;
}

dwt_status dwt_plan_read_profile(dwt_plan p, dwt_kernel_stat* stats, int capacity, int* count) {
  if (!p || (capacity > 0 && !stats)) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  for (const ProfRec& r : p->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      p->slots[r.slot].launches += 1;
      p->slots[r.slot].ms += ms;
      p->slots[r.slot].bytes += r.bytes;
    }
    p->pool.push_back(r.a);
    p->pool.push_back(r.b);
  }
  p->pending.clear();
  const int n = (int)p->slots.size();
  for (int i = 0; i < n && i < capacity; ++i) {
    std::memset(&stats[i], 0, sizeof stats[i]);
    std::snprintf(stats[i].name, sizeof stats[i].name, "%s", p->slots[i].name.c_str());
    stats[i].launches = p->slots[i].launches;
    stats[i].total_ms = p->slots[i].ms;
    stats[i].algorithmic_bytes = p->slots[i].bytes;
  }
  if (count) *count = n;
  p->slots.clear();
  return DWT_OK;
}

dwt_status dwt_plan_autotune(dwt_plan p, dwt_stream stream) {
  if (!p) return DWT_EINVAL;
  std::lock_guard<std::mutex> lk(p->mu);
  if (p->levels == 0) return DWT_OK;
  DeviceGuard g(p->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t pitch = round_up((size_t)p->w * p->es, 128);
  void *in = nullptr, *out = nullptr;
  cudaError_t e = dev_malloc(&in, pitch * p->h);
  if (e == cudaSuccess) e = dev_malloc(&out, pitch * p->h);
  if (e == cudaSuccess) e = cudaMemsetAsync(in, 0x3c, pitch * p->h, s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  apply_cache(p);
  const int saved_scheme = p->scheme, saved_rows = p->strip_rows, saved_stages = p->nstages;
  const bool saved_prof = p->profiling;
  p->profiling = false;
  // best of three timed forward transforms (after two warm-up runs)
  auto time_it = [&](float* best) {
    float t = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
      cudaEventRecord(a, s);
      if (run(p, false, in, pitch, out, pitch, s) != DWT_OK) return false;
      cudaEventRecord(b, s);
      if (cudaEventSynchronize(b) != cudaSuccess) return false;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep >= 2) t = std::min(t, ms);
    }
    *best = t;
    return true;
  };
  // 1. the scheme, each at its default tile
  Tuned best;
  float best_ms = 0.f;
  p->strip_rows = 0;
  p->nstages = kDefaultStages;
  for (int sc = DWT_ROWCOL; e == cudaSuccess && sc < NUM_SCHEMES; ++sc) {
    // an int32 plan set to the integer Iwahashi lifting keeps that
    // transform (only its tile is tuned); others choose among the rest
    const bool iw_int = p->dtype == DWT_I32 && saved_scheme == DWT_IWAHASHI;
    if (iw_int ? sc != DWT_IWAHASHI : !tunable(p->wavelet, p->dtype, sc)) continue;
    p->scheme = sc;
    if (sc == DWT_ROWCOL && ensure_tmp(p) != DWT_OK) continue;
    float t;
    if (time_it(&t) && (best.scheme < 0 || t < best_ms)) {
      best.scheme = sc;
      best_ms = t;
    }
  }
  // 2. the strip height of that scheme, then the ring depth
  best.rows = best.scheme >= 0 ? default_strip_rows(best.scheme, p->wavelet) : kDefaultStripRows;
  best.stages = kDefaultStages;
  if (best.scheme >= 0) {
    p->scheme = best.scheme;
    for (int rows : {6, 8, 10, 12, 16, 24, 32, 48}) {
      if (rows == best.rows) continue;
      p->strip_rows = rows;
      float t;
      if (time_it(&t) && t < best_ms) {
        best.rows = rows;
        best_ms = t;
      }
    }
    p->strip_rows = best.rows;
    for (int st = 1; st <= kMaxStages; ++st) {
      if (st == kDefaultStages) continue;
      p->nstages = st;
      float t;
      if (time_it(&t) && t < best_ms) {
        best.stages = st;
        best_ms = t;
      }
    }
  }
  p->scheme = saved_scheme;
  p->profiling = saved_prof;
  if (p->tile_set) {
    p->strip_rows = saved_rows;
    p->nstages = saved_stages;
  } else {
    p->strip_rows = best.rows;
    p->nstages = best.stages;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(in);
  cudaFree(out);
  if (e != cudaSuccess) return from_cuda(e);
  if (best.scheme < 0) return DWT_EUNSUPPORTED;
  p->auto_scheme = best.scheme;
  cache_store(cache_key(p), best);
  return DWT_OK;
}

dwt_status dwt_plan_destroy(dwt_plan p) {
  if (!p) return DWT_EINVAL;
  {
    DeviceGuard g(p->device);
    // plans used only in batches own no device memory and nothing on the
    // device refers to them: no synchronisation
    const bool owns = !p->ll.empty() || p->tmp || p->stage_in || p->stage_out || p->d_status;
    if (owns && (p->last_stream || !p->pending.empty())) cudaDeviceSynchronize();
    for (void* q : p->ll) cudaFree(q);
    for (void* q : {p->tmp, p->stage_in, p->stage_out, static_cast<void*>(p->d_status)})
      if (q) cudaFree(q);
    for (const ProfRec& r : p->pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (cudaEvent_t ev : p->pool) cudaEventDestroy(ev);
  }
  delete p;
  return DWT_OK;
}

}  // extern "C"
