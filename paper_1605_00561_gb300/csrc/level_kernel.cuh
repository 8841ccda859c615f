// One transform level (or one row-column pass) as a streaming kernel.
//
// Work decomposition.  Each warp owns a strip: 64 quadruple columns wide
// (two per lane) and T quadruple rows tall.  The outer HQ quad columns on
// each side and UP / DOWN quad rows are the lifting halo (the overlapping
// tiles of Sec. 6): they are loaded and lifted but not stored, so that every
// stored coefficient only depends on samples the strip holds.  The warp
// walks down its strip one quad row at a time; every step of the scheme is
// a stage whose window keeps the rows of its input state it still needs
// (vertical neighbours), while horizontal neighbours are exchanged with
// warp shuffles.  What the paper synchronises with a work-group barrier
// between two steps is, here, the hand-over of a row from one stage's
// output to the next stage's window (vertical) and a shuffle (horizontal);
// no CTA-wide barrier is needed.
//
// Loads.  Rows arrive in chunks of kChunkRows quad rows through a per-warp
// ring of shared-memory stages, filled ahead of use: a chunk lying inside
// the image is one 2-D TMA box (cp.async.bulk.tensor, one box per source
// plane) when the source is 16-byte aligned; otherwise each lane issues
// cp.async copies, with whole-sample symmetric mirroring applied to the
// addresses at the image border.  Images with a length-1 axis use a
// synchronous fill that writes zeros for the samples that do not exist.
// Every stage has one mbarrier with 32 expected arrivals per fill; waits on
// it are bounded and report to the launch's status word.
#pragma once

#include <cuda_fp16.h>

#include "programs.cuh"
#include "ptx.cuh"

namespace dwt {
namespace dev {

constexpr uint32_t kWaitProbes = 1u << 24;

template <typename ST>
struct StoreT;
template <>
struct StoreT<float> {
  __device__ __forceinline__ static float to_v(float x) { return x; }
  __device__ __forceinline__ static float from_v(float x) { return x; }
};
template <>
struct StoreT<__half> {
  __device__ __forceinline__ static float to_v(__half x) { return __half2float(x); }
  __device__ __forceinline__ static __half from_v(float x) { return __float2half_rn(x); }
};
template <>
struct StoreT<int> {
  __device__ __forceinline__ static int to_v(int x) { return x; }
  __device__ __forceinline__ static int from_v(int x) { return x; }
};

template <typename ST_, typename VT_, class PROG_, int LOAD_, int STORE_>
struct Cfg {
  using ST = ST_;
  using VT = VT_;
  using PROG = PROG_;
  using Tot = Totals<PROG>;
  static constexpr int LOAD = LOAD_, STORE = STORE_;
  static constexpr int HQ = ((cmax(Tot::LEFT, Tot::RIGHT) + 1) / 2) * 2;
  static constexpr int UQ = 64 - 2 * HQ;
  static constexpr int ES = sizeof(ST);
  static constexpr int A = 16 / ES;  // elements per 16 bytes
  static constexpr int CH = kChunkRows;
  static constexpr int ROWE = (LOAD == SAMPLES ? 128 : 64) + A;
  // bytes of one plane's box; planes start on 128-byte boundaries
  static constexpr int PLANE_BYTES =
      LOAD == SAMPLES ? 2 * CH * ROWE * ES : ((CH * ROWE * ES + 127) / 128) * 128;
  static constexpr int BOX_BYTES = LOAD == SAMPLES ? 2 * CH * ROWE * ES : CH * ROWE * ES;
  static constexpr int NPLANES = LOAD == SAMPLES ? 1 : 4;
  static constexpr int STAGE_BYTES = ((NPLANES * PLANE_BYTES + 127) / 128) * 128;
  static_assert(HQ <= 8, "halo too wide for a 64-quad strip");
};

__device__ __forceinline__ int mirror(int i, int n) {
  // whole-sample symmetric extension (n >= 2): one reflection covers every
  // index within n - 1 of the line; shorter lines fold with period 2(n - 1)
  if (i < 0) i = -i;
  if (i >= n) i = 2 * (n - 1) - i;
  if ((unsigned)i < (unsigned)n) return i;
  const int period = 2 * (n - 1);
  i %= period;
  if (i < 0) i += period;
  return i >= n ? period - i : i;
}

__device__ __forceinline__ int align_down(int x, int a) {
  return x >= 0 ? (x / a) * a : -(((-x) + a - 1) / a) * a;
}

template <class C>
struct Strip {
  using ST = typename C::ST;
  using VT = typename C::VT;
  const LevelArgs& a;
  const TmaMaps& maps;
  int lane, m0, mfirst, yfirst;
  unsigned char* sm;
  uint64_t* bars;

  __device__ __forceinline__ ST* stage(int s) const {
    return reinterpret_cast<ST*>(sm + (size_t)s * C::STAGE_BYTES);
  }
  __device__ __forceinline__ const ST* src_plane(int p) const {
    return static_cast<const ST*>(a.src[p]);
  }

  // ---- fills ---------------------------------------------------------------
  __device__ void fill(int c, int s) const {
    const int y0 = yfirst + c * C::CH;
    uint64_t* bar = &bars[s];
    ST* dst = stage(s);
    const bool tiny = a.W < 2 || a.H < 2;
    if constexpr (C::LOAD == SAMPLES) {
      const int sy0 = 2 * y0, xs = 2 * mfirst;
      const int xal = align_down(xs, C::A), off = xs - xal;
      const bool inside = !tiny && sy0 >= 0 && sy0 + 2 * C::CH <= a.H && xs >= 0 && xs + 128 <= a.W;
      if (inside && a.src_tma) {
        if (lane == 0) {
          ptx::fence_proxy_async_smem();
          ptx::mbar_arrive_expect_tx(bar, C::BOX_BYTES);
          ptx::tma_load_2d(dst, &maps.m[0], xal, sy0, bar);
        } else {
          ptx::mbar_arrive(bar);
        }
        return;
      }
      const ST* src = src_plane(0);
      const long long pitch = a.src_pitch[0];
      if (!tiny && C::ES == 4) {
        for (int j = 0; j < 2 * C::CH; ++j) {
          const ST* rowp = src + (long long)mirror(sy0 + j, a.H) * pitch;
          ST* d = dst + j * C::ROWE + off + 4 * lane;
          const int gx = xs + 4 * lane;
          if (gx >= 0 && gx + 4 <= a.W && ((reinterpret_cast<uintptr_t>(rowp + gx) & 15) == 0)) {
            ptx::cp_async_16(d, rowp + gx);
          } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) ptx::cp_async_4(d + t, rowp + mirror(gx + t, a.W));
          }
        }
        ptx::cp_async_arrive(bar);
        return;
      }
      // synchronous fill: fp16 off the TMA path, or an axis of length 1
      for (int j = 0; j < 2 * C::CH; ++j) {
        const int gy = sy0 + j;
        const bool rabs = (a.H == 1 && gy != 0);
        const ST* rowp = src + (long long)(a.H == 1 ? 0 : mirror(gy, a.H)) * pitch;
        ST* d = dst + j * C::ROWE + off + 4 * lane;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int gx = xs + 4 * lane + t;
          const bool cabs = (a.W == 1 && gx != 0);
          d[t] = (rabs || cabs) ? StoreT<ST>::from_v(VT(0))
                                : rowp[a.W == 1 ? 0 : mirror(gx, a.W)];
        }
      }
      ptx::mbar_arrive(bar);
    } else {
      // four subband planes; the lane covers quads mfirst + 2*lane + {0, 1}
      const int xal = align_down(mfirst, C::A), off = mfirst - xal;
      const bool inside = !tiny && y0 >= 0 && y0 + C::CH <= a.fh && mfirst >= 0 && mfirst + 64 <= a.fw;
      if (inside && a.src_tma) {
        if (lane == 0) {
          ptx::fence_proxy_async_smem();
          ptx::mbar_arrive_expect_tx(bar, 4 * C::BOX_BYTES);
#pragma unroll
          for (int p = 0; p < 4; ++p)
            ptx::tma_load_2d(reinterpret_cast<unsigned char*>(dst) + p * C::PLANE_BYTES, &maps.m[p],
                             xal, y0, bar);
        } else {
          ptx::mbar_arrive(bar);
        }
        return;
      }
      const bool async = !tiny && C::ES == 4;
      const int m = mfirst + 2 * lane;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int py = p >> 1, px = p & 1;
        const int pw = px ? a.fw : a.cw, ph = py ? a.fh : a.ch;
        ST* pd = reinterpret_cast<ST*>(reinterpret_cast<unsigned char*>(dst) + p * C::PLANE_BYTES);
        if (async) {
          // mirroring keeps the parity of a sample index, so a mirrored
          // element of plane p is again in plane p
          int ix[2];
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int mm = m + t;
            ix[t] = (mm >= 0 && mm < pw) ? mm : (mirror(2 * mm + px, a.W) >> 1);
          }
          const bool direct = m >= 0 && m + 2 <= pw;
          for (int r = 0; r < C::CH; ++r) {
            const int y = y0 + r;
            const int iy = (y >= 0 && y < ph) ? y : (mirror(2 * y + py, a.H) >> 1);
            const ST* rowp = src_plane(p) + (long long)iy * a.src_pitch[p];
            ST* d = pd + r * C::ROWE + off + 2 * lane;
            if (direct && (reinterpret_cast<uintptr_t>(rowp + m) & 7) == 0) {
              ptx::cp_async_8(d, rowp + m);
            } else {
              ptx::cp_async_4(d, rowp + ix[0]);
              ptx::cp_async_4(d + 1, rowp + ix[1]);
            }
          }
          continue;
        }
        for (int r = 0; r < C::CH; ++r) {
          const int y = y0 + r;
          ST* d = pd + r * C::ROWE + off + 2 * lane;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            // sample coordinates of this element, mirrored, mapped back to a plane
            const int sy = 2 * y + py, sx = 2 * (m + t) + px;
            bool absent = false;
            int my, mx;
            if (a.H == 1) { my = 0; absent |= sy != 0; } else { my = mirror(sy, a.H); }
            if (a.W == 1) { mx = 0; absent |= sx != 0; } else { mx = mirror(sx, a.W); }
            const int q = ((my & 1) << 1) | (mx & 1);
            const ST* sp = src_plane(q) + (long long)(my >> 1) * a.src_pitch[q] + (mx >> 1);
            d[t] = absent ? StoreT<ST>::from_v(VT(0)) : *sp;
          }
        }
      }
      if (async) ptx::cp_async_arrive(bar);
      else ptx::mbar_arrive(bar);
    }
  }

  // ---- consumer --------------------------------------------------------------
  __device__ __forceinline__ Row<VT> load_row(const ST* st, int r) const {
    Row<VT> o;
    if constexpr (C::LOAD == SAMPLES) {
      const int xs = 2 * mfirst;
      const int off = xs - align_down(xs, C::A);
      const ST* p0 = st + (2 * r) * C::ROWE + off + 4 * lane;
      const ST* p1 = p0 + C::ROWE;
      ST v0[4], v1[4];
      if constexpr (C::ES == 4) {
        *reinterpret_cast<int4*>(v0) = *reinterpret_cast<const int4*>(p0);
        *reinterpret_cast<int4*>(v1) = *reinterpret_cast<const int4*>(p1);
      } else {
        *reinterpret_cast<int2*>(v0) = *reinterpret_cast<const int2*>(p0);
        *reinterpret_cast<int2*>(v1) = *reinterpret_cast<const int2*>(p1);
      }
      o.s[LL][0] = StoreT<ST>::to_v(v0[0]);
      o.s[HL][0] = StoreT<ST>::to_v(v0[1]);
      o.s[LL][1] = StoreT<ST>::to_v(v0[2]);
      o.s[HL][1] = StoreT<ST>::to_v(v0[3]);
      o.s[LH][0] = StoreT<ST>::to_v(v1[0]);
      o.s[HH][0] = StoreT<ST>::to_v(v1[1]);
      o.s[LH][1] = StoreT<ST>::to_v(v1[2]);
      o.s[HH][1] = StoreT<ST>::to_v(v1[3]);
    } else {
      const int off = mfirst - align_down(mfirst, C::A);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const ST* pp = reinterpret_cast<const ST*>(reinterpret_cast<const unsigned char*>(st) +
                                                   p * C::PLANE_BYTES) +
                       r * C::ROWE + off + 2 * lane;
        ST v[2];
        if constexpr (C::ES == 4) {
          *reinterpret_cast<int2*>(v) = *reinterpret_cast<const int2*>(pp);
        } else {
          *reinterpret_cast<int*>(v) = *reinterpret_cast<const int*>(pp);
        }
        o.s[p][0] = StoreT<ST>::to_v(v[0]);
        o.s[p][1] = StoreT<ST>::to_v(v[1]);
      }
    }
    return o;
  }

  // Per-lane output bases, computed once per strip.
  struct Out {
    ST* base[4];
    long long pitch[4];
    int rows[4];
    bool pair[4];   // both quads stored with one vector access
    bool one[2];    // quad a / quad b stored (SUBBANDS) or sample columns (SAMPLES)
    bool lane_ok;
  };

  __device__ __forceinline__ Out out_bases() const {
    Out o;
    const int m = mfirst + 2 * lane;
    o.lane_ok = m >= m0 && m < m0 + C::UQ;
    if constexpr (C::STORE == SUBBANDS) {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int pw = (p & 1) ? a.fw : a.cw;
        o.rows[p] = (p >> 1) ? a.fh : a.ch;
        o.base[p] = static_cast<ST*>(a.dst[p]) + m;
        o.pitch[p] = a.dst_pitch[p];
        o.pair[p] = m + 2 <= pw && ((reinterpret_cast<uintptr_t>(o.base[p]) & (2 * C::ES - 1)) == 0) &&
                    ((a.dst_pitch[p] * C::ES) & (2 * C::ES - 1)) == 0;
        if (p == 0) {
          o.one[0] = m < pw;
          o.one[1] = m + 1 < pw;
        }
      }
    } else {
      const int gx = 2 * m;
      o.base[0] = static_cast<ST*>(a.dst[0]) + gx;
      o.pitch[0] = a.dst_pitch[0];
      o.rows[0] = a.H;
      o.pair[0] = gx + 4 <= a.W && ((reinterpret_cast<uintptr_t>(o.base[0]) & (4 * C::ES - 1)) == 0) &&
                  ((a.dst_pitch[0] * C::ES) & (4 * C::ES - 1)) == 0;
    }
    return o;
  }

  __device__ __forceinline__ void store_row(const Out& o, const Row<VT>& r, int q) const {
    if (!o.lane_ok) return;  // halo lane
    if constexpr (C::STORE == SUBBANDS) {
      const int m = mfirst + 2 * lane;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        if (q >= o.rows[p]) continue;
        ST* rowp = o.base[p] + (long long)q * o.pitch[p];
        const ST v0 = StoreT<ST>::from_v(r.s[p][0]), v1 = StoreT<ST>::from_v(r.s[p][1]);
        if (o.pair[p]) {
          if constexpr (C::ES == 4) {
            int2 pk;
            pk.x = *reinterpret_cast<const int*>(&v0);
            pk.y = *reinterpret_cast<const int*>(&v1);
            *reinterpret_cast<int2*>(rowp) = pk;
          } else {
            __half2 h;
            h.x = *reinterpret_cast<const __half*>(&v0);
            h.y = *reinterpret_cast<const __half*>(&v1);
            *reinterpret_cast<__half2*>(rowp) = h;
          }
        } else {
          const int pw = (p & 1) ? a.fw : a.cw;
          if (m < pw) rowp[0] = v0;
          if (m + 1 < pw) rowp[1] = v1;
        }
      }
    } else {
      const int gx = 2 * (mfirst + 2 * lane);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int gy = 2 * q + rr;
        if (gy >= o.rows[0]) continue;
        ST* rowp = o.base[0] + (long long)gy * o.pitch[0];
        const int sl = rr ? LH : LL, sh = rr ? HH : HL;
        ST v[4] = {StoreT<ST>::from_v(r.s[sl][0]), StoreT<ST>::from_v(r.s[sh][0]),
                   StoreT<ST>::from_v(r.s[sl][1]), StoreT<ST>::from_v(r.s[sh][1])};
        if (o.pair[0]) {
          if constexpr (C::ES == 4) *reinterpret_cast<int4*>(rowp) = *reinterpret_cast<const int4*>(v);
          else *reinterpret_cast<int2*>(rowp) = *reinterpret_cast<const int2*>(v);
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (gx + t < a.W) rowp[t] = v[t];
        }
      }
    }
  }
};

template <class C>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    level_kernel(const __grid_constant__ TmaMaps maps, const __grid_constant__ LevelArgs a,
                 const __grid_constant__ Coefs cf, const __grid_constant__ ConvTaps ct) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cs = blockIdx.x * kWarpsPerCta + warp;
  if (cs >= a.ncs) return;  // whole warp: no CTA-wide synchronisation is used
  const int q0 = blockIdx.y * a.T;
  const int rows_out = min(a.T, a.ch - q0);
  if (rows_out <= 0) return;
  const int NS = a.nstages;

  using Tot = typename C::Tot;
  Strip<C> sp{a, maps, lane, cs * C::UQ, cs * C::UQ - C::HQ, q0 - Tot::UP,
              smem_raw + (size_t)warp * NS * C::STAGE_BYTES,
              reinterpret_cast<uint64_t*>(smem_raw + (size_t)kWarpsPerCta * NS * C::STAGE_BYTES) +
                  warp * kMaxStages};
  if (lane == 0) {
    for (int s = 0; s < NS; ++s) ptx::mbar_init(&sp.bars[s], 32);
    ptx::fence_barrier_init();
  }
  __syncwarp();

  // rows streamed: the strip plus its halo, padded to whole chunks (the
  // extra rows are mirrored image rows, lifted but never stored)
  const int nrows = rows_out + Tot::UP + Tot::DOWN;
  const int nchunks = (nrows + C::CH - 1) / C::CH;
  const int q_end = q0 + rows_out;
  for (int c = 0; c < NS - 1 && c < nchunks; ++c) sp.fill(c, c);

  const typename Strip<C>::Out ob = sp.out_bases();
  Pipe<typename C::VT, typename C::PROG> pipe;
  pipe.reset();
  for (int c = 0; c < nchunks; ++c) {
    const int cn = c + NS - 1;
    if (cn < nchunks) {
      __syncwarp();
      sp.fill(cn, cn % NS);
    }
    const int s = c % NS;
    bool ok = ptx::mbar_wait_bounded(&sp.bars[s], (c / NS) & 1, kWaitProbes);
    ok = __all_sync(kFull, ok);
    if (!ok) {
      if (lane == 0) atomicOr(a.status, 1);
      // let copies already in flight land before the warp leaves
      ptx::cp_async_wait_all();
      for (int k = c; k < nchunks && k < c + NS; ++k)
        ptx::mbar_wait_bounded(&sp.bars[k % NS], (k / NS) & 1, kWaitProbes);
      return;
    }
    const typename C::ST* st = sp.stage(s);
    const int qc = sp.yfirst + c * C::CH - Tot::DOWN;
    // unrolled by two rows: the stage windows rotate with period two, and
    // the loop body stays small enough for the instruction cache
#pragma unroll 2
    for (int r = 0; r < C::CH; ++r) {
      const Row<typename C::VT> in = sp.load_row(st, r);
      const Row<typename C::VT> out = pipe.push(in, cf, ct);
      const int q = qc + r;
      if (q >= q0 && q < q_end) sp.store_row(ob, out, q);
    }
  }
}

// Per-instantiation host glue.
template <class C>
struct Instance {
  static size_t smem(int nstages) {
    return (size_t)kWarpsPerCta * nstages * C::STAGE_BYTES + (size_t)kWarpsPerCta * kMaxStages * 8;
  }
  static KernelInfo info(int nstages) {
    KernelInfo k;
    k.hq = C::HQ;
    k.uq = C::UQ;
    k.up = C::Tot::UP;
    k.down = C::Tot::DOWN;
    k.load = (Layout)C::LOAD;
    k.store = (Layout)C::STORE;
    k.box_w = C::ROWE;
    k.box_h = C::LOAD == SAMPLES ? 2 * C::CH : C::CH;
    k.smem_bytes = smem(nstages);
    k.fn = reinterpret_cast<const void*>(&level_kernel<C>);
    k.supported = true;
    return k;
  }
  static cudaError_t launch(const LevelArgs& a, const TmaMaps& m, const Coefs& cf,
                            const ConvTaps& ct, cudaStream_t s) {
    const size_t bytes = smem(a.nstages);
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
      int optin = 0;
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaError_t e = cudaFuncSetAttribute(&level_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           optin > 0 ? optin : (int)smem(kMaxStages));
      if (e != cudaSuccess) return e;
      configured[dev] = 1;
    }
    dim3 grid((a.ncs + kWarpsPerCta - 1) / kWarpsPerCta, a.nrs);
    level_kernel<C><<<grid, kWarpsPerCta * 32, bytes, s>>>(m, a, cf, ct);
    return cudaGetLastError();
  }
};

}  // namespace dev
}  // namespace dwt
