// The small levels of one image in one launch: 2-D tiles in shared memory.
//
// Below a few million samples per level the streaming kernels of
// level_kernel.cuh are latency-bound: a warp walks its strip row after row,
// through the halo rows as well, so every level costs a chain of dependent
// row steps plus a launch, whatever its size.  Here a level is cut into
// tiles of TR x TC quadruples (the stored interior plus the scheme's halo on
// each side, recomputed by the neighbouring tiles).  A CTA of 256 threads
// holds a tile in registers, QL horizontally adjacent quadruples per
// thread, and applies the scheme's steps to all of them at once: before a
// step that reads other quadruples, every thread publishes the subbands the
// step reads to a shared-memory plane and the CTA synchronises once.  This
// is the paper's own work-group design (Sec. 6): one barrier per step that
// crosses quadruples, none for the starred schemes' local steps (Sec. 4).
//
// One cooperative launch runs several consecutive levels (the fused tail of
// a pyramid): the CTAs take the tiles of a level in turn, then meet at a
// grid barrier before the next level, which reads what the previous level
// wrote (L2-resident at these sizes).  The barrier is one counter that each
// CTA bumps once per crossing; CTA 0 adds 2^31 - (CTAs - 1) instead of 1, so
// each crossing flips the counter's top bit and leaves its other bits as
// they were: it needs no reset between launches or graph replays.  Its wait
// is bounded: a CTA that gives up raises the status word and goes on (it
// still arrives at every later crossing, which keeps the counter in step).
#pragma once

#include "level_kernel.cuh"

namespace dwt {
namespace dev {

// Tile shape of a program: TR x TC quadruples with QL per thread slot, one
// slot per thread; PR / PC rows and columns of never-written padding around
// each shared-memory plane absorb the reads of the outermost halo quads
// (whose results are discarded).
// The largest reach of one step of a program, in quads.
template <class L>
struct MaxStepReach;
template <class... S>
struct MaxStepReach<List<S...>> {
  static constexpr int v = vmax(0, S::UP..., S::DOWN..., S::LEFT..., S::RIGHT...);
};

template <class PROG, int QL_>
struct TileGeom {
  using Tot = Totals<PROG>;
  static constexpr int QL = QL_;
  static constexpr int TR = 32, TC = 32;
  static constexpr int UP = Tot::UP, DOWN = Tot::DOWN, LEFT = Tot::LEFT, RIGHT = Tot::RIGHT;
  static constexpr int IR = TR - UP - DOWN, IC = TC - LEFT - RIGHT;  // stored interior
  // padding: a step's reach in rows, and 4 columns (rows stay 16-byte aligned)
  static constexpr int PR = cmax(1, MaxStepReach<PROG>::v), PC = 4;
  static constexpr int RS = TC + 2 * PC;          // plane row stride (elements)
  static constexpr int PS = (TR + 2 * PR) * RS;   // plane size (elements)
  static constexpr int SLOTS_PER_ROW = TC / QL;
  static_assert(TR * TC / QL == kTileThreads, "one slot per thread");
  static_assert(IR > 0 && IC > 0, "halo wider than the tile");
};

// One element of a 16-byte shared-memory vector of 4-byte values.
template <typename V>
__device__ __forceinline__ V lane_of(const int4& q, int k) {
  const int b = k == 0 ? q.x : k == 1 ? q.y : k == 2 ? q.z : q.w;
  if constexpr (std::is_integral<V>::value) return b;
  else return __int_as_float(b);
}

// Accessor of a tile step: the thread's own quads from registers, the
// others from the published plane (p points at the slot's first quad in
// plane 0).  A neighbouring row over the slot's own columns is read as one
// 16-byte vector (identical vector reads of a step are merged), the columns
// beyond the slot one by one.
template <typename V, int QL, int RS, int PS>
struct TileAcc {
  const Row<V, QL>& own;
  const V* p;
  template <int S, int DY, int DX, int J>
  __device__ __forceinline__ V at() const {
    if constexpr (DY == 0 && J + DX >= 0 && J + DX < QL) {
      return own.s[S][J + DX];
    } else if constexpr (sizeof(V) == 4 && QL == 4 && J + DX >= 0 && J + DX < QL) {
      const int4 q = *reinterpret_cast<const int4*>(p + S * PS + DY * RS);
      return lane_of<V>(q, J + DX);
    } else {
      return p[S * PS + DY * RS + J + DX];
    }
  }
};

// Local steps read nothing but the quad itself.
template <typename V, int QL>
struct OwnAcc {
  const Row<V, QL>& own;
  template <int S, int DY, int DX, int J>
  __device__ __forceinline__ V at() const {
    static_assert(DY == 0 && J + DX >= 0 && J + DX < QL, "a local step reads its own quads only");
    return own.s[S][J + DX];
  }
};

template <class G, typename V, class L>
struct TileSteps;
template <class G, typename V>
struct TileSteps<G, V, List<>> {
  template <class CS>
  __device__ __forceinline__ static void run(Row<V, G::QL>&, V*, int, int&, const CS&, const ConvTaps&) {}
};
template <class G, typename V, class S0, class... S>
struct TileSteps<G, V, List<S0, S...>> {
  template <class CS>
  __device__ __forceinline__ static void run(Row<V, G::QL>& st, V* xb, int slot_off, int& cur, const CS& c,
                                             const ConvTaps& t) {
    constexpr int QL = G::QL;
    // the padding around each plane covers one step's reach
    static_assert(S0::UP <= G::PR && S0::DOWN <= G::PR && S0::LEFT <= G::PC && S0::RIGHT <= G::PC,
                  "a step reaches beyond the plane padding");
    Row<V, QL> o;
    if constexpr (S0::NEIGHBOUR_SRCS != 0) {
      V* buf = xb + cur * 4 * G::PS;
      V* me = buf + slot_off;
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (S0::NEIGHBOUR_SRCS & (1u << s)) {
          if constexpr (sizeof(V) == 4 && QL == 4) {
            // the slot's QL quads as one 16-byte vector (rows are aligned)
            *reinterpret_cast<int4*>(me + s * G::PS) =
                make_int4(bits32(st.s[s][0]), bits32(st.s[s][1]), bits32(st.s[s][2]), bits32(st.s[s][3]));
          } else {
#pragma unroll
            for (int j = 0; j < QL; ++j) me[s * G::PS + j] = st.s[s][j];
          }
        }
      __syncthreads();
      S0::template eval<QL>(st, TileAcc<V, QL, G::RS, G::PS>{st, me}, o, c, t);
      cur ^= 1;
    } else {
      S0::template eval<QL>(st, OwnAcc<V, QL>{st}, o, c, t);
    }
    st = o;
    TileSteps<G, V, List<S...>>::run(st, xb, slot_off, cur, c, t);
  }
};

// Loads of data another CTA of the same launch wrote: from L2 (.cg), never
// a stale L1 line.
template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const int v = __ldcg(reinterpret_cast<const int*>(p));
    T r;
    memcpy(&r, &v, 4);
    return r;
  } else {
    const unsigned short v = __ldcg(reinterpret_cast<const unsigned short*>(p));
    T r;
    memcpy(&r, &v, 2);
    return r;
  }
}

// The QL quads (qy, qx0 .. qx0 + QL - 1) of a level with whole-sample
// symmetric extension (the level has both sides >= 2).
template <class C, int QL>
__device__ __forceinline__ Row<typename C::VT, QL> tile_load(const LevelArgs& a, int qy, int qx0) {
  using ST = typename C::ST;
  using VT = typename C::VT;
  Row<VT, QL> r;
  if constexpr (C::LOAD == SAMPLES) {
    const ST* src = static_cast<const ST*>(a.src[0]);
    const long long pitch = a.src_pitch[0];
    const int x0 = 2 * qx0;
#pragma unroll
    for (int py = 0; py < 2; ++py) {
      const ST* row = src + (long long)mirror(2 * qy + py, a.H) * pitch;
      ST v[2 * QL];
      if (x0 >= 0 && x0 + 2 * QL <= a.W && (reinterpret_cast<uintptr_t>(row + x0) & 15) == 0 &&
          sizeof(ST) * 2 * QL >= 16) {
#pragma unroll
        for (int k = 0; k < (int)(sizeof(ST) * 2 * QL / 16); ++k) {
          const int4 q = __ldcg(reinterpret_cast<const int4*>(row + x0) + k);
          memcpy(&v[k * 16 / sizeof(ST)], &q, 16);
        }
      } else {
#pragma unroll
        for (int t = 0; t < 2 * QL; ++t) v[t] = ld_cg(row + mirror(x0 + t, a.W));
      }
#pragma unroll
      for (int j = 0; j < QL; ++j) {
        r.s[2 * py][j] = StoreT<ST>::to_v(v[2 * j]);
        r.s[2 * py + 1][j] = StoreT<ST>::to_v(v[2 * j + 1]);
      }
    }
  } else {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int py = p >> 1, px = p & 1;
      const int pw = px ? a.fw : a.cw, ph = py ? a.fh : a.ch;
      const ST* base = static_cast<const ST*>(a.src[p]);
      const int y = (qy >= 0 && qy < ph) ? qy : (mirror(2 * qy + py, a.H) >> 1);
      const ST* row = base + (long long)y * a.src_pitch[p];
#pragma unroll
      for (int j = 0; j < QL; ++j) {
        const int m = qx0 + j;
        const int x = (m >= 0 && m < pw) ? m : (mirror(2 * m + px, a.W) >> 1);
        r.s[p][j] = StoreT<ST>::to_v(ld_cg(row + x));
      }
    }
  }
  return r;
}

// Stores the slot's quads that lie in the tile interior and in the level.
template <class C, int QL>
__device__ __forceinline__ void tile_store(const LevelArgs& a, const Row<typename C::VT, QL>& r, int qy, int qx0,
                                           int jlo, int jhi) {
  using ST = typename C::ST;
  if constexpr (C::STORE == SUBBANDS) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int pw = (p & 1) ? a.fw : a.cw, ph = (p >> 1) ? a.fh : a.ch;
      if (qy >= ph) continue;
      ST* row = static_cast<ST*>(a.dst[p]) + (long long)qy * a.dst_pitch[p];
      ST v[QL];
#pragma unroll
      for (int j = 0; j < QL; ++j) v[j] = StoreT<ST>::from_v(r.s[p][j]);
      if (jlo == 0 && jhi == QL && qx0 + QL <= pw && sizeof(ST) == 4) {
        store_run<QL>(row + qx0, v);
      } else {
#pragma unroll
        for (int j = 0; j < QL; ++j)
          if (j >= jlo && j < jhi && qx0 + j < pw) row[qx0 + j] = v[j];
      }
    }
  } else {
    ST* dst = static_cast<ST*>(a.dst[0]);
#pragma unroll
    for (int py = 0; py < 2; ++py) {
      const int y = 2 * qy + py;
      if (y >= a.H) continue;
      ST* row = dst + (long long)y * a.dst_pitch[0];
      ST v[2 * QL];
#pragma unroll
      for (int j = 0; j < QL; ++j) {
        v[2 * j] = StoreT<ST>::from_v(r.s[2 * py][j]);
        v[2 * j + 1] = StoreT<ST>::from_v(r.s[2 * py + 1][j]);
      }
      const int x0 = 2 * qx0;
      if (jlo == 0 && jhi == QL && x0 + 2 * QL <= a.W && sizeof(ST) == 4) {
        store_run<2 * QL>(row + x0, v);
      } else {
#pragma unroll
        for (int t = 0; t < 2 * QL; ++t)
          if (t >= 2 * jlo && t < 2 * jhi && x0 + t < a.W) row[x0 + t] = v[t];
      }
    }
  }
}

// Grid barrier (see the file comment).  Every CTA calls it the same number
// of times; all of the CTA's threads call it.  Returns false (and raises
// *status) if the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, uint32_t limit, int* status) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    __threadfence();
    const unsigned old = atomicAdd(ctr, add);
    for (uint32_t spins = 0;; ++spins) {
      unsigned cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(ctr) : "memory");
      if ((old ^ cur) & 0x80000000u) break;
      if (spins >= limit) {
        ok = 0;
        atomicOr(status, 1);
        break;
      }
      if (spins >= 256) __nanosleep(32);  // a short spin first: most crossings complete within it
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// None of the tail programs reads Convolution taps.
static __constant__ ConvTaps kTileNoTaps;

template <class C>
__global__ void __launch_bounds__(kTileThreads, C::MINB) tail_kernel(const __grid_constant__ TailParams P) {
  using VT = typename C::VT;
  using G = TileGeom<typename C::PROG, C::QL>;
  constexpr int QL = G::QL;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  VT* xb = reinterpret_cast<VT*>(smem_raw);
  // the padding is never written by a step: zero it once (its values only
  // reach discarded halo quads, but they stay deterministic)
  for (int i = threadIdx.x; i < 2 * 4 * G::PS; i += kTileThreads) xb[i] = VT(0);
  ptx::launch_dependents();
  // the previous kernel in the stream may still be running: every read and
  // write of level data comes after this point
  ptx::wait_prerequisites();
  __syncthreads();
  const int r = threadIdx.x / G::SLOTS_PER_ROW;
  const int c0 = (threadIdx.x % G::SLOTS_PER_ROW) * QL;
  const int slot_off = (G::PR + r) * G::RS + G::PC + c0;
  int cur = 0;
  for (int li = 0; li < P.nlevels; ++li) {
    const TileLevel& L = P.lv[li];
    const LevelArgs& a = L.a;
    const auto coefs = CoefSource<typename C::CSRC>::make(L.cf);
    int ntiles = L.ntx * L.nty;
    if (a.hold && blockIdx.x == 0) {
      // failure injection: CTA 0 waits, bounded, on a flag nothing sets,
      // before it loads anything; it then skips its tiles of this level
      __shared__ int held;
      if (threadIdx.x < 32) {
        const bool ok = wait_flag(a.hold, a.spins);
        if (threadIdx.x == 0) {
          held = ok ? 0 : 1;
          if (!ok) atomicOr(a.status, 1);
        }
      }
      __syncthreads();
      if (held) ntiles = 0;
    }
    // the first tile's inputs, then each tile's computation overlaps the
    // loads of the CTA's next tile of the level
    Row<VT, QL> next;
    if ((int)blockIdx.x < ntiles) {
      const int ty = blockIdx.x / L.ntx, tx = blockIdx.x - ty * L.ntx;
      next = tile_load<C, QL>(a, ty * G::IR - G::UP + r, tx * G::IC - G::LEFT + c0);
    }
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int ty = t / L.ntx, tx = t - ty * L.ntx;
      const int qy = ty * G::IR - G::UP + r;
      const int qx0 = tx * G::IC - G::LEFT + c0;
      Row<VT, QL> st = next;
      const int tn = t + gridDim.x;
      if (tn < ntiles) {
        const int nty = tn / L.ntx, ntx = tn - nty * L.ntx;
        next = tile_load<C, QL>(a, nty * G::IR - G::UP + r, ntx * G::IC - G::LEFT + c0);
      }
      TileSteps<G, VT, typename C::PROG>::run(st, xb, slot_off, cur, coefs, kTileNoTaps);
      // interior rows and columns of the tile
      if (r >= G::UP && r < G::UP + G::IR && qy < a.ch) {
        const int jlo = max(0, G::LEFT - c0), jhi = min(QL, G::LEFT + G::IC - c0);
        if (jlo < jhi && qx0 + jlo < a.cw) tile_store<C, QL>(a, st, qy, qx0, jlo, jhi);
      }
    }
    if (li + 1 < P.nlevels) grid_barrier(P.barrier, a.spins, a.status);
  }
}

// Configuration of a tail kernel: storage and arithmetic types, the step
// program, what a level reads and writes, and the coefficient source.
// MINB: resident CTAs per SM the register budget is cut for (4: 64
// registers a thread; the merged Polyphase steps take 2, 128 registers).
template <typename ST_, typename VT_, class PROG_, int LOAD_, int STORE_, class CSRC_, int MINB_ = 4>
struct TailCfg {
  using ST = ST_;
  using VT = VT_;
  using PROG = PROG_;
  using CSRC = CSRC_;
  static constexpr int LOAD = LOAD_, STORE = STORE_;
  static constexpr int QL = 4;
  static constexpr int MINB = MINB_;
};

// Host glue of one tail kernel.
template <class C>
struct TailInstance {
  using G = TileGeom<typename C::PROG, C::QL>;
  static size_t smem() { return sizeof(typename C::VT) * 2 * 4 * (size_t)G::PS; }
  static void geom(int* inner_rows, int* inner_cols) {
    *inner_rows = G::IR;
    *inner_cols = G::IC;
  }
  static const void* fn() { return reinterpret_cast<const void*>(&tail_kernel<C>); }
  static cudaError_t launch(const TailParams& p, int blocks, cudaStream_t s) {
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
      cudaError_t e = cudaFuncSetAttribute(&tail_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());
      if (e != cudaSuccess) return e;
      configured[dev] = 1;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kTileThreads);
    cfg.dynamicSmemBytes = smem();
    cfg.stream = s;
    // cooperative: every CTA resident at once (they meet at grid
    // barriers); programmatic dependent launch as between level kernels
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaError_t e = cudaLaunchKernelEx(&cfg, tail_kernel<C>, p);
    if (e != cudaSuccess) {
      // without programmatic serialisation if the two attributes do not combine
      cudaGetLastError();
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, tail_kernel<C>, p);
    }
    return e;
  }
};

}  // namespace dev
}  // namespace dwt
