// One transform level (or one row-column pass) as a streaming kernel.
//
// Work decomposition.  Each warp owns a strip: 32*QL quadruple columns wide
// (QL per lane) and T quadruple rows tall.  The outer HQ quad columns on
// each side and UP / DOWN quad rows are the lifting halo (the overlapping
// tiles of Sec. 6): they are loaded and lifted but not stored, so that every
// stored coefficient only depends on samples the strip holds.  The warp
// walks down its strip one quad row at a time; every step of the scheme is
// a stage whose window keeps the rows of its input state it still needs
// (vertical neighbours), while horizontal neighbours are exchanged with
// warp shuffles.  What the paper synchronises with a work-group barrier
// between two steps is, here, the hand-over of a row from one stage's
// output to the next stage's window (vertical) and a shuffle (horizontal);
// no CTA-wide barrier is needed.  Each strip is a one-warp CTA (kWarpsPerCta
// consecutive strips per CTA in general; more per CTA measured no faster),
// dispatched border columns first (strip_coords).
//
// Loads.  Rows arrive in chunks of CH quad rows through a per-warp ring of
// shared-memory stages, filled ahead of use: a chunk lying inside the image
// is one 2-D TMA box (cp.async.bulk.tensor, one box per source plane) when
// the source is 16-byte aligned; otherwise each lane issues cp.async copies,
// with whole-sample symmetric mirroring applied to the addresses at the
// image border.  Images with a length-1 axis use a synchronous fill that
// writes zeros for the samples that do not exist.  Every stage has one
// mbarrier with 32 expected arrivals per fill; waits on it are bounded and
// report to the launch's status word.
//
// Stores.  Each lane writes its QL quadruples of a subband row as one vector
// (128-bit for float32 and QL = 4) or, for sample output, its 2*QL samples
// of each sample row.
#pragma once

#include <type_traits>

#include <cuda_fp16.h>

#include "programs.cuh"
#include "ptx.cuh"

namespace dwt {
namespace dev {


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

// Copies of N bytes (N a power of two, 4..32) between aligned addresses.
template <int N>
__device__ __forceinline__ void copy_bytes(void* d, const void* s) {
  if constexpr (N == 32) {
    reinterpret_cast<int4*>(d)[0] = reinterpret_cast<const int4*>(s)[0];
    reinterpret_cast<int4*>(d)[1] = reinterpret_cast<const int4*>(s)[1];
  } else if constexpr (N == 16) {
    *reinterpret_cast<int4*>(d) = *reinterpret_cast<const int4*>(s);
  } else if constexpr (N == 8) {
    *reinterpret_cast<int2*>(d) = *reinterpret_cast<const int2*>(s);
  } else {
    static_assert(N == 4, "unsupported copy size");
    *reinterpret_cast<int*>(d) = *reinterpret_cast<const int*>(s);
  }
}

// The bits of a 4-byte sample.
template <typename T>
__device__ __forceinline__ int bits32(T x) {
  if constexpr (sizeof(T) == 4 && !std::is_integral<T>::value) return __float_as_int(x);
  else return static_cast<int>(x);
}

// Stores the N 4-byte values v at p, where p lies A elements past a 16-byte
// boundary, with the widest aligned stores: 4-byte pieces up to an 8-byte
// boundary, 8-byte pieces up to a 16-byte one, then 16-byte pieces.  The
// vectors are assembled from the values' bits (no reinterpreted arrays).
template <int N, int A, typename T>
__device__ __forceinline__ void store_split(T* p, const T* v) {
  if constexpr (N > 0) {
    if constexpr (A == 0 && N >= 4) {
      *reinterpret_cast<int4*>(p) = make_int4(bits32(v[0]), bits32(v[1]), bits32(v[2]), bits32(v[3]));
      store_split<N - 4, 0>(p + 4, v + 4);
    } else if constexpr (A % 2 == 0 && N >= 2) {
      *reinterpret_cast<int2*>(p) = make_int2(bits32(v[0]), bits32(v[1]));
      store_split<N - 2, (A + 2) % 4>(p + 2, v + 2);
    } else {
      *reinterpret_cast<int*>(p) = bits32(v[0]);
      store_split<N - 1, (A + 1) % 4>(p + 1, v + 1);
    }
  }
}

// N in-bounds 4-byte values at p, whose offset from a 16-byte boundary is
// the same in every lane of the warp (lanes store runs 16 or 32 bytes apart).
template <int N, typename T>
__device__ __forceinline__ void store_run(T* p, const T* v) {
  switch ((reinterpret_cast<uintptr_t>(p) >> 2) & 3) {
    case 0: store_split<N, 0>(p, v); break;
    case 1: store_split<N, 1>(p, v); break;
    case 2: store_split<N, 2>(p, v); break;
    default: store_split<N, 3>(p, v); break;
  }
}

template <typename ST_, typename VT_, class PROG_, int LOAD_, int STORE_, int QL_ = 4, int CH_ = 2,
          int MINW_ = 16, class CSRC_ = RtTag>
struct Cfg {
  using CSRC = CSRC_;  // coefficient source: RtTag (from Coefs) or StCoefs<...>
  using ST = ST_;
  using VT = VT_;
  using PROG = PROG_;
  using Tot = Totals<PROG>;
  static constexpr int LOAD = LOAD_, STORE = STORE_;
  static constexpr int QL = QL_;  // quadruples per lane
  static constexpr int CH = CH_;  // quad rows per ring stage
  static constexpr int MIN_WARPS = MINW_;  // warps per SM the register budget must allow
  static constexpr int WQ = 32 * QL;  // quadruple columns per warp
  // halo quads per side: covers the stencil reach and keeps each lane's
  // first quadruple a multiple of QL (aligned vector stores)
  static constexpr int HQ = ((cmax(Tot::LEFT, Tot::RIGHT) + QL - 1) / QL) * QL;
  static constexpr int UQ = WQ - 2 * HQ;
  static constexpr int ES = sizeof(ST);
  static constexpr int A = 16 / ES;  // elements per 16 bytes
  // smem row: the warp's span plus alignment slack when the box start can
  // be misaligned (a TMA box is at most 256 elements wide)
  static constexpr int SPAN = LOAD == SAMPLES ? 2 * WQ : WQ;
  static constexpr bool ALIGNED_START = LOAD == SAMPLES ? ((2 * HQ) % A == 0 && (2 * UQ) % A == 0)
                                                        : (HQ % A == 0 && UQ % A == 0);
  static constexpr int ROWE = ALIGNED_START ? SPAN : SPAN + A;
  static constexpr int ROWS = LOAD == SAMPLES ? 2 * CH : CH;  // smem rows per plane
  static constexpr int PLANE_BYTES = ((ROWS * ROWE * ES + 127) / 128) * 128;
  static constexpr int BOX_BYTES = ROWS * ROWE * ES;
  static constexpr int NPLANES = LOAD == SAMPLES ? 1 : 4;
  static constexpr int STAGE_BYTES = NPLANES * PLANE_BYTES;
  static_assert(ROWE <= 256, "TMA box wider than 256 elements");
  // A subband plane whose start is not 16-byte aligned while its rows are
  // (HL and HH at column ceil(w/2) of coefficient rows padded to 16 bytes)
  // is loaded by TMA from the aligned column at or before its start (the
  // tensor map is anchored there: no box coordinate is ever unaligned).  A
  // box with A - 1 columns of room takes the shift as it is; a box exactly
  // as wide as the span takes it when the halo quadruples the stencil never
  // reads (HQ - LEFT on the left, HQ - RIGHT on the right) cover A - 1
  // columns, by starting the box up to HQ - RIGHT columns late.
  static constexpr bool WIDE_BOX = ROWE >= SPAN + A - 1;
  static constexpr bool REALIGN =
      LOAD == SUBBANDS && (WIDE_BOX || 2 * HQ - Tot::LEFT - Tot::RIGHT >= A - 1);
  static_assert(UQ > 0 && HQ <= 2 * QL, "halo too wide for the lane layout");
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
  static constexpr int QL = C::QL;
  const LevelArgs& a;
  const TmaMaps& maps;
  int lane, m0, mfirst, yfirst;
  unsigned char* sm;
  uint64_t* bars;
  int stride = C::STAGE_BYTES;  // bytes between ring stages
  bool box = false;             // chunks land in the TMA box layout (see boxed())
  // Subband planes of odd column parity (HL and HH, planes 1 and 3, which
  // share one offset; the even planes start at column 0 of their rows in
  // every layout and are never realigned): the first column of their box
  // in tensor-map coordinates (x1).  A realigned strip (box and a nonzero
  // a.src_off[1]) starts that map a.src_off[1] columns before the planes'
  // first element; otherwise map and plane columns coincide.
  int x1 = 0;

  __device__ __forceinline__ int offu(int px) const {
    if constexpr (C::REALIGN) return (px && box) ? a.src_off[1] : 0;
    else return 0;
  }
  // plane column at shared-memory column 0 of a box row of parity px
  __device__ __forceinline__ int be(int px) const {
    if constexpr (C::REALIGN) return px ? x1 - offu(1) : align_down(mfirst, C::A);
    else return align_down(mfirst, C::A);
  }

  // Box columns of the odd-parity planes: with `realign`, from the offset
  // the host encoded their tensor maps with (a.src_off[1]), else from the
  // planes' own starts.  Called before `box` is decided (with realign) and
  // again if the strip does not take the box layout (without).
  __device__ __forceinline__ void set_box_cols(bool realign) {
    if constexpr (C::REALIGN) {
      const int off = realign ? a.src_off[1] : 0;
      int x = align_down(mfirst + off, C::A);
      if (!C::WIDE_BOX && off != 0 && mfirst + off - x > C::HQ - C::Tot::RIGHT) x += C::A;
      x1 = x;
      box = realign;  // offu() reads the offset while boxed() decides
    }
  }

  __device__ __forceinline__ ST* plane(int s, int p) const {
    return reinterpret_cast<ST*>(sm + (size_t)s * stride + p * C::PLANE_BYTES);
  }
  __device__ __forceinline__ const ST* src_plane(int p) const {
    return static_cast<const ST*>(a.src[p]);
  }
  // first smem column of the lane's elements
  __device__ __forceinline__ int lane_col() const {
    if constexpr (C::LOAD == SAMPLES) {
      const int xs = 2 * mfirst;
      return (xs - align_down(xs, C::A)) + 2 * QL * lane;
    } else {
      return (mfirst - align_down(mfirst, C::A)) + QL * lane;
    }
  }

  // ---- border columns --------------------------------------------------------
  // A strip whose columns leave the image still loads by TMA (the box reads
  // zeros outside the tensor) when every mirrored value its halo needs lies
  // inside the box.  The lanes holding such columns then read the mirrored
  // shared-memory column instead of their own (load_row); in-image columns
  // hold their true value whichever way the chunk was filled.  Columns
  // further out never reach a stored coefficient; they read a clamped,
  // in-box column.
  __device__ __forceinline__ bool cols_inside() const {
    if constexpr (C::LOAD == SAMPLES) return 2 * mfirst >= 0 && 2 * mfirst + C::SPAN <= a.W;
    else return mfirst >= 0 && mfirst + C::WQ <= a.fw;
  }
  // box-relative index of the mirror of sample column x (SAMPLES) or of
  // quad m of a plane of column parity px (SUBBANDS)
  __device__ __forceinline__ int mirror_col(int x, int px) const {
    if constexpr (C::LOAD == SAMPLES) {
      return mirror(x, a.W) - align_down(2 * mfirst, C::A);
    } else {
      return (mirror(2 * x + px, a.W) >> 1) - be(px);
    }
  }
  __device__ __forceinline__ bool cols_by_tma() const {
    if (cols_inside()) return true;
    // the farthest halo element on each side must mirror into the box
    if constexpr (C::LOAD == SAMPLES) {
      const int lo = 2 * mfirst;
      const int m_lo = lo < 0 ? mirror_col(lo, 0) : 0;
      const int m_hi = lo + C::SPAN > a.W ? mirror_col(a.W + 2 * C::HQ, 0) : 0;
      return m_lo >= 0 && m_lo < C::ROWE && m_hi >= 0 && m_hi < C::ROWE;
    } else {
      bool ok = true;
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        const int pw = px ? a.fw : a.cw;
        if (mfirst < 0) {
          const int s = mirror_col(mfirst, px);
          ok = ok && s >= 0 && s < C::ROWE;
        }
        if (mfirst + C::WQ > pw) {
          const int s = mirror_col(pw + C::HQ, px);
          ok = ok && s >= 0 && s < C::ROWE;
        }
      }
      return ok;
    }
  }
  // ---- fills ---------------------------------------------------------------
  // The box a TMA load would bring, copied by the lanes with cp.async: for
  // chunks the TMA engine cannot take (rows to mirror at the top or bottom,
  // a plane whose base or pitch is not 16-byte aligned, as the Mallat bands
  // of most odd sizes are).  The shared-memory layout is the TMA box's, so
  // the consumer side is the same.  Lanes copy consecutive 16-byte groups
  // (4-byte ones on rows that are not 16-byte aligned); columns outside the
  // plane are not copied (they are never read as values).
  __device__ __forceinline__ static bool box_copyable(const void* base, long long pitch_elems) {
    // 4-byte cp.async needs 4-byte aligned rows: always true for 32-bit
    // samples; float16 rows need an even element offset
    return C::ES == 4 ||
           ((reinterpret_cast<uintptr_t>(base) | (uintptr_t)(pitch_elems * C::ES)) & 3) == 0;
  }
  __device__ __forceinline__ void copy_box_row(ST* d, const ST* row, int x0, int pw) const {
    const ST* g = row + x0;
    if ((reinterpret_cast<uintptr_t>(g) & 15) == 0) {
      constexpr int GE = 16 / C::ES;  // elements per group
#pragma unroll
      for (int k = 0; k < (C::ROWE / GE + 31) / 32; ++k) {
        const int gi = lane + 32 * k;
        const int x = x0 + gi * GE;
        if (gi < C::ROWE / GE && x >= 0 && x < pw) {
          if (x + GE <= pw) ptx::cp_async_16(d + gi * GE, g + gi * GE);
          else ptx::cp_async_16_part(d + gi * GE, g + gi * GE, (uint32_t)((pw - x) * C::ES));
        }
      }
    } else {
      constexpr int GE = 4 / C::ES;
#pragma unroll
      for (int k = 0; k < (C::ROWE / GE + 31) / 32; ++k) {
        const int gi = lane + 32 * k;
        const int x = x0 + gi * GE;
        if (gi < C::ROWE / GE && x >= 0 && x < pw) {
          if (x + GE <= pw) ptx::cp_async_4(d + gi * GE, g + gi * GE);
          else ptx::cp_async_4_part(d + gi * GE, g + gi * GE, (uint32_t)((pw - x) * C::ES));
        }
      }
    }
  }

  // Whether every chunk of this strip is filled in the TMA box layout (by
  // the TMA engine where it can, by box copies elsewhere): the box must hold
  // every mirrored column the halo needs, and the planes must allow cp.async.
  // Border lanes then read remapped columns (remap_cols); otherwise every
  // lane's elements are filled with their mirrored values directly.
  __device__ __forceinline__ bool boxed() const {
    if (a.W < 2 || a.H < 2 || !cols_by_tma()) return false;
    if constexpr (C::LOAD == SAMPLES) {
      return box_copyable(a.src[0], a.src_pitch[0]);
    } else {
      return box_copyable(copy_base(0), a.src_pitch[0]) && box_copyable(copy_base(1), a.src_pitch[1]) &&
             box_copyable(copy_base(2), a.src_pitch[2]) && box_copyable(copy_base(3), a.src_pitch[3]);
    }
  }
  // Where box copies of subband plane p start: the column its tensor map
  // starts at (offu(p & 1) columns before the plane's first element).
  __device__ __forceinline__ const ST* copy_base(int p) const { return src_plane(p) - offu(p & 1); }

  __device__ void fill(int c, int s) const {
    const int y0 = yfirst + c * C::CH;
    uint64_t* bar = &bars[s];
    const bool tiny = a.W < 2 || a.H < 2;
    const int col = lane_col();
    if constexpr (C::LOAD == SAMPLES) {
      const int sy0 = 2 * y0, xs = 2 * mfirst;
      if (box && a.src_tma && sy0 >= 0 && sy0 + C::ROWS <= a.H) {
        if (lane == 0) {
          ptx::fence_proxy_async_smem();
          ptx::mbar_arrive_expect_tx(bar, C::BOX_BYTES);
          ptx::tma_load_2d(plane(s, 0), &maps.m[0], align_down(xs, C::A), sy0, bar);
        } else {
          ptx::mbar_arrive(bar);
        }
        return;
      }
      if (box) {
        const ST* src = src_plane(0);
        const int x0 = align_down(xs, C::A);
#pragma unroll 1
        for (int j = 0; j < C::ROWS; ++j)
          copy_box_row(plane(s, 0) + j * C::ROWE, src + (long long)mirror(sy0 + j, a.H) * a.src_pitch[0], x0,
                       a.W);
        ptx::cp_async_arrive(bar);
        return;
      }
      const ST* src = src_plane(0);
      const long long pitch = a.src_pitch[0];
      const int gx = xs + 2 * QL * lane;
      if (!tiny && C::ES == 4) {
        int ix[2 * QL];
#pragma unroll
        for (int t = 0; t < 2 * QL; ++t) ix[t] = mirror(gx + t, a.W);
        const bool direct = gx >= 0 && gx + 2 * QL <= a.W;
        for (int j = 0; j < C::ROWS; ++j) {
          const ST* rowp = src + (long long)mirror(sy0 + j, a.H) * pitch;
          ST* d = plane(s, 0) + j * C::ROWE + col;
          if (direct && ((reinterpret_cast<uintptr_t>(rowp + gx) & 15) == 0)) {
#pragma unroll
            for (int t = 0; t < 2 * QL; t += 4) ptx::cp_async_16(d + t, rowp + gx + t);
          } else {
#pragma unroll
            for (int t = 0; t < 2 * QL; ++t) ptx::cp_async_4(d + t, rowp + ix[t]);
          }
        }
        ptx::cp_async_arrive(bar);
        return;
      }
      // synchronous fill: float16 off the TMA path, or an axis of length 1
      for (int j = 0; j < C::ROWS; ++j) {
        const int gy = sy0 + j;
        const bool rabs = (a.H == 1 && gy != 0);
        const ST* rowp = src + (long long)(a.H == 1 ? 0 : mirror(gy, a.H)) * pitch;
        ST* d = plane(s, 0) + j * C::ROWE + col;
#pragma unroll
        for (int t = 0; t < 2 * QL; ++t) {
          const int x = gx + t;
          const bool cabs = (a.W == 1 && x != 0);
          d[t] = (rabs || cabs) ? StoreT<ST>::from_v(VT(0)) : rowp[a.W == 1 ? 0 : mirror(x, a.W)];
        }
      }
      ptx::mbar_arrive(bar);
    } else {
      // four subband planes; the lane covers quads mfirst + QL*lane + (0..QL-1)
      const int tma = a.src_tma & 15;
      if (box && tma && y0 >= 0 && y0 + C::CH <= a.fh) {
        if (tma == 15) {
          if (lane == 0) {
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive_expect_tx(bar, 4 * C::BOX_BYTES);
#pragma unroll
            for (int p = 0; p < 4; ++p)
              ptx::tma_load_2d(plane(s, p), &maps.m[p], be(p & 1) + offu(p & 1), y0, bar);
          } else {
            ptx::mbar_arrive(bar);
          }
          return;
        }
        // planes with a tensor map by TMA, the others (a base or pitch that
        // is not 16-byte aligned) by box copies; the rows lie inside every
        // plane.  The barrier completes when the TMA bytes have landed and
        // every lane's copies are done (one arrival per lane).
        if (lane == 0) {
          ptx::fence_proxy_async_smem();
          ptx::mbar_expect_tx(bar, (uint32_t)__popc(tma) * C::BOX_BYTES);
#pragma unroll
          for (int p = 0; p < 4; ++p)
            if ((tma >> p) & 1) ptx::tma_load_2d(plane(s, p), &maps.m[p], be(p & 1) + offu(p & 1), y0, bar);
        }
#pragma unroll 1
        for (int p = 0; p < 4; ++p) {
          if ((tma >> p) & 1) continue;
          const int px = p & 1;
          const int pw = px ? a.fw : a.cw;
#pragma unroll 1
          for (int r = 0; r < C::CH; ++r)
            copy_box_row(plane(s, p) + r * C::ROWE, copy_base(p) + (long long)(y0 + r) * a.src_pitch[p],
                         be(px) + offu(px), pw + offu(px));
        }
        ptx::cp_async_arrive(bar);
        return;
      }
      if (box) {
#pragma unroll 1
        for (int p = 0; p < 4; ++p) {
          const int py = p >> 1, px = p & 1;
          const int pw = px ? a.fw : a.cw, ph = py ? a.fh : a.ch;
#pragma unroll 1
          for (int r = 0; r < C::CH; ++r) {
            const int y = y0 + r;
            // mirroring keeps the parity of a sample index: a mirrored row
            // of plane p is again a row of plane p
            const int iy = (y >= 0 && y < ph) ? y : (mirror(2 * y + py, a.H) >> 1);
            copy_box_row(plane(s, p) + r * C::ROWE, copy_base(p) + (long long)iy * a.src_pitch[p],
                         be(px) + offu(px), pw + offu(px));
          }
        }
        ptx::cp_async_arrive(bar);
        return;
      }
      const bool async = !tiny && C::ES == 4;
      const int m = mfirst + QL * lane;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int py = p >> 1, px = p & 1;
        const int pw = px ? a.fw : a.cw, ph = py ? a.fh : a.ch;
        if (async) {
          // mirroring keeps the parity of a sample index, so a mirrored
          // element of plane p is again in plane p
          int ix[QL];
#pragma unroll
          for (int t = 0; t < QL; ++t) {
            const int mm = m + t;
            ix[t] = (mm >= 0 && mm < pw) ? mm : (mirror(2 * mm + px, a.W) >> 1);
          }
          const bool direct = m >= 0 && m + QL <= pw;
          for (int r = 0; r < C::CH; ++r) {
            const int y = y0 + r;
            const int iy = (y >= 0 && y < ph) ? y : (mirror(2 * y + py, a.H) >> 1);
            const ST* rowp = src_plane(p) + (long long)iy * a.src_pitch[p];
            ST* d = plane(s, p) + r * C::ROWE + col;
            if (direct && (reinterpret_cast<uintptr_t>(rowp + m) & (QL * 4 - 1)) == 0) {
              if constexpr (QL == 4) ptx::cp_async_16(d, rowp + m);
              else ptx::cp_async_8(d, rowp + m);
            } else {
#pragma unroll
              for (int t = 0; t < QL; ++t) ptx::cp_async_4(d + t, rowp + ix[t]);
            }
          }
          continue;
        }
        for (int r = 0; r < C::CH; ++r) {
          const int y = y0 + r;
          ST* d = plane(s, p) + r * C::ROWE + col;
#pragma unroll
          for (int t = 0; t < QL; ++t) {
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
  // Border lanes: the shared-memory column each of the lane's elements
  // reads (one byte per element, computed once per strip by remap_cols), and
  // a mask of the elements too far out to reach any stored coefficient.
  struct Remap {
    bool on;
    uint32_t col[2];
    uint32_t zero;
  };

  __device__ __forceinline__ Row<VT, QL> load_row(int s, int r, const Remap& rm) const {
    Row<VT, QL> o;
    const int col = lane_col();
    if constexpr (C::LOAD == SAMPLES) {
      // row 2r: LL HL LL HL ..., row 2r+1: LH HH LH HH ...
      ST v0[2 * QL], v1[2 * QL];
      const ST* p0 = plane(s, 0) + (2 * r) * C::ROWE;
      if (!rm.on) {
        copy_bytes<2 * QL * C::ES>(v0, p0 + col);
        copy_bytes<2 * QL * C::ES>(v1, p0 + C::ROWE + col);
      } else {
#pragma unroll
        for (int t = 0; t < 2 * QL; ++t) {
          const int c = (rm.col[t / 4] >> (8 * (t % 4))) & 0xff;
          const bool z = (rm.zero >> t) & 1;
          v0[t] = z ? StoreT<ST>::from_v(VT(0)) : p0[c];
          v1[t] = z ? StoreT<ST>::from_v(VT(0)) : p0[C::ROWE + c];
        }
      }
#pragma unroll
      for (int j = 0; j < QL; ++j) {
        o.s[LL][j] = StoreT<ST>::to_v(v0[2 * j]);
        o.s[HL][j] = StoreT<ST>::to_v(v0[2 * j + 1]);
        o.s[LH][j] = StoreT<ST>::to_v(v1[2 * j]);
        o.s[HH][j] = StoreT<ST>::to_v(v1[2 * j + 1]);
      }
    } else {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        ST v[QL];
        const ST* pr = plane(s, p) + r * C::ROWE;
        if (!rm.on) {
          copy_bytes<QL * C::ES>(v, pr + col);
        } else {
          const int px = p & 1;
#pragma unroll
          for (int t = 0; t < QL; ++t) {
            const int c = (rm.col[px] >> (8 * t)) & 0xff;
            const bool z = (rm.zero >> (QL * px + t)) & 1;
            v[t] = z ? StoreT<ST>::from_v(VT(0)) : pr[c];
          }
        }
#pragma unroll
        for (int j = 0; j < QL; ++j) o.s[p][j] = StoreT<ST>::to_v(v[j]);
      }
    }
    return o;
  }

  __device__ __forceinline__ Remap remap_cols() const {
    Remap rm{false, {0u, 0u}, 0u};
    if constexpr (C::REALIGN) {
      // a realigned strip whose odd planes sit at other box columns than the
      // even ones: every lane reads its elements one by one (columns clamped
      // into the row; the clamped ones are halo elements no stored value
      // reads); border lanes are remapped below as usual
      if (box && be(1) != be(0)) {
        rm.on = true;
#pragma unroll
        for (int px = 0; px < 2; ++px)
#pragma unroll
          for (int t = 0; t < QL; ++t)
            rm.col[px] |= (uint32_t)min(max(mfirst - be(px) + QL * lane + t, 0), C::ROWE - 1) << (8 * t);
      }
    }
    if (!box || cols_inside()) return rm;
    if constexpr (C::LOAD == SAMPLES) {
      const int xs = 2 * mfirst, xal = align_down(xs, C::A), x0 = xs + 2 * QL * lane;
      rm.on = x0 < 0 || x0 + 2 * QL > a.W;
      if (!rm.on) return rm;
#pragma unroll
      for (int t = 0; t < 2 * QL; ++t) {
        const int x = x0 + t;
        uint32_t c = 0;
        if (x >= -2 * C::HQ && x <= a.W + 2 * C::HQ) c = (uint32_t)min(max(mirror(x, a.W) - xal, 0), C::ROWE - 1);
        else rm.zero |= 1u << t;
        rm.col[t / 4] |= c << (8 * (t % 4));
      }
    } else {
      const int m = mfirst + QL * lane;
      if (m >= 0 && m + QL <= a.fw) return rm;
      rm.on = true;
      rm.col[0] = rm.col[1] = 0u;
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        const int pw = px ? a.fw : a.cw;
#pragma unroll
        for (int t = 0; t < QL; ++t) {
          const int mm = m + t;
          uint32_t c = 0;
          if (mm >= -C::HQ && mm <= pw + C::HQ) {
            const int sm_ = (mm >= 0 && mm < pw) ? mm : (mirror(2 * mm + px, a.W) >> 1);
            c = (uint32_t)min(max(sm_ - be(px), 0), C::ROWE - 1);
          } else {
            rm.zero |= 1u << (QL * px + t);
          }
          rm.col[px] |= c << (8 * t);
        }
      }
    }
    return rm;
  }

  // Per-lane output bases, computed once per strip.
  struct Out {
    ST* base[4];
    long long pitch[4];
    int rows[4];
    bool vec[4];  // the lane's elements of this plane are stored as one vector
    bool lane_ok;
  };

  __device__ __forceinline__ Out out_bases() const {
    Out o;
    const int m = mfirst + QL * lane;
    o.lane_ok = m >= m0 && m < m0 + C::UQ;
    if constexpr (C::STORE == SUBBANDS) {
      constexpr int VB = QL * C::ES;  // bytes of the lane's row segment
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int pw = (p & 1) ? a.fw : a.cw;
        o.rows[p] = (p >> 1) ? a.fh : a.ch;
        o.base[p] = static_cast<ST*>(a.dst[p]) + m;
        o.pitch[p] = a.dst_pitch[p];
        o.vec[p] = m + QL <= pw && ((reinterpret_cast<uintptr_t>(o.base[p]) & (VB - 1)) == 0) &&
                   ((a.dst_pitch[p] * C::ES) & (VB - 1)) == 0;
      }
    } else {
      constexpr int VB = 2 * QL * C::ES;
      const int gx = 2 * m;
      o.base[0] = static_cast<ST*>(a.dst[0]) + gx;
      o.pitch[0] = a.dst_pitch[0];
      o.rows[0] = a.H;
      o.vec[0] = gx + 2 * QL <= a.W && ((reinterpret_cast<uintptr_t>(o.base[0]) & (VB - 1)) == 0) &&
                 ((a.dst_pitch[0] * C::ES) & (VB - 1)) == 0;
    }
    return o;
  }

  __device__ __forceinline__ void store_row(const Out& o, const Row<VT, QL>& r, int q) const {
    if (!o.lane_ok) return;  // halo lane
    const int m = mfirst + QL * lane;
    if constexpr (C::STORE == SUBBANDS) {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        if (q >= o.rows[p]) continue;
        ST* rowp = o.base[p] + (long long)q * o.pitch[p];
        ST v[QL];
#pragma unroll
        for (int j = 0; j < QL; ++j) v[j] = StoreT<ST>::from_v(r.s[p][j]);
        const int pw = (p & 1) ? a.fw : a.cw;
        if (o.vec[p]) {
          copy_bytes<QL * C::ES>(rowp, v);
        } else if (C::ES == 4 && m + QL <= pw) {
          store_run<QL>(rowp, v);
        } else {
#pragma unroll
          for (int j = 0; j < QL; ++j)
            if (m + j < pw) rowp[j] = v[j];
        }
      }
    } else {
      const int gx = 2 * m;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int gy = 2 * q + rr;
        if (gy >= o.rows[0]) continue;
        ST* rowp = o.base[0] + (long long)gy * o.pitch[0];
        const int sl = rr ? LH : LL, sh = rr ? HH : HL;
        ST v[2 * QL];
#pragma unroll
        for (int j = 0; j < QL; ++j) {
          v[2 * j] = StoreT<ST>::from_v(r.s[sl][j]);
          v[2 * j + 1] = StoreT<ST>::from_v(r.s[sh][j]);
        }
        if (o.vec[0]) {
          copy_bytes<2 * QL * C::ES>(rowp, v);
        } else if (C::ES == 4 && gx + 2 * QL <= a.W) {
          store_run<2 * QL>(rowp, v);
        } else {
#pragma unroll
          for (int t = 0; t < 2 * QL; ++t)
            if (gx + t < a.W) rowp[t] = v[t];
        }
      }
    }
  }
};

// Strip row of the j-th row of strips in dispatch order, when one resident
// wave holds P rows of strips.  The rows are dealt to the W = ceil(nrs / P)
// waves round-robin (wave w takes rows w, w + W, w + 2W, ...), so that
// vertically adjacent strips run in consecutive waves: the halo rows a strip
// reads first are the rows its upper neighbour read last, just before, and
// they come from L2.  (Run in the same wave, the two strips read them a
// strip's duration apart, with a wave's worth of traffic in between.)  A
// bijection on [0, nrs): wave w holds ceil((nrs - w) / W) rows.
__device__ __forceinline__ int dealt_row(int j, int nrs, int P) {
  if (P <= 0 || P >= nrs) return j;
  const int W = (nrs + P - 1) / P;
  const int q = nrs / W, r = nrs % W;
  int w, k;
  if (j < r * (q + 1)) {
    w = j / (q + 1);
    k = j - w * (q + 1);
  } else {
    const int jj = j - r * (q + 1);
    w = r + jj / q;
    k = jj - (w - r) * q;
  }
  return k * W + w;
}

// Strip order: the two border columns first (their halo handling makes
// them the longest), then the interior, one row of strips after another in
// the dealt row order.  Blocks are dispatched in this order, so the long
// strips start in the first wave.
__device__ __forceinline__ void strip_coords(int s, int ncs, int nrs, int wave_rows, int& cs, int& rs) {
  if (ncs <= 2) {
    cs = s % ncs;
    rs = dealt_row(s / ncs, nrs, wave_rows);
  } else if (s < 2 * nrs) {
    cs = (s & 1) ? ncs - 1 : 0;
    rs = s >> 1;
  } else {
    const int i = s - 2 * nrs;
    cs = 1 + i % (ncs - 2);
    rs = dealt_row(i / (ncs - 2), nrs, wave_rows);
  }
}

// Waits, bounded, until the completion counters dep[lo..hi] all reach
// `need`.  Lane i watches rows lo + i, lo + i + 32, ...; each lane acquires
// the writes of the strips it watched, and the warp barrier at the end
// passes them on to the lanes that read the data.  Returns false if the
// wait ran out (after `limit` polls, each followed by a short nanosleep).
__device__ __forceinline__ int load_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool wait_rows(const int* dep, int lo, int hi, int need, uint32_t limit) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int r0 = lo; r0 <= hi && ok; r0 += 32) {
    const int r = r0 + lane;
    bool mine = r > hi;
    for (uint32_t spins = 0;; ++spins) {
      if (!mine) mine = load_acquire(dep + r) >= need;
      if (__all_sync(kFull, mine)) break;
      if (spins >= limit) {
        ok = false;
        break;
      }
      __nanosleep(64);
    }
  }
  __syncwarp();
  // the awaited strips were written through the generic proxy; the warp
  // reads them by TMA (async proxy) as well
  ptx::fence_proxy_async_global();
  return ok;
}

// Failure injection: waits, bounded by `limit` polls, until *flag is
// nonzero.  The flag passed is one that nothing sets, so the wait runs out;
// it is taken before the strip issues any load, so no copy is in flight
// when the warp leaves.
__device__ __forceinline__ bool wait_flag(const int* flag, uint32_t limit) {
  for (uint32_t spins = 0; spins < limit; ++spins) {
    if (__any_sync(kFull, load_acquire(flag) != 0)) return true;
    __nanosleep(64);
  }
  return false;
}

// Publishes a finished strip of row rs: after the warp barrier (which
// orders every lane's stores before lane 0's next operation), lane 0 adds
// one to the row's counter with release semantics.  A reduction returns
// nothing, so the warp does not wait for it.
__device__ __forceinline__ void publish_row(int* done, int rs) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0)
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(done + rs) : "memory");
}

// Lift strip (cs, rs): column strip cs, quad rows [rs*T, rs*T + T).  `ring`
// is the warp's shared-memory ring (nstages stages; the stage size the
// caller reserved is passed as `stage_stride`), `bars` its barriers
// (initialised for 32 arrivals), and `chunk_ctr` the warp's running count of
// ring fills: stage and phase of a fill follow from it, so a warp can lift
// several strips in a row.  Returns false if a bounded wait ran out (the
// launch's status word is set).
template <class C>
__device__ __forceinline__ bool run_strip(const LevelArgs& a, const TmaMaps& maps, const Coefs& cf,
                                          const ConvTaps& ct, int cs, int rs, unsigned char* ring,
                                          int stage_stride, uint64_t* bars, uint32_t& chunk_ctr) {
  const int lane = threadIdx.x & 31;
  const int q0 = rs * a.T;
  const int rows_out = min(a.T, a.ch - q0);
  if (rows_out <= 0) return true;
  const int NS = a.nstages;
  using Tot = typename C::Tot;
  Strip<C> sp{a, maps, lane, cs * C::UQ, cs * C::UQ - C::HQ, q0 - Tot::UP, ring, bars};
  sp.stride = stage_stride;
  // the box layout with the planes' realignment, if the strip can take it;
  // otherwise lane copies, which read every plane from its own start
  sp.set_box_cols(true);
  const bool boxed = sp.boxed();
  if (!boxed) sp.set_box_cols(false);
  sp.box = boxed;

  // rows streamed: the strip plus its halo, padded to whole chunks (the
  // extra rows are mirrored image rows, lifted but never stored)
  const int nrows = rows_out + Tot::UP + Tot::DOWN;
  const int nchunks = (nrows + C::CH - 1) / C::CH;
  const int q_end = q0 + rows_out;
  const uint32_t g0 = chunk_ctr;
  for (int c = 0; c < NS - 1 && c < nchunks; ++c) sp.fill(c, (g0 + c) % NS);
  // stage and phase of the chunk being consumed, advanced by one per chunk
  // (no division by the run-time ring depth inside the loop); the chunk
  // filled while it is consumed goes to the stage consumed just before
  int s = (int)(g0 % (uint32_t)NS);
  uint32_t phase = (g0 / (uint32_t)NS) & 1u;

  const typename Strip<C>::Out ob = sp.out_bases();
  const typename Strip<C>::Remap remap = sp.remap_cols();
  const auto coefs = CoefSource<typename C::CSRC>::make(cf);
  Pipe<typename C::VT, C::QL, typename C::PROG> pipe;
  pipe.reset();
  for (int c = 0; c < nchunks; ++c) {
    const int cn = c + NS - 1;
    if (cn < nchunks) {
      __syncwarp();
      sp.fill(cn, s == 0 ? NS - 1 : s - 1);
    }
    bool ok = ptx::mbar_wait_bounded(&bars[s], phase, a.probes);
    ok = __all_sync(kFull, ok);
    if (!ok) {
      if (lane == 0) atomicOr(a.status, 1);
      // let copies already in flight land before the warp leaves (with the
      // default limit, whatever limit the launch set for the wait above)
      ptx::cp_async_wait_all();
      for (int k = c; k < nchunks && k < c + NS; ++k)
        ptx::mbar_wait_bounded(&bars[(g0 + k) % NS], ((g0 + k) / NS) & 1, kDefaultRingProbes);
      chunk_ctr = g0 + nchunks;
      return false;
    }
    const int qc = sp.yfirst + c * C::CH - Tot::DOWN;
    // two rows per unrolled body: the stage windows rotate with period two,
    // and the loop body stays small enough for the instruction cache
#pragma unroll 2
    for (int r = 0; r < C::CH; ++r) {
      const Row<typename C::VT, C::QL> in = sp.load_row(s, r, remap);
      const Row<typename C::VT, C::QL> out = pipe.push(in, coefs, ct);
      const int q = qc + r;
      if (q >= q0 && q < q_end) sp.store_row(ob, out, q);
    }
    if (++s == NS) {
      s = 0;
      phase ^= 1u;
    }
  }
  chunk_ctr = g0 + nchunks;
  return true;
}

template <class C>
__global__ void __launch_bounds__(kWarpsPerCta * 32, C::MIN_WARPS / kWarpsPerCta)
    level_kernel(const __grid_constant__ TmaMaps maps, const __grid_constant__ LevelArgs a,
                 const __grid_constant__ Coefs cf, const __grid_constant__ ConvTaps ct) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int strip = blockIdx.x * kWarpsPerCta + warp;
  if (strip >= a.ncs * a.nrs) return;  // whole warp: no CTA-wide synchronisation is used
  const int NS = a.nstages;
  unsigned char* ring = smem_raw + (size_t)warp * NS * C::STAGE_BYTES;
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem_raw + (size_t)kWarpsPerCta * NS * C::STAGE_BYTES) + warp * kMaxStages;
  ptx::launch_dependents();
  if (lane == 0) {
    for (int s = 0; s < NS; ++s) ptx::mbar_init(&bars[s], 32);
    ptx::fence_barrier_init();
    constexpr int nmaps = C::LOAD == SUBBANDS ? 4 : 1;
#pragma unroll
    for (int p = 0; p < nmaps; ++p)
      if ((a.src_tma >> p) & 1) ptx::prefetch_tensormap(&maps.m[p]);
  }
  __syncwarp();
  if (a.hold && strip == 0 && !wait_flag(a.hold, a.spins)) {
    if (lane == 0) atomicOr(a.status, 1);
    return;
  }
  int cs, rs;
  strip_coords(strip, a.ncs, a.nrs, a.wave_rows, cs, rs);
  // the previous level's kernel may still be running: every read and write
  // of level data comes after this point
  ptx::wait_prerequisites();
  uint32_t chunk_ctr = 0;
  run_strip<C>(a, maps, cf, ct, cs, rs, ring, C::STAGE_BYTES, bars, chunk_ctr);
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
    k.box_h = C::ROWS;
    k.smem_bytes = smem(nstages);
    k.fn = reinterpret_cast<const void*>(&level_kernel<C>);
    k.supported = true;
    k.realign = C::REALIGN;
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
    const long long strips = (long long)a.ncs * a.nrs;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((strips + kWarpsPerCta - 1) / kWarpsPerCta));
    cfg.blockDim = dim3(kWarpsPerCta * 32);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    // programmatic dependent launch: this grid's blocks may start while the
    // previous kernel in the stream finishes (they wait before reading)
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, level_kernel<C>, m, a, cf, ct);
  }
};

}  // namespace dev
}  // namespace dwt
