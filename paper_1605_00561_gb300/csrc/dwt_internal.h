// Internal interface between the host API (dwt_api.cpp) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dwt {

// Storage types (match dwt_dtype).
enum DType : int { F32 = 0, F16S = 1, I32 = 2 };
// Wavelets (match dwt_wavelet).
enum Wavelet : int { W53 = 0, W97 = 1, WDD = 2 };
// Schemes (match dwt_scheme).
enum Scheme : int {
  AUTO = 0, ROWCOL, SWELDENS, IWAHASHI, IWAHASHI_S, EXPLOSIVE, EXPLOSIVE_S,
  MONOLITHIC, MONOLITHIC_S, POLYPHASE, POLYPHASE_S, CONVOLUTION, NUM_SCHEMES
};

// What a launch reads and writes.
//  SAMPLES:  one interleaved sample plane (image, or a row-column intermediate)
//  SUBBANDS: four planes LL, HL, LH, HH (Mallat quadrants / scratch LL)
enum Layout : int { SAMPLES = 0, SUBBANDS = 1 };

// Pass kinds of a launch.
enum Pass : int {
  PASS_FUSED = 0,   // one launch per level: the whole 2-D scheme
  PASS_VERT = 1,    // row-column baseline: vertical 1-D transform
  PASS_HORZ = 2     // row-column baseline: horizontal 1-D transform
};

// CDF 9/7 lifting constants and the DC gain K of the unscaled low-pass; the
// paper defers them to its reference [Daubechies1998] (Sec. 5).  Host code
// (coefficient tables) and device code (compile-time coefficients) share
// these literals.
constexpr double kAlpha = -1.586134342059924;
constexpr double kBeta = -0.052980118572961;
constexpr double kGamma = 0.882911075530934;
constexpr double kDelta = 0.443506852043971;
constexpr double kK97 = 1.230174104914001;

// Default limits of the kernels' bounded waits: probes of a ring stage's
// mbarrier (each probe may suspend the thread briefly) and polls of a row
// counter or flag (each followed by a short nanosleep).  Both run to
// seconds at most; dwt_set_wait_limits changes them for later launches.
constexpr uint32_t kDefaultRingProbes = 1u << 24;
constexpr uint32_t kDefaultDepSpins = 1u << 22;

constexpr int kWarpsPerCta = 1;  // independent warps (one strip each) per CTA
constexpr int kMaxStages = 4;    // ring depth per warp
constexpr int kDefaultStages = 2;
constexpr int kDefaultStripRows = 10;

// Lifting coefficients per predict/update pair and axis.  A coefficient of
// an axis whose length is 1 is zero, which makes that axis' lifting the
// identity (a length-1 line is left untouched).
struct Coefs {
  float ph1[2], ph3[2], uh1[2], uh3[2];  // horizontal: taps at distance 1 and 3 (samples)
  float pv1[2], pv3[2], uv1[2], uv3[2];  // vertical
  float scale[4];                        // LL, HL, LH, HH (forward); reciprocals for the inverse
  int v_on, h_on;                        // integer path: axis has length > 1
};

// 2-D taps of the Convolution scheme, indexed
// [out row type][out col type][in row type][in col type][dy + 3][dx + 3]
// (quad offsets -3..3: DD 13/7 reaches 3 quads, the CDF wavelets 2).
// Forward: out types are (L, H) bands, in types (even, odd) polyphase
// components; inverse: the other way round.  Scaling is folded in.
constexpr int kConvReach = 3;
struct ConvTaps {
  float t[2][2][2][2][2 * kConvReach + 1][2 * kConvReach + 1];
};

// Geometry and buffers of one launch (one level, one pass).
struct LevelArgs {
  // Dimensions of the level's sample plane (forward input / inverse output).
  int W, H;
  int cw, ch;  // ceil(W/2), ceil(H/2): quads / LL size
  int fw, fh;  // floor(W/2), floor(H/2)
  // Strips: column strip cs covers useful quads [cs*UQ, cs*UQ+UQ); row
  // strip rs covers quad rows [rs*T, rs*T+T); strip index rs*ncs + cs.
  int ncs, nrs, T;
  int wave_rows;  // strip rows of one resident wave (dispatch order, see strip_coords); 0: row by row
  int nstages;    // ring depth used (<= kMaxStages)
  // Sources and destinations (element pitches).
  const void* src[4];
  long long src_pitch[4];
  void* dst[4];
  long long dst_pitch[4];
  int src_tma;   // bit p: the tensor map of source plane p is valid (TMA loads it)
  // Subband sources: elements between plane p's first element and the
  // 16-byte-aligned column before it where its tensor map starts (0: the
  // plane starts aligned, or is not loaded realigned).  Only HL and HH
  // (planes 1 and 3, the same offset) are realigned.
  int src_off[4];
  int* status;   // device error word (bit 0: a bounded wait ran out)
  uint32_t probes;  // limit of a ring-stage wait (mbarrier probes)
  uint32_t spins;   // limit of a row-counter or flag wait (polls)
  // Failure injection (tests of the error paths): when set, the launch's
  // first strip waits, bounded by `spins`, for this word to become nonzero;
  // nothing sets it, so the wait runs out and the status word is raised.
  const int* hold;
};

struct TmaMaps {
  CUtensorMap m[4];
};

// Properties a host needs to lay out a launch: horizontal halo quads per
// side (HQ), useful quads per warp (UQ), dynamic shared memory per CTA, and
// the loader/storer layouts.
struct KernelInfo {
  int hq;
  int uq;
  int up, down;  // vertical halo (quad rows) above / below
  Layout load, store;
  int box_w, box_h;  // TMA box of one source plane (elements x rows)
  size_t smem_bytes;
  const void* fn;  // kernel entry (for occupancy queries)
  bool supported;
  bool realign;  // loads subband planes from the aligned column before a misaligned start
};

struct LaunchKey {
  int wavelet, dtype, scheme, pass, inverse;
  // the level may use compile-time coefficients: fused pass, JPEG 2000
  // normalisation, both axes longer than one sample
  int static_coefs;
};

struct LaunchCall {
  const LevelArgs* a;
  const TmaMaps* maps;
  const Coefs* cf;
  const ConvTaps* ct;
  cudaStream_t stream;
};

// ---- fused tail: several small levels of one image in one launch ----------
// (tile_kernel.cuh).  Levels run in 2-D tiles in shared memory, with a grid
// barrier between levels.
constexpr int kMaxTailLevels = 12;
constexpr int kTileThreads = 256;

// One level of a fused tail: geometry and planes as for the streaming
// kernels (the strip fields are unused), its coefficients, and its tiles.
struct TileLevel {
  LevelArgs a;
  Coefs cf;
  int ntx, nty;
};

struct TailParams {
  TileLevel lv[kMaxTailLevels];  // in processing order
  int nlevels;
  unsigned* barrier;  // grid barrier counter (device memory, any value)
};

// Stored interior of a tile (quads), shared memory and entry of a kernel.
struct TailInfo {
  int inner_rows, inner_cols;
  size_t smem_bytes;
  const void* fn;
};

struct TailCall {
  const TailParams* p;
  int blocks;
  cudaStream_t stream;
};

// Returns true when the group has a tail kernel for `k`; then fills *info
// and/or launches.
using TailFn = bool (*)(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err);

bool tail_sweldens(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);
bool tail_iwahashi(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);
bool tail_iwahashi_s(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);
bool tail_explosive(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);
bool tail_explosive_s(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);
bool tail_monolithic(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);
bool tail_monolithic_s(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);
bool tail_polyphase(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);
bool tail_polyphase_s(const LaunchKey&, TailInfo*, const TailCall*, cudaError_t*);

// Returns true when the group handles `k`; then fills *info and/or launches.
using GroupFn = bool (*)(const LaunchKey& k, int nstages, KernelInfo* info, const LaunchCall* call,
                         cudaError_t* err);

bool group_sweldens(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_iwahashi(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_iwahashi_s(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_explosive(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_explosive_s(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_monolithic(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_monolithic_s(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_polyphase(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_polyphase_s(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_convolution(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);
bool group_rowcol(const LaunchKey&, int, KernelInfo*, const LaunchCall*, cudaError_t*);

}  // namespace dwt
