/*
 * libdwt -- multi-level 2-D discrete wavelet transform on one GB300 GPU.
 *
 * The transform is the one stated in the paper (Barina, Kula, Zemcik,
 * "Parallel Wavelet Schemes for Images"): an image is split into its four
 * polyphase components (LL, HL, LH, HH; Sec. 2.3) and mapped by a chain of
 * 2-D lifting steps (Sec. 2.4-4) built from the 1-D predict/update pairs of
 * the wavelet (Sec. 2.2, Sec. 5).  Every scheme (separable, single-loop,
 * Iwahashi, Explosive, Monolithic, Polyphase, their starred variants and
 * Convolution) computes the same coefficients up to rounding (Sec. 7).  In
 * float32 the rounding differs by scheme: the unstarred Polyphase with
 * CDF 9/7 evaluates each merged step V = PU + 1 as one 2-D FIR and rounds
 * about twice as much as the lifting schemes (about 1e-3 against 3-7e-4
 * after one level on 8-bit samples, up to 2.2e-3 after six); DD 13/7, whose
 * coefficients are dyadic, stays at or below 4e-4 in every scheme.
 *
 * Conventions shared by every entry point:
 *   - Images are row-major 2-D planes with a row pitch in BYTES (a multiple
 *     of the element size, as are the plane addresses).  Device pointers
 *     must be CUDA device (or managed) memory; host pointers are rejected
 *     with DWT_EINVAL, never dereferenced on the GPU.
 *   - Speed: planes whose row pitch is a multiple of 16 bytes are loaded by
 *     the TMA engine, the HL and HH bands of odd widths included; rows of
 *     odd widths packed without padding cannot be, and are copied by the
 *     threads (for 5001 x 3333 float32, 1.3-1.4x slower; float16 inverse
 *     2.9x).  Padding rows to 128 bytes, as cudaMallocPitch does, avoids it.
 *   - Output layout (forward) / input layout (inverse): Mallat packing of a
 *     w x h plane.  At level k the level's input is W_k x H_k (W_0 = w,
 *     W_{k+1} = ceil(W_k / 2)); its LL band is ceil(W_k/2) x ceil(H_k/2) at
 *     the top-left, HL (horizontal high-pass) at the top-right, LH at the
 *     bottom-left and HH at the bottom-right; level k+1 recurses into LL.
 *   - Boundary: whole-sample symmetric extension; a dimension of length 1
 *     is left untouched.  Even samples are low-pass (JPEG 2000 origin).
 *   - Normalisation (default): JPEG 2000, i.e. low-pass DC gain 1 and
 *     high-pass Nyquist gain 2 (5/3 unscaled; 9/7 low x 1/K, high x K).
 *   - All calls that take a stream are asynchronous with respect to the
 *     host; errors detected on the host are returned as dwt_status and
 *     never abort or throw across the ABI.  Device-side failures (a bounded
 *     wait that ran out) are reported through dwt_plan_device_status() or a
 *     batch's status array.
 *   - The transform is out-of-place: input and output must not overlap.
 *   - A plan owns its scratch memory; one plan must not be in flight on two
 *     streams at once (use one plan per concurrent slot).
 *   - Once a plan has made one single-image call (which allocates its device
 *     memory), its dwt2_forward / dwt2_inverse calls can be captured into a
 *     CUDA graph by stream capture and replayed; the levels keep their
 *     programmatic-dependent-launch edges.  dwt_batch_submit cannot be
 *     captured (it waits on its upload ring).
 *
 * All functions are thread-safe for distinct plans.
 */
#ifndef LIBDWT_DWT_H
#define LIBDWT_DWT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* dwt_stream;

typedef struct dwt_plan_s* dwt_plan;

typedef enum {
  DWT_OK = 0,
  DWT_EINVAL = 1,       /* bad argument: size, level count, pitch, pointer, aliasing */
  DWT_ENOMEM = 2,       /* device or host allocation failed */
  DWT_EUNSUPPORTED = 3, /* valid but not provided (e.g. 9/7 with int32) */
  DWT_ECUDA = 4,        /* a CUDA runtime call failed */
  DWT_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
  DWT_EBUSY = 6         /* a resource is in use (reserved: no call of this version returns it) */
} dwt_status;

typedef enum {
  DWT_CDF53 = 0, /* P = -1/2 (1 + z^-1), U = 1/4 (1 + z) (Sec. 5)                  */
  DWT_CDF97 = 1, /* two pairs (alpha, beta), (gamma, delta) (Sec. 5)              */
  DWT_DD137 = 2  /* Deslauriers-Dubuc 13/7: degree-3 P and U (Sec. 5); float32, every
                    scheme                                                         */
} dwt_wavelet;

typedef enum {
  DWT_F32 = 0,  /* float32 storage and arithmetic                                    */
  DWT_F16S = 1, /* float16 storage, float32 arithmetic                              */
  DWT_I32 = 2   /* int32, reversible 5/3 with JPEG 2000 floor rounding, bit-exact    */
} dwt_dtype;

typedef enum {
  DWT_AUTO = 0,        /* chosen by the autotuner (persisted cache)                 */
  DWT_ROWCOL = 1,      /* separable, all columns then all rows through global memory */
  DWT_SWELDENS = 2,    /* separable single-loop: T^H_P | T^V_P | S^H_U | S^V_U (Sec. 2.5) */
  DWT_IWAHASHI = 3,    /* T^I_P | R^I_{P,U} | S^I_U (Sec. 2.6)                       */
  DWT_IWAHASHI_S = 4,  /* Iwahashi* (Sec. 4)                                        */
  DWT_EXPLOSIVE = 5,   /* T^E_P | R^E_{P,U} | S^E_U (Sec. 3.1)                      */
  DWT_EXPLOSIVE_S = 6, /* Explosive* (Sec. 4)                                       */
  DWT_MONOLITHIC = 7,  /* T_P | S_U (Sec. 3.2)                                      */
  DWT_MONOLITHIC_S = 8,/* Monolithic* (Sec. 4)                                      */
  DWT_POLYPHASE = 9,   /* N_{P,U} (Sec. 2.3)                                        */
  DWT_POLYPHASE_S = 10,/* Polyphase* (Sec. 4)                                       */
  DWT_CONVOLUTION = 11 /* four 2-D FIR filters with subsampling (Sec. 2.3)          */
} dwt_scheme;

typedef enum { DWT_NORM_JPEG2000 = 0, DWT_NORM_ZETA = 1 } dwt_norm;

/* Create a plan for a w x h image, `levels` levels (0 = plain copy), wavelet
 * and storage type.  Host-only: the plan's device memory (its status word
 * and one LL buffer per level after the first, each of ceil(W_k/2) x
 * ceil(H_k/2) elements with rows at a 128-byte pitch, about w*h/3 elements
 * in all) is allocated by its first single-image call, so plans used only
 * in batches never touch device memory and are cheap to create and
 * destroy.  Errors: DWT_EINVAL for w or h outside 1..2^28, levels < 0,
 * levels above the number of halvings until both dimensions are 1, or
 * out == NULL; DWT_EUNSUPPORTED for DWT_I32 with a wavelet other than 5/3
 * and for DWT_DD137 with a storage type other than DWT_F32; DWT_ENOMEM;
 * DWT_ECUDA. */
dwt_status dwt_plan_create(int w, int h, dwt_wavelet wavelet, int levels, dwt_dtype dtype,
                           dwt_plan* out);

/* Select the lifting scheme (default DWT_AUTO).  DWT_I32 supports
 * DWT_ROWCOL and DWT_SWELDENS, which compute the JPEG 2000 reversible 5/3
 * (its step order with floors is not shared by the non-separable schemes),
 * and DWT_IWAHASHI, which selects a different reversible transform: the
 * non-separable Iwahashi scheme (Sec. 2.6) with each 2-D step's whole
 * update rounded once, half up (T: HH += (d(LL) - 2 (h(LH) + v(HL)) + 2)
 * >> 2; R: HL += (v(HH) - 2 h(LL) + 2) >> 2, LH += (h(HH) - 2 v(LL) + 2) >>
 * 2; S: LL += (4 (h(HL) + v(LH)) - d(HH) + 8) >> 4; the inverse subtracts
 * the same updates in the order S, R, T), exactly reversible but not
 * JPEG 2000 compatible.  DWT_AUTO and the autotuner never switch an int32
 * plan to it, and batches refuse it (DWT_EUNSUPPORTED).  Other schemes give
 * DWT_EUNSUPPORTED for DWT_I32.  DWT_ROWCOL allocates a w x h intermediate
 * plane. */
dwt_status dwt_plan_set_scheme(dwt_plan plan, dwt_scheme scheme);

/* Tile shape of the kernels (autotuner knobs).  strip_rows: target number
 * of quadruple rows a warp streams (0 = the default of the scheme a call
 * runs: 10; 32 for Iwahashi, Iwahashi*, Explosive and Explosive* with CDF
 * 9/7 or DD 13/7 and for Polyphase; 32 (5/3) or 48 (9/7) for Convolution;
 * 24 for Monolithic, Monolithic* and Polyphase* with DD 13/7); a level too
 * small to fill the GPU once with such strips uses shorter ones, down to 2
 * rows.
 * stages: depth of each warp's shared-memory ring of row chunks, 1..4
 * (0 = default 2); deeper rings keep more loads in flight per warp,
 * shallower ones let more warps reside.  Errors: DWT_EINVAL for values out
 * of range. */
dwt_status dwt_plan_set_tile(dwt_plan plan, int strip_rows, int stages);

/* Fused tail of the pyramid (the paper's multi-level transform, Sec. 1,
 * run as in-tile levels, Sec. 6): levels whose input has at most
 * `max_pixels` samples, and both sides >= 2, run together in one launch in
 * which each level is cut into 2-D tiles held in shared memory (one
 * barrier per step that reads other quadruples) and the levels are
 * separated by a grid-wide barrier.  The larger levels keep one streaming
 * launch each.  -1 restores the default (512 x 512 samples), 0 turns the
 * fusion off.  Row-column and Convolution plans never fuse.  The result is
 * the same transform (float: within rounding of the per-level kernels;
 * int32: bit-identical).  Errors: DWT_EINVAL for values below -1. */
dwt_status dwt_plan_set_fusion(dwt_plan plan, long long max_pixels);
dwt_status dwt_plan_get_fusion(dwt_plan plan, long long* max_pixels);

/* The tile the plan's calls use: set by dwt_plan_set_tile, else the
 * autotuner's choice for this plan (from dwt_plan_autotune or the cache
 * file), else the defaults.  Either pointer may be NULL. */
dwt_status dwt_plan_get_tile(dwt_plan plan, int* strip_rows, int* stages);

/* The scheme a call will actually run (DWT_AUTO resolved). */
dwt_status dwt_plan_get_scheme(dwt_plan plan, dwt_scheme* scheme);

/* Float paths only: DWT_NORM_ZETA applies the paper's scaling step (low-pass
 * x zeta, high-pass x 1/zeta per axis; zeta = sqrt(2) for 5/3, Sec. 5). */
dwt_status dwt_plan_set_normalization(dwt_plan plan, dwt_norm norm);

/* Forward transform.  d_in: w x h samples, d_out: w x h Mallat-packed
 * coefficients, both device memory of the plan's dtype, pitches in bytes
 * (>= w * element size, multiple of the element size).  The input is
 * read-only.  Asynchronous on `stream`. */
dwt_status dwt2_forward(dwt_plan plan, const void* d_in, size_t in_pitch_bytes, void* d_out,
                        size_t out_pitch_bytes, dwt_stream stream);

/* Inverse transform: Mallat-packed coefficients in, samples out. */
dwt_status dwt2_inverse(dwt_plan plan, const void* d_coef, size_t coef_pitch_bytes, void* d_out,
                        size_t out_pitch_bytes, dwt_stream stream);

/* Forward transform for callers that cannot allocate device memory: a
 * real-time loop that must not call cudaMalloc (it can synchronise the
 * device and take unbounded time), an embedded or plug-in caller whose host
 * application owns every device allocation, or a memory-capped process
 * that has already spent its budget.  The paper has no counterpart; it is
 * the plan-free twin of dwt2_forward with the default scheme (Monolithic*
 * for float, the separable JPEG 2000 order for int32) and the tile a fresh
 * plan takes.  The caller passes the input and output as for dwt2_forward;
 * the LL scratch of the pyramid and a device status word live in one
 * file-scope device array of this library, 32 MiB plus 256 bytes, which
 * every GPU that loads the library holds until the process exits.  Images
 * whose LL scratch (row pitch ceil(w/2) elements rounded up to 128 bytes,
 * times ceil(h/2) + ceil(h/4) rows; none for levels <= 1) exceeds 32 MiB --
 * above about 4096 x 4096 float32 -- and sides outside 1..2^28 are rejected
 * with DWT_EINVAL.  The call makes no cudaMalloc, cudaFree or other
 * allocating call.  The first call on each device looks up the array's
 * device address (once per device, with that device current); make that
 * first call before any stream capture.  All calls share the array and it
 * keeps the previous call's contents: calls that overlap on the GPU (other
 * streams, or another thread) race on it, so serialise them.  A bounded
 * device wait that runs out raises the array's status word, which
 * dwt_noalloc_device_status reads. */
dwt_status dwt2_forward_noalloc(int w, int h, dwt_wavelet wavelet, int levels, dwt_dtype dtype,
                                const void* d_in, size_t in_pitch_bytes, void* d_out,
                                size_t out_pitch_bytes, dwt_stream stream);

/* Synchronise `stream` (the stream of the dwt2_forward_noalloc calls) and
 * report whether a bounded device wait of any such call on the current
 * device ran out since the previous query: DWT_ETIMEOUT (the output of the
 * call concerned is incomplete) or DWT_OK; the word is cleared.  Reads one
 * device word with a copy into host memory; allocates nothing.  DWT_ECUDA
 * if a CUDA call fails. */
dwt_status dwt_noalloc_device_status(dwt_stream stream);

/* Same transforms with HOST buffers: the call copies the input to device
 * staging owned by the plan, transforms it, and copies the result back into
 * h_out, all on `stream`.  h_in / h_out should be page-locked for the
 * copies to overlap; pageable memory works but synchronises.  The host
 * output is valid after the stream is synchronised. */
dwt_status dwt2_forward_host(dwt_plan plan, const void* h_in, size_t in_pitch_bytes, void* h_out,
                             size_t out_pitch_bytes, dwt_stream stream);
dwt_status dwt2_inverse_host(dwt_plan plan, const void* h_coef, size_t coef_pitch_bytes,
                             void* h_out, size_t out_pitch_bytes, dwt_stream stream);

/* Many transforms in one persistent launch.  Each request names a plan, its
 * device buffers and a direction; different sizes, level counts, wavelets,
 * dtypes and directions may be mixed.  Every level of every request runs
 * in one kernel: persistent one-warp blocks pull (image, level, strip) work
 * items from a global queue, ordered level-major across the requests, and
 * a level's strips wait, with a bounded spin, until the previous level of
 * the same image is done.  The scheme is fixed per dtype whatever the plan
 * selects: Monolithic* (Sec. 4) for float32 and float16 storage, the
 * separable JPEG 2000 lifting order for reversible int32 5/3; the plans'
 * normalisation applies, and their tile where the caller set one with
 * dwt_plan_set_tile (otherwise batches take 48-row strips and a 4-stage
 * ring, which suit the persistent kernel).  Each request's LL scratch and the
 * work list live in one work area that the call takes from a
 * library-owned stream-ordered memory pool and returns at the end of the
 * launch (the pool keeps its peak size for later batches), so batches
 * leave the plans' own scratch alone.  d_status (device memory, n ints,
 * may be NULL) is cleared and then receives DWT_ETIMEOUT for any request
 * whose wait or copy gave up.  A plan only supplies parameters here and
 * may appear in any number of requests; outputs may not overlap each other
 * or any input (DWT_EINVAL).  Batches take every plan: CDF 5/3 and 9/7 in
 * float32 and float16 storage, DD 13/7 in float32, reversible 5/3 in int32.
 * The call uploads its work list from a ring of page-locked buffers and may
 * wait for the upload of the batch that last used its slot, so it cannot be
 * captured into a CUDA graph. */
typedef struct {
  dwt_plan plan;
  const void* in;
  size_t in_pitch;
  void* out;
  size_t out_pitch;
  int inverse;
} dwt_request;

dwt_status dwt_batch_submit(const dwt_request* reqs, int n, dwt_stream stream, int* d_status);

/* Synchronise with the plan's last stream and report device-side failures
 * of its calls since the previous query (DWT_OK or DWT_ETIMEOUT). */
dwt_status dwt_plan_device_status(dwt_plan plan);

/* Limits of the kernels' bounded device waits, for launches made after the
 * call (process-wide): ring_probes bounds the wait for a row chunk's load
 * (mbarrier probes), dep_spins the wait of a batch strip for the rows it
 * reads and of an injected hold (polls a short sleep apart).  0 restores a
 * default (2^24 probes, 2^22 polls: seconds at most).  A wait that runs out
 * sets the status word that dwt_plan_device_status,
 * dwt_noalloc_device_status or a batch's status array report. */
dwt_status dwt_set_wait_limits(unsigned int ring_probes, unsigned int dep_spins);

/* Host-side failure injection, for tests of the error paths (nothing here
 * faults or hangs the GPU).  Each kind lets `skip` events pass and then
 * acts on the next `count`; DWT_INJECT_NONE clears every kind.
 *   DWT_INJECT_ENOMEM:    a device or page-locked allocation of the library
 *                         fails as cudaErrorMemoryAllocation would.
 *   DWT_INJECT_HOLD:      the first strip of a single-image level launch
 *                         (plan or no-alloc call) waits, bounded by
 *                         dep_spins, on a device flag that nothing sets, so
 *                         that the wait runs out and reports DWT_ETIMEOUT.
 *   DWT_INJECT_BATCH_DEP: in a batch, the second level of request 0 waits
 *                         for one more finished strip per row than its rows
 *                         have, a count nothing reaches; the request's
 *                         status slot receives DWT_ETIMEOUT.
 * Errors: DWT_EINVAL for an unknown kind or negative counts. */
typedef enum {
  DWT_INJECT_NONE = 0,
  DWT_INJECT_ENOMEM = 1,
  DWT_INJECT_HOLD = 2,
  DWT_INJECT_BATCH_DEP = 3
} dwt_injection;
dwt_status dwt_debug_inject(dwt_injection what, int skip, int count);

/* Per-kernel timing of a plan's calls, for measurement.  When enabled, each
 * launch is bracketed by CUDA events on the launching stream; reading the
 * profile synchronises on them.  Slot names are "<pass>/L<level>". */
typedef struct {
  char name[32];
  int launches;
  double total_ms;
  double algorithmic_bytes; /* bytes the launch must move, summed over launches */
} dwt_kernel_stat;

dwt_status dwt_plan_set_profiling(dwt_plan plan, int enable);
dwt_status dwt_plan_read_profile(dwt_plan plan, dwt_kernel_stat* stats, int capacity, int* count);

/* Run the autotuner for this plan now: time the forward transform of a
 * trial image (device memory allocated and freed here) for every scheme the
 * plan's wavelet and dtype support, each at its default strip height, then
 * the strip height (6..48 rows) and the ring depth (1..4 stages) for the
 * fastest scheme.  The choice applies to this plan (the scheme if it is
 * DWT_AUTO, the tile unless the caller set one) and is appended to the
 * cache file named by the environment variable DWT_AUTOTUNE_CACHE (if set),
 * which later plans of the same GPU, size, wavelet, dtype and level count
 * read.  The halo width follows from the scheme and wavelet. */
dwt_status dwt_plan_autotune(dwt_plan plan, dwt_stream stream);

/* Counts of the forward program a scheme runs, computed at compile time
 * from the same step lists as the kernels: multiply-accumulates per
 * quadruple (every tap of every term of every step; the scaling step and
 * the unit diagonal of a merged matrix are not operations), barriers (steps
 * that read other quadruples: the paper's memory barriers, Sec. 5, Table of
 * operations and barriers) and the shared-memory words per quadruple the
 * tile kernel of the fused tail publishes before those steps.  Row-column
 * reports its two passes together.  Host-only: needs no GPU.  Any pointer
 * may be NULL.  Errors: DWT_EINVAL for an unknown wavelet or scheme. */
dwt_status dwt_scheme_counts(dwt_wavelet wavelet, dwt_scheme scheme, int* macs, int* barriers,
                             int* smem_words);

dwt_status dwt_plan_destroy(dwt_plan plan);

const char* dwt_status_string(dwt_status status);

/* Library version "major.minor.patch". */
const char* dwt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBDWT_DWT_H */
