// Instantiation helpers shared by the kernel translation units.  Each unit
// owns a group of schemes and answers "kernel info" and "launch" requests
// for the (wavelet, dtype, direction) combinations of its group.
#pragma once

#include <type_traits>

#include "level_kernel.cuh"
#include "tile_kernel.cuh"

namespace dwt {

namespace dev {

template <class C>
inline bool run(int nstages, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  using I = Instance<C>;
  if (info) *info = I::info(nstages);
  if (call) *err = I::launch(*call->a, *call->maps, *call->cf, *call->ct, call->stream);
  return true;
}

// Quadruples per lane: four (128-bit vectors, fewer instructions and
// shuffles per sample) except for Convolution, whose windows at four exceed
// the register file, and the unstarred Polyphase with CDF 5/3, which the
// compiler does not build at four (it fails within 128 registers).  A ring
// stage holds the same bytes either way.
template <int SCHEME, int WL>
constexpr int kQuadsPerLane = (SCHEME == CONVOLUTION || (SCHEME == POLYPHASE && WL == W53)) ? 2 : 4;

// Resident warps per SM the register budget is cut for: 16 (128 registers)
// in general; 12 (168 registers) for the three-step schemes with two pairs
// or degree-3 steps and for the unstarred Polyphase with two pairs, which
// need them at four quadruples per lane (DD 13/7 runs 1.3-2.2x faster at 12
// than squeezed into 128 registers; Polyphase 9/7 at four quadruples and 12
// warps is 8-16 % faster at 8192^2 than at two and 16); 8 for Convolution
// and for Polyphase(*) with DD 13/7, whose merged steps are 7 x 7 stencils.
template <int SCHEME, int WL>
constexpr int kMinWarps =
    SCHEME == CONVOLUTION ? 8
    : ((SCHEME == POLYPHASE || SCHEME == POLYPHASE_S) && WL == WDD) ? 8
    : (SCHEME == POLYPHASE && WL == W97) ? 12
    : ((WL == W97 || WL == WDD) &&
       (SCHEME == IWAHASHI || SCHEME == IWAHASHI_S || SCHEME == EXPLOSIVE || SCHEME == EXPLOSIVE_S))
        ? 12
        : 16;

// Every scheme takes the degree-3 DD 13/7 pair (Polyphase and Convolution
// with the degree-6 products of P and U).
template <int SCHEME>
constexpr bool kHasDegree3 = true;

// Convolution with compile-time taps needs no tap table in registers
// (112-127 registers against 255 with the runtime table): 16 warps per SM.
template <int SCHEME, int WL, bool STATIC>
constexpr int kMinWarpsCfg = (SCHEME == CONVOLUTION && STATIC) ? 16 : kMinWarps<SCHEME, WL>;

// STATIC: coefficients folded in at compile time (StCoefs), for levels with
// JPEG 2000 normalisation and both axes longer than one sample.
template <int SCHEME, int WL, typename ST, bool INV, bool STATIC = false>
using FusedCfg = Cfg<ST, float, typename FusedProgram<SCHEME, WL, INV>::type, INV ? SUBBANDS : SAMPLES,
                     INV ? SAMPLES : SUBBANDS, kQuadsPerLane<SCHEME, WL>, 8 / kQuadsPerLane<SCHEME, WL>,
                     kMinWarpsCfg<SCHEME, WL, STATIC>, std::conditional_t<STATIC, StCoefs<WL, INV>, RtTag>>;

template <int SCHEME, int WL, typename ST, bool STATIC>
inline bool fused_dir(bool inv, int ns, KernelInfo* info, const LaunchCall* call, cudaError_t* err) {
  return inv ? run<FusedCfg<SCHEME, WL, ST, true, STATIC>>(ns, info, call, err)
             : run<FusedCfg<SCHEME, WL, ST, false, STATIC>>(ns, info, call, err);
}

// The float combinations of one fused scheme; schemes listed with
// WITH_STATIC also carry compile-time-coefficient kernels, taken when the
// launch allows them.
template <int SCHEME, bool WITH_STATIC = false>
inline bool fused_float(const LaunchKey& k, int ns, KernelInfo* info, const LaunchCall* call,
                        cudaError_t* err) {
  if (k.pass != PASS_FUSED || k.scheme != SCHEME) return false;
  const bool inv = k.inverse != 0;
  if constexpr (WITH_STATIC) {
    if (k.static_coefs) {
      if (k.wavelet == W53 && k.dtype == F32) return fused_dir<SCHEME, W53, float, true>(inv, ns, info, call, err);
      if (k.wavelet == W97 && k.dtype == F32) return fused_dir<SCHEME, W97, float, true>(inv, ns, info, call, err);
      if (k.wavelet == W53 && k.dtype == F16S) return fused_dir<SCHEME, W53, __half, true>(inv, ns, info, call, err);
      if (k.wavelet == W97 && k.dtype == F16S) return fused_dir<SCHEME, W97, __half, true>(inv, ns, info, call, err);
    }
  }
  if (k.wavelet == W53 && k.dtype == F32) return fused_dir<SCHEME, W53, float, false>(inv, ns, info, call, err);
  if (k.wavelet == W97 && k.dtype == F32) return fused_dir<SCHEME, W97, float, false>(inv, ns, info, call, err);
  if constexpr (kHasDegree3<SCHEME>) {
    if (k.wavelet == WDD && k.dtype == F32) {
      if (WITH_STATIC && k.static_coefs) return fused_dir<SCHEME, WDD, float, true>(inv, ns, info, call, err);
      return fused_dir<SCHEME, WDD, float, false>(inv, ns, info, call, err);
    }
  }
  if (k.wavelet == W53 && k.dtype == F16S) return fused_dir<SCHEME, W53, __half, false>(inv, ns, info, call, err);
  if (k.wavelet == W97 && k.dtype == F16S) return fused_dir<SCHEME, W97, __half, false>(inv, ns, info, call, err);
  return false;
}

// ---- fused-tail kernels (tile_kernel.cuh) ----------------------------------
template <class C>
inline bool run_tail(TailInfo* info, const TailCall* call, cudaError_t* err) {
  using I = TailInstance<C>;
  if (info) {
    I::geom(&info->inner_rows, &info->inner_cols);
    info->smem_bytes = I::smem();
    info->fn = I::fn();
  }
  if (call) *err = I::launch(*call->p, call->blocks, call->stream);
  return true;
}

template <int SCHEME, int WL, typename ST, bool INV, bool STATIC>
using TailFusedCfg = TailCfg<ST, float, typename FusedProgram<SCHEME, WL, INV>::type, INV ? SUBBANDS : SAMPLES,
                             INV ? SAMPLES : SUBBANDS, std::conditional_t<STATIC, StCoefs<WL, INV>, RtTag>,
                             (SCHEME == POLYPHASE || SCHEME == POLYPHASE_S) ? 2 : 4>;

template <int SCHEME, int WL, typename ST, bool STATIC>
inline bool tail_dir(bool inv, TailInfo* info, const TailCall* call, cudaError_t* err) {
  return inv ? run_tail<TailFusedCfg<SCHEME, WL, ST, true, STATIC>>(info, call, err)
             : run_tail<TailFusedCfg<SCHEME, WL, ST, false, STATIC>>(info, call, err);
}

// The float tail kernels of one scheme: CDF 5/3 and 9/7 in float32 and
// float16 storage, DD 13/7 in float32 where the scheme takes it; static
// coefficients for JPEG 2000 normalisation (a tail level has both sides >= 2).
template <int SCHEME>
inline bool tail_float(const LaunchKey& k, TailInfo* info, const TailCall* call, cudaError_t* err) {
  if (k.pass != PASS_FUSED || k.scheme != SCHEME) return false;
  const bool inv = k.inverse != 0;
  const bool st = k.static_coefs != 0;
  if (k.wavelet == W53 && k.dtype == F32)
    return st ? tail_dir<SCHEME, W53, float, true>(inv, info, call, err)
              : tail_dir<SCHEME, W53, float, false>(inv, info, call, err);
  if (k.wavelet == W97 && k.dtype == F32)
    return st ? tail_dir<SCHEME, W97, float, true>(inv, info, call, err)
              : tail_dir<SCHEME, W97, float, false>(inv, info, call, err);
  if (k.wavelet == W53 && k.dtype == F16S)
    return st ? tail_dir<SCHEME, W53, __half, true>(inv, info, call, err)
              : tail_dir<SCHEME, W53, __half, false>(inv, info, call, err);
  if (k.wavelet == W97 && k.dtype == F16S)
    return st ? tail_dir<SCHEME, W97, __half, true>(inv, info, call, err)
              : tail_dir<SCHEME, W97, __half, false>(inv, info, call, err);
  if constexpr (kHasDegree3<SCHEME>) {
    if (k.wavelet == WDD && k.dtype == F32)
      return st ? tail_dir<SCHEME, WDD, float, true>(inv, info, call, err)
                : tail_dir<SCHEME, WDD, float, false>(inv, info, call, err);
  }
  return false;
}

}  // namespace dev
}  // namespace dwt
