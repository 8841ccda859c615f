// Descriptors of the persistent batch kernel (batch.cu), shared with the
// host API.  Not part of the public ABI.
#pragma once

#include "dwt_internal.h"

namespace dwt {

// Kinds of level a batch can hold (scheme fixed per kind: Monolithic* for
// float, including DD 13/7 in float32, the separable JPEG 2000 order for
// reversible 5/3).  The float kinds
// fold their coefficients in at compile time (JPEG 2000 normalisation, both
// axes longer than one sample); the _RT kinds read them from the
// descriptor and serve every other level.
enum BatchKind : int {
  BK_97_F32_FWD = 0, BK_97_F32_INV, BK_53_F32_FWD, BK_53_F32_INV, BK_53_I32_FWD, BK_53_I32_INV,
  BK_97_F16_FWD, BK_97_F16_INV, BK_53_F16_FWD, BK_53_F16_INV,
  BK_97_F32_FWD_RT, BK_97_F32_INV_RT, BK_53_F32_FWD_RT, BK_53_F32_INV_RT,
  BK_97_F16_FWD_RT, BK_97_F16_INV_RT, BK_53_F16_FWD_RT, BK_53_F16_INV_RT,
  BK_DD_F32_FWD, BK_DD_F32_INV, BK_DD_F32_FWD_RT, BK_DD_F32_INV_RT, BK_COUNT
};

// The kind that serves a level without compile-time coefficients.
inline int batch_runtime_kind(int kind) {
  switch (kind) {
    case BK_97_F32_FWD: return BK_97_F32_FWD_RT;
    case BK_97_F32_INV: return BK_97_F32_INV_RT;
    case BK_53_F32_FWD: return BK_53_F32_FWD_RT;
    case BK_53_F32_INV: return BK_53_F32_INV_RT;
    case BK_97_F16_FWD: return BK_97_F16_FWD_RT;
    case BK_97_F16_INV: return BK_97_F16_INV_RT;
    case BK_53_F16_FWD: return BK_53_F16_FWD_RT;
    case BK_53_F16_INV: return BK_53_F16_INV_RT;
    case BK_DD_F32_FWD: return BK_DD_F32_FWD_RT;
    case BK_DD_F32_INV: return BK_DD_F32_INV_RT;
    default: return kind;  // integer kinds take no float coefficients
  }
}

// One (request, level): everything a strip of it needs.  The tensor maps
// come first; their own alignment (that of CUtensorMap, at least the 64
// bytes TMA requires) aligns every element of an array of these.
// Strips are numbered row-major: strip = rs * a.ncs + cs.
struct BatchLevel {
  TmaMaps maps;
  LevelArgs a;
  Coefs cf;
  int kind;
  int request;
  int row_base;      // index of this level's strip row 0 in the row arrays
  int dep_row_base;  // the same for the level whose output it reads, or -1
  int dep_ncs;       // column strips per row of that level: the count a row of it waits for
};

static_assert(alignof(BatchLevel) % 64 == 0, "tensor maps in a BatchLevel array must stay 64-byte aligned");

struct BatchItem {
  int level;
  int strip;
};

struct BatchParams {
  const BatchLevel* levels;
  const BatchItem* items;
  // per strip row of every level: the first and last strip rows of the
  // level it reads that must be complete before the row may start
  const int2* row_deps;
  int nitems;
  int* head;        // next item to take
  int* row_done;    // per strip row of every level: column strips finished
  int* req_status;  // per request
};

bool batch_kind_info(int kind, KernelInfo* k);
size_t batch_smem_bytes();
const void* batch_kernel_fn();
// with_dd: the batch holds DD 13/7 requests (the kernel that dispatches
// their kinds as well)
cudaError_t launch_batch(const BatchParams& p, int blocks, bool with_dd, cudaStream_t s);

}  // namespace dwt
