// Descriptors of the persistent batch kernel (batch.cu), shared with the
// host API.  Not part of the public ABI.
#pragma once

#include "dwt_internal.h"

namespace dwt {

// Kinds of request a batch can hold (scheme fixed per kind: Monolithic* for
// float, the separable JPEG 2000 order for reversible 5/3).
enum BatchKind : int {
  BK_97_F32_FWD = 0, BK_97_F32_INV, BK_53_F32_FWD, BK_53_F32_INV, BK_53_I32_FWD, BK_53_I32_INV,
  BK_97_F16_FWD, BK_97_F16_INV, BK_53_F16_FWD, BK_53_F16_INV, BK_COUNT
};


// One (request, step): everything a strip of it needs.  The tensor maps come
// first so that every element of an array of these is 64-byte aligned.
struct alignas(64) BatchLevel {
  TmaMaps maps;
  LevelArgs a;
  Coefs cf;
  int kind;
  int request;
  int nstrips;
  int dep;  // index of the level whose strips this one waits for, or -1
};

struct BatchItem {
  int level;
  int strip;
};

struct BatchParams {
  const BatchLevel* levels;
  const BatchItem* items;
  int nitems;
  int* head;        // next item to take
  int* done;        // per level: strips finished
  int* req_status;  // per request, may be null
};

bool batch_kind_info(int kind, KernelInfo* k);
size_t batch_smem_bytes();
const void* batch_kernel_fn();
cudaError_t launch_batch(const BatchParams& p, int blocks, cudaStream_t s);

}  // namespace dwt
