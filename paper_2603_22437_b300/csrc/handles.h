// Opaque handle types of the C ABI and the helpers shared by the files that
// implement its entry points (abi.cu, noalloc.cu, batcher.cu).
#pragma once
#include <cuda_runtime.h>

#include "circuits.h"
#include "internal.h"

struct mmfhe_ctx {
    mmfhe::Context *c;
};
struct mmfhe_keys {
    mmfhe::Keys k;
};
struct mmfhe_plan {
    mmfhe::Plan *p;
};

namespace mmfhe {

// Evaluate a plan on `batch` windows (abi.cu); windows with the same key set
// form one batch.  Pointers may be host or device memory.
void eval_windows(Context &c, const Plan &p, const Keys *const *keys, const uint64_t *const *in_cts, size_t batch,
                  uint64_t *const *out_cts, cudaStream_t st);
// True unless p is device (or managed) memory.
bool is_host_ptr(const void *p);

}  // namespace mmfhe
