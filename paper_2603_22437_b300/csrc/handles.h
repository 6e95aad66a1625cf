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

// Evaluate a plan on `batch` windows (abi.cu).  Windows with the same key set
// form one batch; with mix_users, windows of different key sets share batches
// of up to MAX_KEY_WINDOWS (each window switched with its own keys).
// Pointers may be host or device memory.
// in_scale: the inputs' encryption scale (bookkeeping only: no word depends
// on it); out_scales (nullable) receives the outputs' tracked scales.
void eval_windows(Context &c, const Plan &p, const Keys *const *keys, const uint64_t *const *in_cts, size_t batch,
                  uint64_t *const *out_cts, cudaStream_t st, bool mix_users = false, double in_scale = 1.0,
                  std::vector<double> *out_scales = nullptr);
// Message returned by mmfhe_last_error(NULL) on the calling thread (abi.cu).
void set_thread_error(const std::string &msg);
// True unless p is device (or managed) memory.
bool is_host_ptr(const void *p);
// Upload one switching key ([dnum][2][L+1+K][N], coefficient form, host or
// device words) into the evaluation domain in Montgomery form (abi.cu).
Buf load_key(Context &c, const uint64_t *words);

}  // namespace mmfhe
