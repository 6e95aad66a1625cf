// Autotuner: times the tile-shape variants of the NTT passes and the window
// group of the key inner product on the caller's batch shape, and keeps the
// fastest in the context.  Every variant computes the same words, so tuning
// changes only speed.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "engine.h"
#include "handles.h"
#include "internal.h"
#include "kernels.h"

namespace mmfhe {

namespace {

constexpr int TUNE_REPS = 3;

// Best-of-TUNE_REPS CUDA-event time of f() on stream st, after one warm-up call.
template <typename F>
float time_best(cudaStream_t st, F f) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    f();
    float best = 1e30f;
    for (int r = 0; r < TUNE_REPS; r++) {
        CK(cudaEventRecord(a, st));
        f();
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

}  // namespace

void autotune(Context &c, int batch, int level) {
    if (batch < 1 || level < 0 || level > c.L) throw Error(MMFHE_ERR_BAD_ARG, "autotune: bad batch or level");
    const bool prof = c.profiling, trace = c.tracing;
    c.profiling = c.tracing = false;
    cudaStream_t st = nullptr;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    Tune best = c.tune;
    try {
        const int nl = level + 1, nre = nl + c.num_p, beta = c.lv[level].beta;
        // NTT: forward + inverse of the batch's ciphertext rows (zero words are valid residues)
        Buf x(c.pool.get(), (size_t)batch * 2 * nl * c.n);
        CK(cudaMemsetAsync(x.get(), 0, x.words() * 8, st));
        const int cws[2] = {8, 16}, rts[2] = {128, 256};
        float bt = 1e30f;
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                c.tune.cols_w = cws[i];
                c.tune.rows_t = rts[j];
                const float ms = time_best(st, [&] {
                    ntt_q_blocks(c, x.get(), (size_t)batch * 2, nl, false, st);
                    ntt_q_blocks(c, x.get(), (size_t)batch * 2, nl, true, st);
                });
                best.ntt_ms[2 * i + j] = ms;
                if (ms < bt) {
                    bt = ms;
                    best.cols_w = cws[i];
                    best.rows_t = rts[j];
                }
            }
        x.release();
        // key inner product of one rotation: digits, own rows and a key of this level's shape
        Buf dg(c.pool.get(), (size_t)batch * beta * nre * c.n), own(c.pool.get(), (size_t)batch * nl * c.n);
        Buf key(c.pool.get(), (size_t)c.dnum * 2 * (c.num_q + c.num_p) * c.n), u(c.pool.get(), (size_t)batch * 2 * nre * c.n);
        CK(cudaMemsetAsync(dg.get(), 0, dg.words() * 8, st));
        CK(cudaMemsetAsync(own.get(), 0, own.words() * 8, st));
        CK(cudaMemsetAsync(key.get(), 0, key.words() * 8, st));
        const uint32_t g = galois_elt(c, 1);
        KeyPtrs kp;
        kp.k[0] = key.get();
        kp.n = 1;
        const int wgs[4] = {1, 2, 4, 8};
        float bk = 1e30f;
        for (int pipe = 0; pipe < 2; pipe++)
            for (int i = 0; i < 4; i++) {
                c.tune.keyip_wg = wgs[i];
                c.tune.keyip_pipe = pipe;
                const float ms = time_best(st, [&] {
                    k_launch_keyip(c, u.get(), dg.get(), own.get(), (size_t)nl * c.n, 0, kp, batch, level, beta, g,
                                   st);
                });
                (pipe ? best.keyip_pipe_ms : best.keyip_ms)[i] = ms;
                if (ms < bk) {
                    bk = ms;
                    best.keyip_wg = wgs[i];
                    best.keyip_pipe = pipe;
                }
            }
        dg.release();
        own.release();
        key.release();
        // fused ModUp + ModDown passes: converted rows per CTA (uses the tiles picked above)
        c.tune.cols_w = best.cols_w;
        c.tune.rows_t = best.rows_t;
        Buf y(c.pool.get(), (size_t)batch * nl * c.n), dig(c.pool.get(), (size_t)batch * beta * nre * c.n);
        Buf z(c.pool.get(), (size_t)batch * 2 * c.num_p * c.n), v(c.pool.get(), (size_t)batch * 2 * nl * c.n);
        Buf out(c.pool.get(), (size_t)batch * 2 * nl * c.n);
        CK(cudaMemsetAsync(y.get(), 0, y.words() * 8, st));
        CK(cudaMemsetAsync(z.get(), 0, z.words() * 8, st));
        CK(cudaMemsetAsync(u.get(), 0, u.words() * 8, st));
        const CombineArgs ca{out.get(), u.get(), nullptr, nullptr, 0, 1, nullptr};
        const int rgs[3] = {1, 2, 4};
        float bg = 1e30f;
        for (int cp = 0; cp < 2; cp++)
            for (int i = 0; i < 3; i++) {
                c.tune.conv_rows = rgs[i];
                c.tune.combine_pipe = cp;
                const float ms = time_best(st, [&] {
                    launch_modup_ntt(c, dig.get(), y.get(), batch, level, st);
                    launch_moddown_ntt(c, v.get(), z.get(), ca, batch, level, st);
                });
                (cp ? best.combine_pipe_ms : best.conv_ms)[i] = ms;
                if (ms < bg) {
                    bg = ms;
                    best.conv_rows = rgs[i];
                    best.combine_pipe = cp;
                }
            }
        CK(cudaStreamSynchronize(st));
    } catch (...) {
        cudaStreamDestroy(st);
        c.profiling = prof;
        c.tracing = trace;
        throw;
    }
    cudaStreamDestroy(st);
    c.tune = best;
    c.profiling = prof;
    c.tracing = trace;
}

}  // namespace mmfhe

using namespace mmfhe;

namespace {

mmfhe_status tfail(Context *c, mmfhe_status code, const char *msg) {
    if (c) c->last_error = msg;
    return code;
}

void to_abi(const Tune &t, mmfhe_tuning *out) {
    out->ntt_cols_width = (uint32_t)t.cols_w;
    out->ntt_rows_threads = (uint32_t)t.rows_t;
    out->keyip_windows = (uint32_t)t.keyip_wg;
    std::copy(t.ntt_ms, t.ntt_ms + 4, out->ntt_ms);
    std::copy(t.keyip_ms, t.keyip_ms + 4, out->keyip_ms);
    out->conv_rows = (uint32_t)t.conv_rows;
    std::copy(t.conv_ms, t.conv_ms + 3, out->conv_ms);
    out->keyip_fused = (uint32_t)t.keyip_fused;
    out->keyip_pipe = (uint32_t)t.keyip_pipe;
    std::copy(t.keyip_pipe_ms, t.keyip_pipe_ms + 4, out->keyip_pipe_ms);
    out->combine_pipe = (uint32_t)t.combine_pipe;
    std::copy(t.combine_pipe_ms, t.combine_pipe_ms + 3, out->combine_pipe_ms);
}

}  // namespace

extern "C" {

mmfhe_status mmfhe_autotune(mmfhe_ctx *ctx, uint32_t batch, uint32_t level, mmfhe_tuning *out) {
    Context *c = nullptr;
    try {
        if (!ctx || !ctx->c) throw Error(MMFHE_ERR_BAD_ARG, "null context");
        c = ctx->c;
        CK(cudaSetDevice(c->device));
        autotune(*c, (int)batch, (int)level);
        if (out) to_abi(c->tune, out);
    } catch (const Error &e) {
        return tfail(c, e.code, e.what());
    } catch (const std::exception &e) {
        return tfail(c, MMFHE_ERR_CUDA, e.what());
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_tuning_get(const mmfhe_ctx *ctx, mmfhe_tuning *out) {
    if (!ctx || !ctx->c || !out) return tfail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    to_abi(ctx->c->tune, out);
    return MMFHE_OK;
}

mmfhe_status mmfhe_tuning_set(mmfhe_ctx *ctx, const mmfhe_tuning *in) {
    if (!ctx || !ctx->c || !in) return tfail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    Context *c = ctx->c;
    const uint32_t w = in->ntt_cols_width, r = in->ntt_rows_threads, k = in->keyip_windows, g = in->conv_rows;
    if ((w != 8 && w != 16) || (r != 128 && r != 256) || (k != 1 && k != 2 && k != 4 && k != 8) ||
        (g != 1 && g != 2 && g != 4) || in->keyip_fused > 1 || in->keyip_pipe > 1 || in->combine_pipe > 1)
        return tfail(c, MMFHE_ERR_BAD_ARG, "unsupported tile shape");
    c->tune.combine_pipe = (int)in->combine_pipe;
    c->tune.keyip_fused = (int)in->keyip_fused;
    c->tune.keyip_pipe = (int)in->keyip_pipe;
    c->tune.conv_rows = (int)g;
    c->tune.cols_w = (int)w;
    c->tune.rows_t = (int)r;
    c->tune.keyip_wg = (int)k;
    return MMFHE_OK;
}

}  // extern "C"
