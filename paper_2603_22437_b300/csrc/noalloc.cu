// mmfhe_keyswitch_noalloc: the key switch of mmfhe_keyswitch with every
// intermediate in a fixed, statically allocated device array instead of
// memory obtained from cudaMalloc.
//
// Who needs it: code that runs where device allocation is not allowed --
// for example inside a host callback or a section that must not take the
// allocator's lock, a process whose device memory is handed out in full to
// another allocator up front, or an embedded host runtime that forbids
// cudaMalloc/cudaFree after start-up.  Such callers still own their input
// and output buffers; this entry point adds no allocation of its own.
//
// The scratch array below is file-scope device memory: every GPU that loads
// the library holds it until the process exits.  Host code cannot use the
// name g_ks_scratch as a device address (on the host it is only a stand-in
// symbol); its device address is obtained with cudaGetSymbolAddress, with the
// context's device current, on the first call made with each context.
#include <cuda_runtime.h>

#include "engine.h"
#include "handles.h"
#include "internal.h"
#include "kernels.h"

using namespace mmfhe;


namespace {

constexpr size_t kScratchWords = MMFHE_NOALLOC_SCRATCH_BYTES / sizeof(uint64_t);
static __device__ __align__(256) uint64_t g_ks_scratch[kScratchWords];

// Device address of the scratch array, looked up once per context with the
// context's device current (the caller has made it current) and kept in the
// context, so a context created after a device reset looks it up afresh.
uint64_t *scratch_address(Context &c) {
    if (!c.noalloc_scratch) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_ks_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            throw Error(MMFHE_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") + cudaGetErrorString(e));
        }
        c.noalloc_scratch = (uint64_t *)p;
    }
    return c.noalloc_scratch;
}

// Row map without heap use: rows [0, period) map to the given prime ids.
RowMap map_q(int nl, uint32_t block_stride) {
    RowMap m{};
    m.period = (uint32_t)nl;
    m.block_stride = block_stride;
    for (int i = 0; i < nl; i++) m.pid[i] = (uint8_t)i;
    return m;
}

// True for device memory of `device` itself and for managed memory; false for
// host memory and for another GPU's memory (the kernels run on `device` and
// would fault on a peer's pointer).
bool is_device_ptr(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

mmfhe_status fail(Context *c, mmfhe_status code, const char *msg) {
    if (c) c->last_error = msg;
    return code;
}

}  // namespace

extern "C" mmfhe_status mmfhe_keyswitch_noalloc(mmfhe_ctx *ctx, const mmfhe_keys *keys, int which, int32_t rotation,
                                                uint64_t *out, const uint64_t *d, size_t batch, uint32_t level,
                                                void *stream) {
    Context *c = nullptr;
    try {
        if (!ctx || !ctx->c) throw Error(MMFHE_ERR_BAD_ARG, "null context");
        c = ctx->c;
        CK(cudaSetDevice(c->device));
        if (!keys || keys->k.ctx != c) throw Error(MMFHE_ERR_PARAM_MISMATCH, "keys belong to another context");
        if ((int)level > c->L) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "level above the top level");
        if (batch == 0) return MMFHE_OK;
        if (!out || !d) throw Error(MMFHE_ERR_BAD_ARG, "null pointer");
        if (!is_device_ptr(out, c->device) || !is_device_ptr(d, c->device) || ((uintptr_t)out & 15) ||
            ((uintptr_t)d & 15))
            throw Error(MMFHE_ERR_BAD_ARG, "keyswitch_noalloc needs 16-byte aligned pointers to the context's device");
        const Keys &K = keys->k;
        const KeyPtrs key = which == 0 ? relin_key(K) : galois_key(K, norm_rot(*c, rotation));
        cudaStream_t st = (cudaStream_t)stream;
        const int nl = (int)level + 1, nre = nl + c->num_p;
        const LevelConsts &lc = c->lv[level];
        const int beta = lc.beta;
        const size_t B = batch, N = c->n;
        // scratch regions (rows of N words): D = NTT(d) [B][nl], G = digits
        // [B][beta][nre], U = inner product [B][2][nre], V = ModDown
        // conversion [B][2][nl], O = result in the evaluation domain [B][2][nl]
        const size_t rows = B * ((size_t)nl + (size_t)beta * nre + 2 * (size_t)nre + 4 * (size_t)nl);
        if (rows * N > kScratchWords)
            throw Error(MMFHE_ERR_BAD_ARG, "keyswitch_noalloc: batch x level needs " + std::to_string(rows * N * 8) +
                                                " bytes of scratch, more than the fixed " +
                                                std::to_string((size_t)MMFHE_NOALLOC_SCRATCH_BYTES) + " bytes");
        uint64_t *S = scratch_address(*c);
        uint64_t *Dr = S;
        uint64_t *Gr = Dr + B * nl * N;
        uint64_t *Ur = Gr + B * beta * nre * N;
        uint64_t *Vr = Ur + B * 2 * nre * N;
        uint64_t *Or = Vr + B * 2 * nl * N;
        // No region has to start at zero: every word read below is written
        // earlier in this call.
        // 1. evaluation form of d (the caller's d is the coefficient form ModUp needs)
        RowsView src{const_cast<uint64_t *>(d), map_q(nl, nl), B * nl};
        RowsView dst{Dr, map_q(nl, nl), B * nl};
        launch_ntt(*c, src, dst, false, st);
        // 2. ModUp: FastBConv of each digit, then NTT of the converted rows
        k_launch_modup_bconv(*c, Gr, d, Dr, (size_t)nl * N, (int)B, (int)level, modup_consts(*c, (int)level), st);
        for (int j = 0; j < beta; j++) {
            RowMap m{};
            m.period = (uint32_t)nre;
            m.block_stride = (uint32_t)(beta * nre);
            for (int t = 0; t < nre; t++) {
                bool own = t <= (int)level && t >= lc.digits[j].front() && t <= lc.digits[j].back();
                m.pid[t] = own ? SKIP : (uint8_t)(t <= (int)level ? t : c->num_q + (t - nl));
            }
            RowsView v{Gr + (size_t)j * nre * N, m, B * nre};
            launch_ntt(*c, v, v, false, st);
        }
        // 3. key inner product, 4. ModDown
        k_launch_keyip(*c, Ur, Gr, Gr, (size_t)beta * nre * N, (size_t)nre * N, key, (int)B, (int)level, beta, 1, st);
        RowMap pm{};
        pm.period = (uint32_t)nre;
        pm.block_stride = (uint32_t)nre;
        for (int t = 0; t < nre; t++) pm.pid[t] = t < nl ? SKIP : (uint8_t)(c->num_q + (t - nl));
        RowsView pv{Ur, pm, B * 2 * nre};
        launch_ntt(*c, pv, pv, true, st);
        ModDownConsts dc = moddown_consts(*c);
        k_launch_moddown_bconv(*c, Vr, Ur, (int)B, (int)level, dc, st);
        RowsView vv{Vr, map_q(nl, nl), B * 2 * nl};
        launch_ntt(*c, vv, vv, false, st);
        k_launch_moddown_combine(*c, Or, Ur, Vr, nullptr, nullptr, 0, 1, (int)B, (int)level, dc, st);
        // 5. back to coefficient form, straight into the caller's output
        RowsView os{Or, map_q(nl, nl), B * 2 * nl};
        RowsView od{out, map_q(nl, nl), B * 2 * nl};
        launch_ntt(*c, os, od, true, st);
        CK(cudaGetLastError());
    } catch (const Error &e) {
        return fail(c, e.code, e.what());
    } catch (const std::exception &e) {
        return fail(c, MMFHE_ERR_CUDA, e.what());
    } catch (...) {
        return fail(c, MMFHE_ERR_CUDA, "unknown error");
    }
    return MMFHE_OK;
}
