// Batched negacyclic NTT / inverse NTT over 64-bit RNS limbs: kernels and
// launch templates, compiled once per ring dimension (ntt_l10.cu .. ntt_l16.cu).
//
// Merged (twisted) Cooley-Tukey forward transform with bit-reversed output:
// row j of the result holds a(psi^(2 brv(j) + 1)); the Gentleman-Sande inverse
// takes that order back to coefficients and multiplies by N^-1.  Stage s
// (2^s butterfly groups, distance N / 2^(s+1)) uses twiddle psi^brv(2^s + i)
// for group i.
//
// Two passes per transform, each staged once through shared memory:
//  * "cols": stages 0 .. S1-1 only couple elements with equal index mod
//    T1 = N / 2^S1, so a CTA loads CW (8 or 16) adjacent columns of H = 2^S1
//    elements at stride T1 (64- or 128-byte row segments);
//  * "rows": stages S1 .. logN-1 stay inside contiguous blocks of T1
//    elements; a CTA of RT (128 or 256) threads loads RT / (T1 / 16) blocks.
// CW and RT are tile shapes chosen per context by the autotuner (tune.cu).
// Inside a pass every thread owns 16 elements of one column / block and runs
// the pass's stages in rounds of at most 4: load the 16 elements of its
// butterfly groups from shared memory into registers, apply the round's
// stages in registers, store back.  A 256-element column therefore costs two
// shared-memory round trips for its 8 stages.  All index arithmetic is fixed
// at compile time per ring dimension (template on log N).
// Values stay lazily reduced (forward [0, 4q), inverse [0, 2q)) until the
// last pass.  Launch: grid.y = row, grid.x = tile within the row.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "internal.h"
#include "kernels.h"
#include "modarith.cuh"

namespace mmfhe {

namespace {


// Every pass stages 16 words per thread: a loop over them with a compile-time
// trip count, so the loads of several iterations are in flight together.
#define MMFHE_TILE_LOOP(e, NT) _Pragma("unroll 8") for (int it_ = 0, e = threadIdx.x; it_ < 16; it_++, e += (NT))

// Position of register element (group g, index j) of a round covering local
// stages [A, A+R) of a sub-transform of size 2^LOG, for thread t that owns
// 16 >> R groups: j fills bits [POS, POS+R) with POS = LOG - A - R, the group
// number o = t * (16 >> R) + g fills the other bits.
template <int LOG, int A, int R>
__device__ __forceinline__ int elem_index(int t, int g, int j) {
    constexpr int POS = LOG - A - R;
    const int o = t * (16 >> R) + g;
    return ((o >> POS) << (POS + R)) | (j << POS) | (o & ((1 << POS) - 1));
}

// One round of R stages on 16 register-resident elements.
//   ADDR(h) -> shared-memory address of local element h
//   TWI(s, h) -> twiddle index of stage s (local stage, 0-based) for lower element h
template <int LOG, int A, int R, bool FWD, typename Addr, typename Twi>
__device__ __forceinline__ void ntt_round(uint64_t *sm, int t, uint64_t q, const uint64_t *__restrict__ W,
                                          const uint64_t *__restrict__ Wp, Addr addr, Twi twi) {
    constexpr int G = 16 >> R;
    constexpr int M = 1 << R;
    uint64_t x[16];
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int j = 0; j < M; j++) x[g * M + j] = sm[addr(elem_index<LOG, A, R>(t, g, j))];
    // At local stage u the butterflies (j, j + dist) whose lower index j shares
    // its top u bits use one twiddle: it is loaded once per run of dist pairs.
#pragma unroll
    for (int uu = 0; uu < R; uu++) {
        const int u = FWD ? uu : R - 1 - uu;
        const int dist = 1 << (R - 1 - u);
#pragma unroll
        for (int g = 0; g < G; g++) {
            uint64_t w = 0, wp = 0;
#pragma unroll
            for (int j = 0; j < M; j++) {
                if (j & dist) continue;
                if ((j & (dist - 1)) == 0) {   // first pair of a run sharing the twiddle
                    const int widx = twi(A + u, elem_index<LOG, A, R>(t, g, j));
                    w = __ldg(W + widx);
                    wp = __ldg(Wp + widx);
                }
                if (FWD)
                    mm::ct_butterfly(x[g * M + j], x[g * M + j + dist], w, wp, q);
                else
                    mm::gs_butterfly(x[g * M + j], x[g * M + j + dist], w, wp, q);
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int j = 0; j < M; j++) sm[addr(elem_index<LOG, A, R>(t, g, j))] = x[g * M + j];
}

// Tile geometry of the two passes.  CW = columns per CTA of the strided pass,
// RT = threads per CTA of the contiguous pass (both picked by the autotuner).
template <int LOGN, int CW = 16, int RT = 256>
struct Geo {
    static constexpr int S1 = (LOGN + 1) / 2;       // stages of the strided pass
    static constexpr int LOGT = LOGN - S1;          // stages of the contiguous pass
    static constexpr int H = 1 << S1;               // column length
    static constexpr int T1 = 1 << LOGT;            // block length
    static constexpr int R1C = S1 < 4 ? S1 : 4;     // round split of the strided pass
    static constexpr int R2C = S1 - R1C;
    static constexpr int R1R = LOGT < 4 ? LOGT : 4; // round split of the contiguous pass
    static constexpr int R2R = LOGT - R1R;
    static constexpr int TPC = H / 16;              // threads per column
    static constexpr int COLS = CW;
    static constexpr int COLS_THREADS = CW * TPC;
    static constexpr int TPR = T1 / 16;             // threads per block
    static constexpr int ROWS = (RT / TPR) < H ? (RT / TPR) : H;   // blocks per CTA
    static constexpr int ROWS_THREADS = ROWS * TPR;
    static constexpr int RS = T1 + T1 / 16;         // padded block stride in shared memory
    // resident CTAs the register budget is sized for (64 registers a thread)
    static constexpr int COLS_MINB = (1024 / COLS_THREADS) < 32 ? (1024 / COLS_THREADS) : 32;
    static constexpr int ROWS_MINB = (1024 / ROWS_THREADS) < 32 ? (1024 / ROWS_THREADS) : 32;
};

// Tile staging by asynchronous 8-byte copies global -> shared: a thread's
// 16 words are all in flight at once and hold no registers until the wait.
__device__ __forceinline__ void cp_async8(uint64_t *smem_dst, const uint64_t *gsrc) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}
// Completes this thread's copies (the barrier that follows publishes them).
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
// Closes the group of this thread's copies issued since the last commit.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Bulk prefetch of bytes (multiple of 16, 16-byte aligned start) into L2.
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Period row and block of grid row r (compact list of active rows).
__device__ __forceinline__ void row_decode(const RowMap &m, uint32_t r, uint32_t &blk, uint32_t &p) {
    blk = r / m.nact;
    p = m.act[r % m.nact];
}
__device__ __forceinline__ size_t row_at(const RowMap &m, uint32_t blk, uint32_t p, int logn) {
    return ((size_t)blk * m.block_stride + p - m.row0) << logn;
}

// Stages of the strided pass on a staged tile sm[H][COLS] (between the
// barriers that follow the load and precede the store).
template <int LOGN, bool FWD, int CW>
__device__ __forceinline__ void cols_rounds(uint64_t *sm, uint64_t q, uint32_t pid, const Twiddles &tw) {
    using Gm = Geo<LOGN, CW>;
    const int c = threadIdx.x % Gm::COLS, t = threadIdx.x / Gm::COLS;
    const uint64_t *W = (FWD ? tw.fw : tw.iw) + ((size_t)pid << LOGN);
    const uint64_t *Wp = (FWD ? tw.fw_sh : tw.iw_sh) + ((size_t)pid << LOGN);
    auto addr = [c](int h) { return h * Gm::COLS + c; };
    auto twi = [](int s, int h) { return (1 << s) + (h >> (Gm::S1 - s)); };
    if (FWD) {
        ntt_round<Gm::S1, 0, Gm::R1C, true>(sm, t, q, W, Wp, addr, twi);
        if (Gm::R2C > 0) {
            __syncthreads();
            ntt_round<Gm::S1, Gm::R1C, (Gm::R2C > 0 ? Gm::R2C : 1), true>(sm, t, q, W, Wp, addr, twi);
        }
    } else {
        if (Gm::R2C > 0) {
            ntt_round<Gm::S1, Gm::R1C, (Gm::R2C > 0 ? Gm::R2C : 1), false>(sm, t, q, W, Wp, addr, twi);
            __syncthreads();
        }
        ntt_round<Gm::S1, 0, Gm::R1C, false>(sm, t, q, W, Wp, addr, twi);
    }
}

// Stages of the contiguous pass on ROWS staged blocks (padded stride RS),
// the first being block hi0 of its row.
template <int LOGN, bool FWD, int RT>
__device__ __forceinline__ void rows_rounds(uint64_t *sm, int hi0, uint64_t q, uint32_t pid, const Twiddles &tw) {
    using Gm = Geo<LOGN, 16, RT>;
    const int t = threadIdx.x % Gm::TPR, rr = threadIdx.x / Gm::TPR;
    const int hi = hi0 + rr;
    const uint64_t *W = (FWD ? tw.fw : tw.iw) + ((size_t)pid << LOGN);
    const uint64_t *Wp = (FWD ? tw.fw_sh : tw.iw_sh) + ((size_t)pid << LOGN);
    uint64_t *row = sm + rr * Gm::RS;
    auto addr = [](int l) { return l + (l >> 4); };
    auto twi = [hi](int u, int l) {
        const int s = Gm::S1 + u;
        return (1 << s) + (hi << u) + (l >> (Gm::LOGT - u));
    };
    if (FWD) {
        ntt_round<Gm::LOGT, 0, Gm::R1R, true>(row, t, q, W, Wp, addr, twi);
        if (Gm::R2R > 0) {
            __syncthreads();
            ntt_round<Gm::LOGT, Gm::R1R, (Gm::R2R > 0 ? Gm::R2R : 1), true>(row, t, q, W, Wp, addr, twi);
        }
    } else {
        if (Gm::R2R > 0) {
            ntt_round<Gm::LOGT, Gm::R1R, (Gm::R2R > 0 ? Gm::R2R : 1), false>(row, t, q, W, Wp, addr, twi);
            __syncthreads();
        }
        ntt_round<Gm::LOGT, 0, Gm::R1R, false>(row, t, q, W, Wp, addr, twi);
    }
}

// Strided pass. FWD: stages 0..S1-1 (reads src, writes dst); inverse: stages
// S1-1..0 in place on dst, then the factor oscale[pid] (N^-1 when null).
template <int LOGN, bool FWD, int CW>
__global__ void __launch_bounds__(Geo<LOGN, CW>::COLS_THREADS, Geo<LOGN, CW>::COLS_MINB)
    k_ntt_cols(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst, RowMap md, ModTab mt, Twiddles tw,
               const uint64_t *__restrict__ oscale, const uint64_t *__restrict__ oscale_sh) {
    using Gm = Geo<LOGN, CW>;
    __shared__ uint64_t sm[Gm::H * Gm::COLS];
    uint32_t blk, p;
    row_decode(md, blockIdx.y, blk, p);
    const uint32_t pid = md.pid[p];
    const uint64_t *S = (FWD ? src + row_at(ms, blk, p, LOGN) : dst + row_at(md, blk, p, LOGN));
    uint64_t *D = dst + row_at(md, blk, p, LOGN);
    const int lo0 = blockIdx.x * Gm::COLS;
    const uint64_t q = mt.q[pid];
    MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) cp_async8(&sm[e], &S[(size_t)(e / Gm::COLS) * Gm::T1 + lo0 + (e % Gm::COLS)]);
    cp_async_wait_all();
    __syncthreads();
    cols_rounds<LOGN, FWD, CW>(sm, q, pid, tw);
    __syncthreads();
    if (FWD) {
        MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) D[(size_t)(e / Gm::COLS) * Gm::T1 + lo0 + (e % Gm::COLS)] = sm[e];
    } else {
        const uint64_t ni = oscale ? oscale[pid] : tw.ninv[pid], nip = oscale ? oscale_sh[pid] : tw.ninv_sh[pid];
        MMFHE_TILE_LOOP(e, Gm::COLS_THREADS)
            D[(size_t)(e / Gm::COLS) * Gm::T1 + lo0 + (e % Gm::COLS)] = mm::mul_shoup(sm[e], ni, nip, q);
    }
}

// Contiguous pass. FWD: stages S1..logN-1 in place on dst, final reduction to
// [0, q); inverse: stages logN-1..S1 (reads src, writes dst).
template <int LOGN, bool FWD, int RT>
__global__ void __launch_bounds__(Geo<LOGN, 16, RT>::ROWS_THREADS, Geo<LOGN, 16, RT>::ROWS_MINB)
    k_ntt_rows(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst, RowMap md, ModTab mt, Twiddles tw) {
    using Gm = Geo<LOGN, 16, RT>;
    __shared__ uint64_t sm[Gm::ROWS * Gm::RS];
    uint32_t blk, p;
    row_decode(md, blockIdx.y, blk, p);
    const uint32_t pid = md.pid[p];
    const uint64_t *S = (FWD ? dst + row_at(md, blk, p, LOGN) : src + row_at(ms, blk, p, LOGN));
    uint64_t *D = dst + row_at(md, blk, p, LOGN);
    const int hi0 = blockIdx.x * Gm::ROWS;
    const uint64_t q = mt.q[pid];
    const size_t base = (size_t)hi0 * Gm::T1;
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int rr = e / Gm::T1, l = e % Gm::T1;
        cp_async8(&sm[rr * Gm::RS + l + (l >> 4)], &S[base + e]);
    }
    cp_async_wait_all();
    __syncthreads();
    rows_rounds<LOGN, FWD, RT>(sm, hi0, q, pid, tw);
    __syncthreads();
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int r2 = e / Gm::T1, l = e % Gm::T1;
        uint64_t v = sm[r2 * Gm::RS + l + (l >> 4)];
        D[base + e] = FWD ? mm::reduce_4q(v, q) : v;
    }
}

// Per-row constants of a converted group, staged in shared memory: prime,
// q^-1 mod 2^64, the Montgomery factors f[r][k] (k < 8) and, for the
// centered conversion, c(-P) mod q and the half moduli of the sources.
template <int RG>
struct ConvConsts {
    uint64_t q[RG], qinv[RG], negp[RG], f[RG][8], half[8];
    uint32_t pid[RG];
};

// Base-conversion staging of the tiles of a group of nr <= RG rows: element
// (h, lo0 + c) of tile r is sum_k X[k][h * T1 + lo0 + c] * f[r][k], reduced
// once by Montgomery (the factors are in Montgomery form).  The NT source
// words of an element are loaded once for all rows of the group.  CENTERED
// adds c * negp[r] with c = #{k : X[k] > P_k / 2} (the ModDown conversion).
template <int LOGN, int CW, int RG, int NT, bool CENTERED>
__device__ __forceinline__ void conv_load(uint64_t *tiles, int nr, const uint64_t *__restrict__ X, int lo0,
                                          const ConvConsts<RG> &cc) {
    using Gm = Geo<LOGN, CW>;
    constexpr int TILE = Gm::H * Gm::COLS;
    MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) {
        const size_t idx = (size_t)(e / Gm::COLS) * Gm::T1 + lo0 + (e % Gm::COLS);
        uint64_t x[NT], neg = 0;
#pragma unroll
        for (int k = 0; k < NT; k++) {
            x[k] = X[((size_t)k << LOGN) + idx];
            if (CENTERED) neg += x[k] > cc.half[k] ? 1u : 0u;
        }
#pragma unroll
        for (int r = 0; r < RG; r++) {
            if (r >= nr) break;
            uint64_t hi = 0, lo = 0;
#pragma unroll
            for (int k = 0; k < NT; k++) mm::mac128(hi, lo, x[k], cc.f[r][k]);
            if (CENTERED) mm::mac128(hi, lo, neg, cc.negp[r]);
            tiles[r * TILE + e] = mm::redc(hi, lo, cc.q[r], cc.qinv[r]);
        }
    }
}

// Term counts above 4 (no parameter set here has them) share one loop.
template <int LOGN, int CW, int RG, bool CENTERED>
__device__ __forceinline__ void conv_load_any(uint64_t *tiles, int nr, const uint64_t *__restrict__ X, int nt,
                                              int lo0, const ConvConsts<RG> &cc) {
    using Gm = Geo<LOGN, CW>;
    constexpr int TILE = Gm::H * Gm::COLS;
    MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) {
        const size_t idx = (size_t)(e / Gm::COLS) * Gm::T1 + lo0 + (e % Gm::COLS);
        uint64_t neg = 0;
        if (CENTERED)
            for (int k = 0; k < nt; k++) neg += X[((size_t)k << LOGN) + idx] > cc.half[k] ? 1u : 0u;
        for (int r = 0; r < nr; r++) {
            uint64_t hi = 0, lo = 0;
            for (int k = 0; k < nt; k++) mm::mac128(hi, lo, X[((size_t)k << LOGN) + idx], cc.f[r][k]);
            if (CENTERED) mm::mac128(hi, lo, neg, cc.negp[r]);
            tiles[r * TILE + e] = mm::redc(hi, lo, cc.q[r], cc.qinv[r]);
        }
    }
}

template <int LOGN, int CW, int RG, bool CENTERED>
__device__ __forceinline__ void conv_dispatch(uint64_t *tiles, int nr, const uint64_t *X, int nt, int lo0,
                                              const ConvConsts<RG> &cc) {
    switch (nt) {   // uniform per CTA: the term loop is unrolled for the common counts
    case 1: conv_load<LOGN, CW, RG, 1, CENTERED>(tiles, nr, X, lo0, cc); break;
    case 2: conv_load<LOGN, CW, RG, 2, CENTERED>(tiles, nr, X, lo0, cc); break;
    case 3: conv_load<LOGN, CW, RG, 3, CENTERED>(tiles, nr, X, lo0, cc); break;
    case 4: conv_load<LOGN, CW, RG, 4, CENTERED>(tiles, nr, X, lo0, cc); break;
    default: conv_load_any<LOGN, CW, RG, CENTERED>(tiles, nr, X, nt, lo0, cc); break;
    }
}

// Stages 0..S1-1 of every tile of the group, then the tiles' stores.
template <int LOGN, int CW, int RG>
__device__ __forceinline__ void cols_finish_group(uint64_t *tiles, int nr, const ConvConsts<RG> &cc, uint64_t *dst,
                                                  const RowMap &md, const RowGroups &gr, uint32_t g, uint32_t blk,
                                                  int lo0, const Twiddles &tw) {
    using Gm = Geo<LOGN, CW>;
    constexpr int TILE = Gm::H * Gm::COLS;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RG; r++) {
        if (r >= nr) break;   // nr is uniform per CTA
        cols_rounds<LOGN, true, CW>(tiles + r * TILE, cc.q[r], cc.pid[r], tw);
    }
    __syncthreads();
    for (int r = 0; r < nr; r++) {
        uint64_t *D = dst + row_at(md, blk, md.act[gr.start[g] + r], LOGN);
        const uint64_t *T = tiles + r * TILE;
        MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) D[(size_t)(e / Gm::COLS) * Gm::T1 + lo0 + (e % Gm::COLS)] = T[e];
    }
}

// Fused ModUp strided pass on a group of digit rows (window blk, period rows
// p = j * nre + t of one digit j): each starts from
// sum_u y[blk][j*alpha+u] * Qhat_{j,u} mod prime(t), 128-bit products with the
// factor in Montgomery form reduced once (alpha * q_src * q_t < q_t * 2^64
// because alpha <= 8 and q_src < 2^61).  Tiles in dynamic shared memory.
template <int LOGN, int CW, int RG>
__global__ void __launch_bounds__(Geo<LOGN, CW>::COLS_THREADS, Geo<LOGN, CW>::COLS_MINB)
    k_ntt_cols_modup(const uint64_t *__restrict__ y, int nl, int nre, int alpha, int j0, uint64_t *dst, RowMap md,
                     RowGroups gr, const uint64_t *__restrict__ m_mont, ModTab mt, Twiddles tw) {
    using Gm = Geo<LOGN, CW>;
    extern __shared__ uint64_t tiles[];
    __shared__ ConvConsts<RG> cc;
    const uint32_t blk = blockIdx.y / gr.n, g = blockIdx.y % gr.n;
    const int nr = gr.count[g];
    const int j = j0 + (int)md.act[gr.start[g]] / nre;
    const int i0 = j * alpha, cnt = min(alpha, nl - i0);
    if (threadIdx.x < nr) {
        const int r = threadIdx.x;
        const uint32_t p = md.act[gr.start[g] + r], pid = md.pid[p];
        const int t = (int)p % nre;
        cc.q[r] = mt.q[pid];
        cc.qinv[r] = mt.qinv[pid];
        cc.pid[r] = pid;
        for (int u = 0; u < cnt; u++) cc.f[r][u] = m_mont[((size_t)j * MAX_ALPHA + u) * MAXROWMAP + t];
    }
    __syncthreads();
    const uint64_t *Y = y + (((size_t)blk * nl + i0) << LOGN);
    const int lo0 = blockIdx.x * Gm::COLS;
    conv_dispatch<LOGN, CW, RG, false>(tiles, nr, Y, cnt, lo0, cc);
    cols_finish_group<LOGN, CW, RG>(tiles, nr, cc, dst, md, gr, g, blk, lo0, tw);
}

// Key inner product word of window w (relative to a.w0), output part h,
// extended row t, position x: the beta 128-bit products (keys in Montgomery
// form) summed and reduced once, exactly as k_launch_keyip stores it.
template <int KB>
__device__ __forceinline__ uint64_t keyip_word(const KeyipArgs &a, uint32_t w, int h, int t, uint32_t x, int logn,
                                              uint64_t q, uint64_t qinv) {
    const uint32_t px = a.galois == 1 ? x : mm::galois_perm(x, a.galois, logn);
    const int krow = t <= a.level ? t : a.L1 + (t - a.level - 1);
    const int jown = t <= a.level ? t / a.alpha : -1;
    const size_t wa = (size_t)a.w0 + w;
    const uint64_t *K = a.key.k[a.key.n == 1 ? 0 : wa];
    const uint64_t *D = a.digits + ((wa * a.beta * a.nre + t) << logn) + px;
    uint64_t hi = 0, lo = 0;
#pragma unroll
    for (int j = 0; j < KB; j++) {
        if (j >= a.beta) break;
        const uint64_t kv = K[((((size_t)j * 2 + h) * a.key_rows + krow) << logn) + x];
        const uint64_t d = j == jown ? a.own[wa * a.own_stride + ((size_t)t << logn) + px]
                                     : D[((size_t)j * a.nre) << logn];
        mm::mac128(hi, lo, d, kv);
    }
    return mm::redc(hi, lo, q, qinv);
}

// Inverse contiguous pass over the P rows of the key inner product, whose
// words are formed in the load: row r = (w * 2 + h) * K + k of z holds
// part h of window w at special prime k.
template <int LOGN, int RT, int KB>
__global__ void __launch_bounds__(Geo<LOGN, 16, RT>::ROWS_THREADS, Geo<LOGN, 16, RT>::ROWS_MINB)
    k_ntt_rows_inv_keyip(KeyipArgs a, int K, int pid_p0, uint64_t *z, ModTab mt, Twiddles tw) {
    using Gm = Geo<LOGN, 16, RT>;
    __shared__ uint64_t sm[Gm::ROWS * Gm::RS];
    const uint32_t r = blockIdx.y, blk = r / (uint32_t)K;
    const int k = (int)(r % (uint32_t)K), t = a.level + 1 + k;
    const uint32_t pid = (uint32_t)(pid_p0 + k);
    const int hi0 = blockIdx.x * Gm::ROWS;
    const uint64_t q = mt.q[pid], qinv = mt.qinv[pid];
    const size_t base = (size_t)hi0 * Gm::T1;
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int rr = e / Gm::T1, l = e % Gm::T1;
        sm[rr * Gm::RS + l + (l >> 4)] = keyip_word<KB>(a, blk >> 1, (int)(blk & 1), t, (uint32_t)(base + e), LOGN, q, qinv);
    }
    __syncthreads();
    rows_rounds<LOGN, false, RT>(sm, hi0, q, pid, tw);
    __syncthreads();
    uint64_t *D = z + ((size_t)r << LOGN);
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int r2 = e / Gm::T1, l = e % Gm::T1;
        D[base + e] = sm[r2 * Gm::RS + l + (l >> 4)];
    }
}

// Fused ModDown strided pass on a group of rows (blk = window * 2 + h, p = i):
// each starts from the centered conversion
// v_i = sum_k z_k Phat_k + c (-P) mod q_i, c = #{k : z_k > p_k / 2}, in one
// Montgomery reduction (K (p_max - 1)(q - 1) + K (q - 1) < q 2^64 for K <= 8).
template <int LOGN, int CW, int RG>
__global__ void __launch_bounds__(Geo<LOGN, CW>::COLS_THREADS, Geo<LOGN, CW>::COLS_MINB)
    k_ntt_cols_moddown(const uint64_t *__restrict__ z, int K, int pid_p0, uint64_t *dst, RowMap md, RowGroups gr,
                       const uint64_t *__restrict__ phat_mont, const uint64_t *__restrict__ negp_mont, ModTab mt,
                       Twiddles tw) {
    using Gm = Geo<LOGN, CW>;
    extern __shared__ uint64_t tiles[];
    __shared__ ConvConsts<RG> cc;
    const uint32_t blk = blockIdx.y / gr.n, g = blockIdx.y % gr.n;
    const int nr = gr.count[g];
    if (threadIdx.x < nr) {
        const int r = threadIdx.x;
        const uint32_t pid = md.pid[md.act[gr.start[g] + r]];
        cc.q[r] = mt.q[pid];
        cc.qinv[r] = mt.qinv[pid];
        cc.pid[r] = pid;
        cc.negp[r] = negp_mont[pid];
        for (int k = 0; k < K; k++) cc.f[r][k] = phat_mont[(size_t)k * MMFHE_MAX_Q + pid];
    }
    if (threadIdx.x < K) cc.half[threadIdx.x] = mt.q[pid_p0 + threadIdx.x] >> 1;
    __syncthreads();
    const uint64_t *Z = z + (((size_t)blk * K) << LOGN);
    const int lo0 = blockIdx.x * Gm::COLS;
    conv_dispatch<LOGN, CW, RG, true>(tiles, nr, Z, K, lo0, cc);
    cols_finish_group<LOGN, CW, RG>(tiles, nr, cc, dst, md, gr, g, blk, lo0, tw);
}

// Fused ModDown contiguous pass: forward stages on v (rows blk = window * 2 + h,
// p = i, in place on vtmp) and the combine
//   out = (u - v) P^-1 + add_h[perm(x)] + plus  (mod q_i),
// u read from a.u (KB = 0) or formed from the key inner product's operands.
template <int LOGN, int RT, int KB>
__global__ void __launch_bounds__(Geo<LOGN, 16, RT>::ROWS_THREADS, Geo<LOGN, 16, RT>::ROWS_MINB)
    k_ntt_rows_combine(const uint64_t *__restrict__ v, RowMap mv, CombineArgs a, int nre,
                       const uint64_t *__restrict__ Pinv, const uint64_t *__restrict__ Pinv_sh, ModTab mt,
                       Twiddles tw, KeyipArgs ka) {
    using Gm = Geo<LOGN, 16, RT>;
    __shared__ uint64_t sm[Gm::ROWS * Gm::RS];
    uint32_t blk, p;
    row_decode(mv, blockIdx.y, blk, p);
    const uint32_t pid = mv.pid[p];
    const int nl = (int)mv.period;
    const uint64_t *S = v + row_at(mv, blk, p, LOGN);
    const int hi0 = blockIdx.x * Gm::ROWS;
    const uint64_t q = mt.q[pid];
    const size_t base = (size_t)hi0 * Gm::T1;
    const uint64_t *U = KB ? nullptr : a.u + (((size_t)blk * (a.u_stride ? a.u_stride : (size_t)nre) + p) << LOGN);
    const uint64_t *A = (blk & 1) ? a.add1 : a.add0;
    if (A) A += (size_t)(blk >> 1) * a.add_stride + ((size_t)p << LOGN);
    const uint64_t *Pl = a.plus ? a.plus + (((size_t)blk * nl + p) << LOGN) : nullptr;
    if (threadIdx.x == 0) {
        // the epilogue's contiguous operands travel to L2 while the stages run
        constexpr uint32_t seg = Gm::ROWS * Gm::T1 * 8;
        if (!KB) l2_prefetch(U + base, seg);
        if (Pl) l2_prefetch(Pl + base, seg);
        if (A && a.galois == 1) l2_prefetch(A + base, seg);
    }
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int rr = e / Gm::T1, l = e % Gm::T1;
        cp_async8(&sm[rr * Gm::RS + l + (l >> 4)], &S[base + e]);
    }
    cp_async_wait_all();
    __syncthreads();
    rows_rounds<LOGN, true, RT>(sm, hi0, q, pid, tw);
    __syncthreads();
    const uint64_t pi = Pinv[pid], pis = Pinv_sh[pid], qinv = mt.qinv[pid];
    uint64_t *O = a.out + (((size_t)blk * nl + p) << LOGN);
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int r2 = e / Gm::T1, l = e % Gm::T1;
        const uint32_t x = (uint32_t)(base + e);
        const uint64_t vv = mm::reduce_4q(sm[r2 * Gm::RS + l + (l >> 4)], q);
        const uint64_t uu = KB ? keyip_word<KB ? KB : 1>(ka, blk >> 1, (int)(blk & 1), (int)p, x, LOGN, q, qinv) : U[x];
        uint64_t res = mm::mul_shoup(mm::sub_mod(uu, vv, q), pi, pis, q);
        if (A) res = mm::add_mod(res, A[a.galois == 1 ? x : mm::galois_perm(x, a.galois, LOGN)], q);
        if (Pl) res = mm::add_mod(res, Pl[x], q);
        O[x] = res;
    }
}

// The combine of k_ntt_rows_combine (u read from a.u) with its tiles
// pipelined: a CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... (tile
// = row * (H / ROWS) + block of ROWS) and copies the v tile of the next one
// into its second shared buffer (asynchronous copies) while the current
// tile's stages and epilogue run; the next tile's contiguous epilogue
// operands go to L2 at the same time.  Same words.
template <int LOGN, int RT>
__global__ void __launch_bounds__(Geo<LOGN, 16, RT>::ROWS_THREADS, Geo<LOGN, 16, RT>::ROWS_MINB)
    k_ntt_rows_combine_pipe(const uint64_t *__restrict__ v, RowMap mv, CombineArgs a, int nre,
                            const uint64_t *__restrict__ Pinv, const uint64_t *__restrict__ Pinv_sh, ModTab mt,
                            Twiddles tw, uint32_t ntiles) {
    using Gm = Geo<LOGN, 16, RT>;
    constexpr uint32_t XT = Gm::H / Gm::ROWS;           // tiles per row
    constexpr uint32_t seg = Gm::ROWS * Gm::T1 * 8;     // bytes of a tile's contiguous operand
    __shared__ uint64_t sm[2][Gm::ROWS * Gm::RS];
    const int nl = (int)mv.period;
    struct Tile {
        uint32_t blk, p;
        size_t base;
        const uint64_t *U, *A, *Pl;
    };
    auto locate = [&](uint32_t tile) {
        Tile t;
        row_decode(mv, tile / XT, t.blk, t.p);
        t.base = (size_t)(tile % XT) * Gm::ROWS * Gm::T1;
        t.U = a.u + (((size_t)t.blk * (a.u_stride ? a.u_stride : (size_t)nre) + t.p) << LOGN);
        t.A = (t.blk & 1) ? a.add1 : a.add0;
        if (t.A) t.A += (size_t)(t.blk >> 1) * a.add_stride + ((size_t)t.p << LOGN);
        t.Pl = a.plus ? a.plus + (((size_t)t.blk * nl + t.p) << LOGN) : nullptr;
        return t;
    };
    auto issue = [&](uint32_t tile, int s) {
        const Tile t = locate(tile);
        const uint64_t *S = v + row_at(mv, t.blk, t.p, LOGN);
        MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
            int rr = e / Gm::T1, l = e % Gm::T1;
            cp_async8(&sm[s][rr * Gm::RS + l + (l >> 4)], &S[t.base + e]);
        }
        if (threadIdx.x == 0) {
            l2_prefetch(t.U + t.base, seg);
            if (t.Pl) l2_prefetch(t.Pl + t.base, seg);
            if (t.A && a.galois == 1) l2_prefetch(t.A + t.base, seg);
        }
    };
    uint32_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    issue(tile, 0);
    cp_async_commit();
    for (int s = 0; tile < ntiles; tile += gridDim.x, s ^= 1) {
        if (tile + gridDim.x < ntiles) issue(tile + gridDim.x, s ^ 1);
        cp_async_commit();      // possibly empty: one group always trails the current tile's
        cp_async_wait<1>();     // this thread's copies of the current tile have landed
        __syncthreads();        // ... and everyone's
        const Tile t = locate(tile);
        const uint32_t pid = mv.pid[t.p];
        const uint64_t q = mt.q[pid];
        const int hi0 = (int)(tile % XT) * Gm::ROWS;
        rows_rounds<LOGN, true, RT>(sm[s], hi0, q, pid, tw);
        __syncthreads();
        const uint64_t pi = Pinv[pid], pis = Pinv_sh[pid];
        uint64_t *O = a.out + (((size_t)t.blk * nl + t.p) << LOGN);
        MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
            int r2 = e / Gm::T1, l = e % Gm::T1;
            const uint32_t x = (uint32_t)(t.base + e);
            const uint64_t vv = mm::reduce_4q(sm[s][r2 * Gm::RS + l + (l >> 4)], q);
            uint64_t res = mm::mul_shoup(mm::sub_mod(t.U[x], vv, q), pi, pis, q);
            if (t.A) res = mm::add_mod(res, t.A[a.galois == 1 ? x : mm::galois_perm(x, a.galois, LOGN)], q);
            if (t.Pl) res = mm::add_mod(res, t.Pl[x], q);
            O[x] = res;
        }
        __syncthreads();        // sm[s] is refilled for the tile after next
    }
    cp_async_wait<0>();
}

// Butterflies of one pass over nr rows: N/2 per stage.
template <int LOGN>
double bf_cols(size_t nr) { return (double)nr * (double)(1u << (LOGN - 1)) * Geo<LOGN>::S1; }
template <int LOGN>
double bf_rows(size_t nr) { return (double)nr * (double)(1u << (LOGN - 1)) * Geo<LOGN>::LOGT; }

template <int LOGN, int CW, bool FWD>
void cols_pass(Context &c, const uint64_t *sb, const RowMap &ms, uint64_t *db, const RowMap &md, size_t nr,
               double bytes, const uint64_t *os, const uint64_t *os_sh, cudaStream_t st) {
    using Gm = Geo<LOGN, CW>;
    dim3 g(Gm::T1 / Gm::COLS, (unsigned)nr), b(Gm::COLS_THREADS);
    kernel_begin(c, st);
    k_ntt_cols<LOGN, FWD, CW><<<g, b, 0, st>>>(sb, ms, db, md, c.mods, c.tw, os, os_sh);
    kernel_end(c, FWD ? "ntt_fwd_cols" : "ntt_inv_cols", g, b, bytes, st, bf_cols<LOGN>(nr));
}

template <int LOGN, int RT, bool FWD>
void rows_pass(Context &c, const uint64_t *sb, const RowMap &ms, uint64_t *db, const RowMap &md, size_t nr,
               double bytes, cudaStream_t st) {
    using Gm = Geo<LOGN, 16, RT>;
    dim3 g(Gm::H / Gm::ROWS, (unsigned)nr), b(Gm::ROWS_THREADS);
    kernel_begin(c, st);
    k_ntt_rows<LOGN, FWD, RT><<<g, b, 0, st>>>(sb, ms, db, md, c.mods, c.tw);
    kernel_end(c, FWD ? "ntt_fwd_rows" : "ntt_inv_rows", g, b, bytes, st, bf_rows<LOGN>(nr));
}

// Both passes of a transform, with the tile shapes the context's tuning picked.
template <int LOGN>
void ntt_launch_t(Context &c, const uint64_t *sb, RowMap ms, uint64_t *db, RowMap md, size_t nr, bool inverse,
                  double bytes, const uint64_t *os, const uint64_t *os_sh, cudaStream_t st) {
    const bool c8 = c.tune.cols_w == 8, r128 = c.tune.rows_t == 128;
    if (!inverse) {
        if (c8) cols_pass<LOGN, 8, true>(c, sb, ms, db, md, nr, bytes, nullptr, nullptr, st);
        else cols_pass<LOGN, 16, true>(c, sb, ms, db, md, nr, bytes, nullptr, nullptr, st);
        if (r128) rows_pass<LOGN, 128, true>(c, db, md, db, md, nr, bytes, st);
        else rows_pass<LOGN, 256, true>(c, db, md, db, md, nr, bytes, st);
    } else {
        if (r128) rows_pass<LOGN, 128, false>(c, sb, ms, db, md, nr, bytes, st);
        else rows_pass<LOGN, 256, false>(c, sb, ms, db, md, nr, bytes, st);
        if (c8) cols_pass<LOGN, 8, false>(c, db, md, db, md, nr, bytes, os, os_sh, st);
        else cols_pass<LOGN, 16, false>(c, db, md, db, md, nr, bytes, os, os_sh, st);
    }
}

// Dynamic shared memory of a group's tiles (opted in above 48 KB once per kernel).
template <typename Kern>
void smem_opt_in(Kern k, size_t bytes) {
    if (bytes > 48 * 1024) CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <int LOGN, int CW, int RG>
void modup_cols_pass(Context &c, uint64_t *digits, const uint64_t *y, const RowMap &md, const RowGroups &gr,
                     size_t nblk, int nl, int nre, int j0, const uint64_t *m_mont, double bytes, size_t nr,
                     double macs, cudaStream_t st) {
    using Gm = Geo<LOGN, CW>;
    const size_t smem = (size_t)RG * Gm::H * Gm::COLS * 8;
    static bool opted = false;
    if (!opted) {
        smem_opt_in(k_ntt_cols_modup<LOGN, CW, RG>, smem);
        opted = true;
    }
    dim3 g(Gm::T1 / Gm::COLS, (unsigned)(nblk * gr.n)), b(Gm::COLS_THREADS);
    kernel_begin(c, st);
    k_ntt_cols_modup<LOGN, CW, RG><<<g, b, smem, st>>>(y, nl, nre, c.alpha, j0, digits, md, gr, m_mont, c.mods, c.tw);
    kernel_end(c, "ntt_modup_cols", g, b, bytes, st, bf_cols<LOGN>(nr), macs);
}

template <int LOGN, int CW>
void modup_cols_rg(Context &c, uint64_t *digits, const uint64_t *y, const RowMap &md, const RowGroups &gr, size_t nblk,
                   int nl, int nre, int j0, const uint64_t *m_mont, double bytes, size_t nr, double macs,
                   cudaStream_t st) {
    if (c.tune.conv_rows == 4) modup_cols_pass<LOGN, CW, 4>(c, digits, y, md, gr, nblk, nl, nre, j0, m_mont, bytes, nr, macs, st);
    else if (c.tune.conv_rows == 2) modup_cols_pass<LOGN, CW, 2>(c, digits, y, md, gr, nblk, nl, nre, j0, m_mont, bytes, nr, macs, st);
    else modup_cols_pass<LOGN, CW, 1>(c, digits, y, md, gr, nblk, nl, nre, j0, m_mont, bytes, nr, macs, st);
}

template <int LOGN>
void modup_launch_t(Context &c, uint64_t *digits, const uint64_t *y, const RowMap &md, const RowGroups &gr,
                    size_t nblk, int nl, int nre, int j0, const uint64_t *m_mont, double bytes_cols, double bytes_rows,
                    double macs, cudaStream_t st) {
    const size_t nr = nblk * md.nact;
    if (c.tune.cols_w == 8) modup_cols_rg<LOGN, 8>(c, digits, y, md, gr, nblk, nl, nre, j0, m_mont, bytes_cols, nr, macs, st);
    else modup_cols_rg<LOGN, 16>(c, digits, y, md, gr, nblk, nl, nre, j0, m_mont, bytes_cols, nr, macs, st);
    if (c.tune.rows_t == 128) rows_pass<LOGN, 128, true>(c, digits, md, digits, md, nr, bytes_rows, st);
    else rows_pass<LOGN, 256, true>(c, digits, md, digits, md, nr, bytes_rows, st);
}

template <int LOGN, int CW, int RG>
void moddown_cols_pass(Context &c, uint64_t *vtmp, const uint64_t *z, const RowMap &mv, const RowGroups &gr,
                       size_t nblk, double bytes, size_t nr, double macs, cudaStream_t st) {
    using Gm = Geo<LOGN, CW>;
    const size_t smem = (size_t)RG * Gm::H * Gm::COLS * 8;
    static bool opted = false;
    if (!opted) {
        smem_opt_in(k_ntt_cols_moddown<LOGN, CW, RG>, smem);
        opted = true;
    }
    dim3 g(Gm::T1 / Gm::COLS, (unsigned)(nblk * gr.n)), b(Gm::COLS_THREADS);
    kernel_begin(c, st);
    k_ntt_cols_moddown<LOGN, CW, RG><<<g, b, smem, st>>>(z, c.num_p, c.num_q, vtmp, mv, gr, c.d_dn_phat_mont,
                                                         c.d_dn_negp_mont, c.mods, c.tw);
    kernel_end(c, "ntt_moddown_cols", g, b, bytes, st, bf_cols<LOGN>(nr), macs);
}

template <int LOGN, int CW>
void moddown_cols_rg(Context &c, uint64_t *vtmp, const uint64_t *z, const RowMap &mv, const RowGroups &gr, size_t nblk,
                     double bytes, size_t nr, double macs, cudaStream_t st) {
    if (c.tune.conv_rows == 4) moddown_cols_pass<LOGN, CW, 4>(c, vtmp, z, mv, gr, nblk, bytes, nr, macs, st);
    else if (c.tune.conv_rows == 2) moddown_cols_pass<LOGN, CW, 2>(c, vtmp, z, mv, gr, nblk, bytes, nr, macs, st);
    else moddown_cols_pass<LOGN, CW, 1>(c, vtmp, z, mv, gr, nblk, bytes, nr, macs, st);
}

template <int LOGN, int RT>
void combine_rows_pass(Context &c, uint64_t *vtmp, const RowMap &mv, size_t nr, const CombineArgs &a, int nre,
                       double bytes, const KeyipArgs *ka, cudaStream_t st) {
    using Gm = Geo<LOGN, 16, RT>;
    dim3 g(Gm::H / Gm::ROWS, (unsigned)nr), b(Gm::ROWS_THREADS);
    // the pipelined combine keeps two tile buffers in static shared memory (at most 48 KB)
    if constexpr (2 * Gm::ROWS * Gm::RS * 8 <= 48 * 1024) {
        if (!ka && c.tune.combine_pipe) {
            // persistent CTAs: as many as fit on the GPU at once
            static int per_sm = 0;
            if (!per_sm)
                CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ntt_rows_combine_pipe<LOGN, RT>,
                                                                  Gm::ROWS_THREADS, 0));
            const uint32_t ntiles = (uint32_t)(Gm::H / Gm::ROWS) * (uint32_t)nr;
            dim3 gp((unsigned)std::min<size_t>(ntiles, (size_t)c.sm_count * std::max(per_sm, 1)));
            kernel_begin(c, st);
            k_ntt_rows_combine_pipe<LOGN, RT><<<gp, b, 0, st>>>(vtmp, mv, a, nre, c.d_dn_Pinv, c.d_dn_Pinv_sh,
                                                                 c.mods, c.tw, ntiles);
            kernel_end(c, "ntt_combine_rows", gp, b, bytes, st, bf_rows<LOGN>(nr));
            return;
        }
    }
    kernel_begin(c, st);
    if (!ka) {
        k_ntt_rows_combine<LOGN, RT, 0><<<g, b, 0, st>>>(vtmp, mv, a, nre, c.d_dn_Pinv, c.d_dn_Pinv_sh, c.mods, c.tw,
                                                         KeyipArgs{});
        kernel_end(c, "ntt_combine_rows", g, b, bytes, st, bf_rows<LOGN>(nr));
        return;
    }
    if (ka->beta <= 4)
        k_ntt_rows_combine<LOGN, RT, 4><<<g, b, 0, st>>>(vtmp, mv, a, nre, c.d_dn_Pinv, c.d_dn_Pinv_sh, c.mods, c.tw, *ka);
    else
        k_ntt_rows_combine<LOGN, RT, MAX_DNUM><<<g, b, 0, st>>>(vtmp, mv, a, nre, c.d_dn_Pinv, c.d_dn_Pinv_sh, c.mods,
                                                                c.tw, *ka);
    kernel_end(c, "ntt_combine_keyip_rows", g, b, bytes, st, bf_rows<LOGN>(nr), (double)nr * c.n * ka->beta);
}

template <int LOGN>
void moddown_launch_t(Context &c, uint64_t *vtmp, const uint64_t *z, const RowMap &mv, const RowGroups &gr,
                      size_t nblk, const CombineArgs &a, int nre, double bytes_cols, double bytes_rows,
                      double macs, const KeyipArgs *ka, cudaStream_t st) {
    const size_t nr = nblk * mv.nact;
    if (c.tune.cols_w == 8) moddown_cols_rg<LOGN, 8>(c, vtmp, z, mv, gr, nblk, bytes_cols, nr, macs, st);
    else moddown_cols_rg<LOGN, 16>(c, vtmp, z, mv, gr, nblk, bytes_cols, nr, macs, st);
    if (c.tune.rows_t == 128) combine_rows_pass<LOGN, 128>(c, vtmp, mv, nr, a, nre, bytes_rows, ka, st);
    else combine_rows_pass<LOGN, 256>(c, vtmp, mv, nr, a, nre, bytes_rows, ka, st);
}

template <int LOGN, int RT>
void inv_keyip_rows_pass(Context &c, uint64_t *z, const KeyipArgs &ka, size_t nr, double bytes, cudaStream_t st) {
    using Gm = Geo<LOGN, 16, RT>;
    dim3 g(Gm::H / Gm::ROWS, (unsigned)nr), b(Gm::ROWS_THREADS);
    kernel_begin(c, st);
    if (ka.beta <= 4)
        k_ntt_rows_inv_keyip<LOGN, RT, 4><<<g, b, 0, st>>>(ka, c.num_p, c.num_q, z, c.mods, c.tw);
    else
        k_ntt_rows_inv_keyip<LOGN, RT, MAX_DNUM><<<g, b, 0, st>>>(ka, c.num_p, c.num_q, z, c.mods, c.tw);
    kernel_end(c, "ntt_inv_keyip_rows", g, b, bytes, st, bf_rows<LOGN>(nr), (double)nr * c.n * ka.beta);
}

// The P rows of the key inner product into z ([rows of (window, h)][K][N]):
// the contiguous inverse pass forming them, then the strided inverse pass
// with the factor oscale[pid].
template <int LOGN>
void keyip_p_inv_launch_t(Context &c, uint64_t *z, const KeyipArgs &ka, const RowMap &mz, size_t nr,
                          double bytes_rows, double bytes_cols, const uint64_t *os, const uint64_t *os_sh,
                          cudaStream_t st) {
    if (c.tune.rows_t == 128) inv_keyip_rows_pass<LOGN, 128>(c, z, ka, nr, bytes_rows, st);
    else inv_keyip_rows_pass<LOGN, 256>(c, z, ka, nr, bytes_rows, st);
    if (c.tune.cols_w == 8) cols_pass<LOGN, 8, false>(c, z, mz, z, mz, nr, bytes_cols, os, os_sh, st);
    else cols_pass<LOGN, 16, false>(c, z, mz, z, mz, nr, bytes_cols, os, os_sh, st);
}

}  // namespace
}  // namespace mmfhe
