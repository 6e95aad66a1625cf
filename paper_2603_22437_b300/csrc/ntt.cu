// Batched negacyclic NTT / inverse NTT over 64-bit RNS limbs.
//
// Merged (twisted) Cooley-Tukey forward transform with bit-reversed output:
// row j of the result holds a(psi^(2 brv(j) + 1)); the Gentleman-Sande inverse
// takes that order back to coefficients and multiplies by N^-1.  Stage s
// (2^s butterfly groups, distance N / 2^(s+1)) uses twiddle psi^brv(2^s + i)
// for group i.
//
// Two passes per transform, each staged once through shared memory:
//  * "cols": stages 0 .. S1-1 only couple elements with equal index mod
//    T1 = N / 2^S1, so a CTA loads 16 adjacent columns of H = 2^S1 elements
//    at stride T1 (128-byte row segments);
//  * "rows": stages S1 .. logN-1 stay inside contiguous blocks of T1
//    elements; a CTA loads whole blocks.
// Inside a pass every thread owns 16 elements of one column / block and runs
// the pass's stages in rounds of at most 4: load the 16 elements of its
// butterfly groups from shared memory into registers, apply the round's
// stages in registers, store back.  A 256-element column therefore costs two
// shared-memory round trips for its 8 stages.  All index arithmetic is fixed
// at compile time per ring dimension (template on log N).
// Values stay lazily reduced (forward [0, 4q), inverse [0, 2q)) until the
// last pass.  Launch: grid.y = row, grid.x = tile within the row.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "internal.h"
#include "kernels.h"
#include "modarith.cuh"

namespace mmfhe {

namespace {

constexpr int COLS = 16;        // columns per CTA in the strided pass

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

template <int LOGN>
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
    static constexpr int COLS_THREADS = COLS * TPC;
    static constexpr int TPR = T1 / 16;             // threads per block
    static constexpr int ROWS = (256 / TPR) < H ? (256 / TPR) : H;   // blocks per CTA
    static constexpr int RS = T1 + T1 / 16;         // padded block stride in shared memory
};

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
template <int LOGN, bool FWD>
__device__ __forceinline__ void cols_rounds(uint64_t *sm, uint64_t q, uint32_t pid, const Twiddles &tw) {
    using Gm = Geo<LOGN>;
    const int c = threadIdx.x % COLS, t = threadIdx.x / COLS;
    const uint64_t *W = (FWD ? tw.fw : tw.iw) + ((size_t)pid << LOGN);
    const uint64_t *Wp = (FWD ? tw.fw_sh : tw.iw_sh) + ((size_t)pid << LOGN);
    auto addr = [c](int h) { return h * COLS + c; };
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
template <int LOGN, bool FWD>
__device__ __forceinline__ void rows_rounds(uint64_t *sm, int hi0, uint64_t q, uint32_t pid, const Twiddles &tw) {
    using Gm = Geo<LOGN>;
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
template <int LOGN, bool FWD>
__global__ void __launch_bounds__(Geo<LOGN>::COLS_THREADS, 4)
    k_ntt_cols(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst, RowMap md, ModTab mt, Twiddles tw,
               const uint64_t *__restrict__ oscale, const uint64_t *__restrict__ oscale_sh) {
    using Gm = Geo<LOGN>;
    __shared__ uint64_t sm[Gm::H * COLS];
    uint32_t blk, p;
    row_decode(md, blockIdx.y, blk, p);
    const uint32_t pid = md.pid[p];
    const uint64_t *S = (FWD ? src + row_at(ms, blk, p, LOGN) : dst + row_at(md, blk, p, LOGN));
    uint64_t *D = dst + row_at(md, blk, p, LOGN);
    const int lo0 = blockIdx.x * COLS;
    const uint64_t q = mt.q[pid];
    MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) sm[e] = S[(size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS)];
    __syncthreads();
    cols_rounds<LOGN, FWD>(sm, q, pid, tw);
    __syncthreads();
    if (FWD) {
        MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) D[(size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS)] = sm[e];
    } else {
        const uint64_t ni = oscale ? oscale[pid] : tw.ninv[pid], nip = oscale ? oscale_sh[pid] : tw.ninv_sh[pid];
        MMFHE_TILE_LOOP(e, Gm::COLS_THREADS)
            D[(size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS)] = mm::mul_shoup(sm[e], ni, nip, q);
    }
}

// Contiguous pass. FWD: stages S1..logN-1 in place on dst, final reduction to
// [0, q); inverse: stages logN-1..S1 (reads src, writes dst).
template <int LOGN, bool FWD>
__global__ void __launch_bounds__(256, 4)
    k_ntt_rows(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst, RowMap md, ModTab mt, Twiddles tw) {
    using Gm = Geo<LOGN>;
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
        sm[rr * Gm::RS + l + (l >> 4)] = S[base + e];
    }
    __syncthreads();
    rows_rounds<LOGN, FWD>(sm, hi0, q, pid, tw);
    __syncthreads();
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int r2 = e / Gm::T1, l = e % Gm::T1;
        uint64_t v = sm[r2 * Gm::RS + l + (l >> 4)];
        D[base + e] = FWD ? mm::reduce_4q(v, q) : v;
    }
}

// Base-conversion staging of a strided-pass tile: element (h, lo0 + c) of the
// tile is sum_k X[k][h * T1 + lo0 + c] * F[k * fstride] reduced once by
// Montgomery (F in Montgomery form).  CENTERED adds c * negp with
// c = #{k : X[k] > P[k] / 2} (the centered correction of the ModDown conversion).
template <int LOGN, int NT, bool CENTERED = false>
__device__ __forceinline__ void conv_load(uint64_t *sm, const uint64_t *__restrict__ X, const uint64_t *__restrict__ F,
                                          int fstride, int lo0, uint64_t q, uint64_t qinv,
                                          const uint64_t *P = nullptr, uint64_t negp = 0) {
    using Gm = Geo<LOGN>;
    uint64_t f[NT], half[NT];
#pragma unroll
    for (int k = 0; k < NT; k++) {
        f[k] = F[(size_t)k * fstride];
        half[k] = CENTERED ? P[k] >> 1 : 0;
    }
    MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) {
        const size_t idx = (size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS);
        uint64_t hi = 0, lo = 0, neg = 0;
#pragma unroll
        for (int k = 0; k < NT; k++) {
            const uint64_t x = X[((size_t)k << LOGN) + idx];
            if (CENTERED) neg += x > half[k] ? 1u : 0u;
            mm::mac128(hi, lo, x, f[k]);
        }
        if (CENTERED) mm::mac128(hi, lo, neg, negp);
        sm[e] = mm::redc(hi, lo, q, qinv);
    }
}

// Fused ModUp strided pass: digit row (window blk, period row p = j * nre + t)
// starts from sum_u y[blk][j*alpha+u] * Qhat_{j,u} mod prime(t), accumulated
// as 128-bit products with the factor in Montgomery form and reduced once
// (alpha * q_src * q_t < q_t * 2^64 because alpha <= 8 and q_src < 2^61).
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::COLS_THREADS, 4)
    k_ntt_cols_modup(const uint64_t *__restrict__ y, int nl, int nre, int alpha, int j0, uint64_t *dst, RowMap md,
                     const uint64_t *__restrict__ m_mont, ModTab mt, Twiddles tw) {
    using Gm = Geo<LOGN>;
    __shared__ uint64_t sm[Gm::H * COLS];
    uint32_t blk, p;
    row_decode(md, blockIdx.y, blk, p);
    const uint32_t pid = md.pid[p];
    const int j = j0 + (int)p / nre, t = (int)p % nre;
    const int i0 = j * alpha, cnt = min(alpha, nl - i0);
    const uint64_t *Y = y + (((size_t)blk * nl + i0) << LOGN);
    uint64_t *D = dst + row_at(md, blk, p, LOGN);
    const int lo0 = blockIdx.x * COLS;
    const uint64_t q = mt.q[pid], qinv = mt.qinv[pid];
    const uint64_t *F = m_mont + (size_t)j * MAX_ALPHA * MAXROWMAP + t;
    switch (cnt) {   // uniform per CTA: the term loop is unrolled for the digit's prime count
    case 1: conv_load<LOGN, 1>(sm, Y, F, MAXROWMAP, lo0, q, qinv); break;
    case 2: conv_load<LOGN, 2>(sm, Y, F, MAXROWMAP, lo0, q, qinv); break;
    case 3: conv_load<LOGN, 3>(sm, Y, F, MAXROWMAP, lo0, q, qinv); break;
    case 4: conv_load<LOGN, 4>(sm, Y, F, MAXROWMAP, lo0, q, qinv); break;
    case 5: conv_load<LOGN, 5>(sm, Y, F, MAXROWMAP, lo0, q, qinv); break;
    case 6: conv_load<LOGN, 6>(sm, Y, F, MAXROWMAP, lo0, q, qinv); break;
    case 7: conv_load<LOGN, 7>(sm, Y, F, MAXROWMAP, lo0, q, qinv); break;
    default: conv_load<LOGN, 8>(sm, Y, F, MAXROWMAP, lo0, q, qinv); break;
    }
    __syncthreads();
    cols_rounds<LOGN, true>(sm, q, pid, tw);
    __syncthreads();
    MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) D[(size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS)] = sm[e];
}

// Fused ModDown strided pass: row (blk = window * 2 + h, p = i) starts from the
// centered conversion v_i = sum_k z_k Phat_k + c (-P) mod q_i, c = #{k : z_k > p_k / 2},
// in one Montgomery reduction (K (p_max - 1)(q - 1) + K (q - 1) < q 2^64 for K <= 8).
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::COLS_THREADS, 4)
    k_ntt_cols_moddown(const uint64_t *__restrict__ z, int K, int pid_p0, uint64_t *dst, RowMap md,
                       const uint64_t *__restrict__ phat_mont, const uint64_t *__restrict__ negp_mont, ModTab mt,
                       Twiddles tw) {
    using Gm = Geo<LOGN>;
    __shared__ uint64_t sm[Gm::H * COLS];
    uint32_t blk, p;
    row_decode(md, blockIdx.y, blk, p);
    const uint32_t pid = md.pid[p];
    const uint64_t *Z = z + (((size_t)blk * K) << LOGN);
    uint64_t *D = dst + row_at(md, blk, p, LOGN);
    const int lo0 = blockIdx.x * COLS;
    const uint64_t q = mt.q[pid], qinv = mt.qinv[pid];
    const uint64_t *F = phat_mont + pid;
    const uint64_t np = negp_mont[pid];
    const uint64_t *Hp = mt.q + pid_p0;
    switch (K) {   // uniform: the term loop is unrolled for the number of special primes
    case 1: conv_load<LOGN, 1, true>(sm, Z, F, MMFHE_MAX_Q, lo0, q, qinv, Hp, np); break;
    case 2: conv_load<LOGN, 2, true>(sm, Z, F, MMFHE_MAX_Q, lo0, q, qinv, Hp, np); break;
    case 3: conv_load<LOGN, 3, true>(sm, Z, F, MMFHE_MAX_Q, lo0, q, qinv, Hp, np); break;
    case 4: conv_load<LOGN, 4, true>(sm, Z, F, MMFHE_MAX_Q, lo0, q, qinv, Hp, np); break;
    case 5: conv_load<LOGN, 5, true>(sm, Z, F, MMFHE_MAX_Q, lo0, q, qinv, Hp, np); break;
    case 6: conv_load<LOGN, 6, true>(sm, Z, F, MMFHE_MAX_Q, lo0, q, qinv, Hp, np); break;
    case 7: conv_load<LOGN, 7, true>(sm, Z, F, MMFHE_MAX_Q, lo0, q, qinv, Hp, np); break;
    default: conv_load<LOGN, 8, true>(sm, Z, F, MMFHE_MAX_Q, lo0, q, qinv, Hp, np); break;
    }
    __syncthreads();
    cols_rounds<LOGN, true>(sm, q, pid, tw);
    __syncthreads();
    MMFHE_TILE_LOOP(e, Gm::COLS_THREADS) D[(size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS)] = sm[e];
}

// Fused ModDown contiguous pass: forward stages on v (rows blk = window * 2 + h,
// p = i, in place on vtmp) and the combine
//   out = (u - v) P^-1 + add_h[perm(x)] + plus  (mod q_i).
template <int LOGN>
__global__ void __launch_bounds__(256, 4)
    k_ntt_rows_combine(const uint64_t *__restrict__ v, RowMap mv, CombineArgs a, int nre,
                       const uint64_t *__restrict__ Pinv, const uint64_t *__restrict__ Pinv_sh, ModTab mt,
                       Twiddles tw) {
    using Gm = Geo<LOGN>;
    __shared__ uint64_t sm[Gm::ROWS * Gm::RS];
    uint32_t blk, p;
    row_decode(mv, blockIdx.y, blk, p);
    const uint32_t pid = mv.pid[p];
    const int nl = (int)mv.period;
    const uint64_t *S = v + row_at(mv, blk, p, LOGN);
    const int hi0 = blockIdx.x * Gm::ROWS;
    const uint64_t q = mt.q[pid];
    const size_t base = (size_t)hi0 * Gm::T1;
    const uint64_t *U = a.u + (((size_t)blk * nre + p) << LOGN);
    const uint64_t *A = (blk & 1) ? a.add1 : a.add0;
    if (A) A += (size_t)(blk >> 1) * a.add_stride + ((size_t)p << LOGN);
    const uint64_t *Pl = a.plus ? a.plus + (((size_t)blk * nl + p) << LOGN) : nullptr;
    if (threadIdx.x == 0) {
        // the epilogue's contiguous operands travel to L2 while the stages run
        constexpr uint32_t seg = Gm::ROWS * Gm::T1 * 8;
        l2_prefetch(U + base, seg);
        if (Pl) l2_prefetch(Pl + base, seg);
        if (A && a.galois == 1) l2_prefetch(A + base, seg);
    }
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int rr = e / Gm::T1, l = e % Gm::T1;
        sm[rr * Gm::RS + l + (l >> 4)] = S[base + e];
    }
    __syncthreads();
    rows_rounds<LOGN, true>(sm, hi0, q, pid, tw);
    __syncthreads();
    const uint64_t pi = Pinv[pid], pis = Pinv_sh[pid];
    uint64_t *O = a.out + (((size_t)blk * nl + p) << LOGN);
    MMFHE_TILE_LOOP(e, Gm::ROWS * Gm::TPR) {
        int r2 = e / Gm::T1, l = e % Gm::T1;
        const uint32_t x = (uint32_t)(base + e);
        const uint64_t vv = mm::reduce_4q(sm[r2 * Gm::RS + l + (l >> 4)], q);
        uint64_t res = mm::mul_shoup(mm::sub_mod(U[x], vv, q), pi, pis, q);
        if (A) res = mm::add_mod(res, A[a.galois == 1 ? x : mm::galois_perm(x, a.galois, LOGN)], q);
        if (Pl) res = mm::add_mod(res, Pl[x], q);
        O[x] = res;
    }
}

__global__ void k_copy_rows(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst, RowMap md, int logn) {
    uint32_t blk, p;
    row_decode(md, blockIdx.y, blk, p);
    const uint64_t *S = src + row_at(ms, blk, p, logn);
    uint64_t *D = dst + row_at(md, blk, p, logn);
    const uint32_t n = 1u << logn;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) D[i] = S[i];
}

}  // namespace

RowMap make_map(uint32_t period, uint32_t block_stride, const std::vector<int> &pids) {
    if (period == 0 || period > (uint32_t)MAXROWMAP || pids.size() != period) throw Error(MMFHE_ERR_BAD_ARG, "row map too large");
    RowMap m{};
    m.period = period;
    m.block_stride = block_stride;
    for (uint32_t i = 0; i < period; i++) m.pid[i] = pids[i] < 0 ? SKIP : (uint8_t)pids[i];
    return m;
}

// Fill the active-row list of md (non-SKIP period rows) into both maps.
static uint32_t set_active(RowMap &ms, RowMap &md) {
    if (ms.period != md.period) throw Error(MMFHE_ERR_BAD_ARG, "row maps differ in period");
    uint32_t n = 0;
    for (uint32_t p = 0; p < md.period; p++)
        if (md.pid[p] != SKIP) md.act[n++] = (uint8_t)p;
    md.nact = n;
    for (uint32_t k = 0; k < n; k++) ms.act[k] = md.act[k];
    ms.nact = n;
    return n;
}

static cudaEvent_t next_event(Context &c) {
    if (c.event_next == c.event_pool.size()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c.event_pool.push_back(e);
    }
    return c.event_pool[c.event_next++];
}

void kernel_begin(Context &c, cudaStream_t st) {
    if (!c.profiling) return;
    cudaEvent_t e = next_event(c);
    CK(cudaEventRecord(e, st));
    c.prof.push_back(Context::ProfRec{nullptr, e, nullptr, 0.0, 0.0});
}

void kernel_end(Context &c, const char *name, dim3 g, dim3 b, double bytes, cudaStream_t st, double butterflies) {
    c.launches++;
    if (c.tracing) {
        char buf[160];
        snprintf(buf, sizeof buf, "%s g(%u,%u,%u) b(%u,%u,%u)", name, g.x, g.y, g.z, b.x, b.y, b.z);
        c.trace.emplace_back(buf);
    }
    if (c.profiling && !c.prof.empty()) {
        Context::ProfRec &r = c.prof.back();
        r.name = name;
        r.bytes = bytes;
        r.butterflies = butterflies;
        r.stop = next_event(c);
        CK(cudaEventRecord(r.stop, st));
    }
}

#define MMFHE_LOGN_DISPATCH(logn, CALL)                                              \
    switch (logn) {                                                                  \
    case 10: CALL(10); break;                                                        \
    case 11: CALL(11); break;                                                        \
    case 12: CALL(12); break;                                                        \
    case 13: CALL(13); break;                                                        \
    case 14: CALL(14); break;                                                        \
    case 15: CALL(15); break;                                                        \
    case 16: CALL(16); break;                                                        \
    default: throw Error(MMFHE_ERR_BAD_ARG, "unsupported ring dimension");          \
    }

// Butterflies of one pass over nr rows: N/2 per stage.
template <int LOGN>
static double bf_cols(size_t nr) { return (double)nr * (double)(1u << (LOGN - 1)) * Geo<LOGN>::S1; }
template <int LOGN>
static double bf_rows(size_t nr) { return (double)nr * (double)(1u << (LOGN - 1)) * Geo<LOGN>::LOGT; }

template <int LOGN>
static void ntt_launch_t(Context &c, const uint64_t *sb, RowMap ms, uint64_t *db, RowMap md, size_t nr, bool inverse,
                         double bytes, const uint64_t *os, const uint64_t *os_sh, cudaStream_t st) {
    using Gm = Geo<LOGN>;
    dim3 gc(Gm::T1 / COLS, (unsigned)nr), bc(Gm::COLS_THREADS);
    dim3 gr(Gm::H / Gm::ROWS, (unsigned)nr), br(Gm::ROWS * Gm::TPR);
    const double bfc = bf_cols<LOGN>(nr), bfr = bf_rows<LOGN>(nr);
    if (!inverse) {
        kernel_begin(c, st);
        k_ntt_cols<LOGN, true><<<gc, bc, 0, st>>>(sb, ms, db, md, c.mods, c.tw, nullptr, nullptr);
        kernel_end(c, "ntt_fwd_cols", gc, bc, bytes, st, bfc);
        kernel_begin(c, st);
        k_ntt_rows<LOGN, true><<<gr, br, 0, st>>>(db, md, db, md, c.mods, c.tw);
        kernel_end(c, "ntt_fwd_rows", gr, br, bytes, st, bfr);
    } else {
        kernel_begin(c, st);
        k_ntt_rows<LOGN, false><<<gr, br, 0, st>>>(sb, ms, db, md, c.mods, c.tw);
        kernel_end(c, "ntt_inv_rows", gr, br, bytes, st, bfr);
        kernel_begin(c, st);
        k_ntt_cols<LOGN, false><<<gc, bc, 0, st>>>(db, md, db, md, c.mods, c.tw, os, os_sh);
        kernel_end(c, "ntt_inv_cols", gc, bc, bytes, st, bfc);
    }
}

void launch_ntt(Context &c, const RowsView &src, const RowsView &dst, bool inverse, cudaStream_t st,
                const uint64_t *oscale, const uint64_t *oscale_sh) {
    if (src.rows == 0) return;
    RowMap ms = src.map, md = dst.map;
    if (src.rows % ms.period) throw Error(MMFHE_ERR_BAD_ARG, "row count is not a whole number of blocks");
    const uint32_t nact = set_active(ms, md);
    if (nact == 0) return;
    const size_t blocks = src.rows / ms.period;
    // grid.y is limited to 65535 rows per launch: split on block boundaries
    const size_t chunk = 65535 / nact;
    for (size_t b0 = 0; b0 < blocks; b0 += chunk) {
        const size_t nb = std::min(chunk, blocks - b0);
        const uint64_t *sb = src.base + ((b0 * ms.block_stride) << c.logn);
        uint64_t *db = dst.base + ((b0 * md.block_stride) << c.logn);
        const size_t nr = nb * nact;
        const double bytes = 2.0 * (double)nr * c.n * 8;   // each pass reads and writes every transformed row once
#define MMFHE_NTT_CALL(L) ntt_launch_t<L>(c, sb, ms, db, md, nr, inverse, bytes, oscale, oscale_sh, st)
        MMFHE_LOGN_DISPATCH(c.logn, MMFHE_NTT_CALL)
#undef MMFHE_NTT_CALL
    }
    CK(cudaGetLastError());
}

void launch_copy_rows(Context &c, const RowsView &src, const RowsView &dst, cudaStream_t st) {
    if (src.rows == 0) return;
    RowMap ms = src.map, md = dst.map;
    if (src.rows % ms.period) throw Error(MMFHE_ERR_BAD_ARG, "row count is not a whole number of blocks");
    const uint32_t nact = set_active(ms, md);
    if (nact == 0) return;
    const size_t blocks = src.rows / ms.period;
    const size_t chunk = 65535 / nact;
    for (size_t b0 = 0; b0 < blocks; b0 += chunk) {
        const size_t nb = std::min(chunk, blocks - b0);
        const uint64_t *sb = src.base + ((b0 * ms.block_stride) << c.logn);
        uint64_t *db = dst.base + ((b0 * md.block_stride) << c.logn);
        const size_t nr = nb * nact;
        dim3 g(std::max(1u, c.n / 1024), (unsigned)nr), b(256);
        kernel_begin(c, st);
        k_copy_rows<<<g, b, 0, st>>>(sb, ms, db, md, c.logn);
        kernel_end(c, "copy_rows", g, b, 2.0 * (double)nr * c.n * 8, st);
    }
    CK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// fused key-switch NTTs
// ---------------------------------------------------------------------------
template <int LOGN>
static void modup_launch_t(Context &c, uint64_t *digits, const uint64_t *y, const RowMap &md, size_t nr, int nl,
                           int nre, int j0, const uint64_t *m_mont, double bytes_cols, double bytes_rows,
                           cudaStream_t st) {
    using Gm = Geo<LOGN>;
    dim3 gc(Gm::T1 / COLS, (unsigned)nr), bc(Gm::COLS_THREADS);
    dim3 gr(Gm::H / Gm::ROWS, (unsigned)nr), br(Gm::ROWS * Gm::TPR);
    kernel_begin(c, st);
    k_ntt_cols_modup<LOGN><<<gc, bc, 0, st>>>(y, nl, nre, c.alpha, j0, digits, md, m_mont, c.mods, c.tw);
    kernel_end(c, "ntt_modup_cols", gc, bc, bytes_cols, st, bf_cols<LOGN>(nr));
    kernel_begin(c, st);
    k_ntt_rows<LOGN, true><<<gr, br, 0, st>>>(digits, md, digits, md, c.mods, c.tw);
    kernel_end(c, "ntt_fwd_rows", gr, br, bytes_rows, st, bf_rows<LOGN>(nr));
}

void launch_modup_ntt(Context &c, uint64_t *digits, const uint64_t *y, int B, int level, cudaStream_t st) {
    const LevelConsts &lc = c.lv[level];
    const int nl = level + 1, nre = nl + c.num_p, beta = lc.beta;
    if (B == 0) return;
    // digits per launch: a launch's period (digits x nre rows) fits one row map
    const int per = std::max(1, std::min(beta, MAXROWMAP / nre));
    for (int j0 = 0; j0 < beta; j0 += per) {
        const int nj = std::min(per, beta - j0);
        std::vector<int> pids(nj * nre);
        for (int jj = 0; jj < nj; jj++) {
            const auto &D = lc.digits[j0 + jj];
            for (int t = 0; t < nre; t++) {
                const bool own = t >= D.front() && t <= D.back();
                pids[jj * nre + t] = own ? -1 : (t < nl ? t : c.num_q + (t - nl));
            }
        }
        RowMap md = make_map(nj * nre, beta * nre, pids), ms = md;
        const uint32_t nact = set_active(ms, md);
        uint64_t *dbase = digits + (((size_t)j0 * nre) << c.logn);
        const size_t chunk = 65535 / nact;
        for (size_t b0 = 0; b0 < (size_t)B; b0 += chunk) {
            const size_t nb = std::min(chunk, (size_t)B - b0);
            const size_t nr = nb * nact;
            uint64_t *db = dbase + ((b0 * beta * nre) << c.logn);
            const uint64_t *yb = y + ((b0 * nl) << c.logn);
            const double row = (double)c.n * 8;
            // reads each window's y rows of the launched digits once, writes every converted row;
            // the contiguous pass reads and writes every row
            int src_rows = 0;
            for (int jj = 0; jj < nj; jj++) src_rows += (int)lc.digits[j0 + jj].size();
            const double bc_ = row * ((double)nr + (double)nb * src_rows), br_ = 2.0 * row * (double)nr;
#define MMFHE_MODUP_CALL(L) modup_launch_t<L>(c, db, yb, md, nr, nl, nre, j0, lc.d_up_mm, bc_, br_, st)
            MMFHE_LOGN_DISPATCH(c.logn, MMFHE_MODUP_CALL)
#undef MMFHE_MODUP_CALL
        }
    }
    CK(cudaGetLastError());
}

template <int LOGN>
static void moddown_launch_t(Context &c, uint64_t *vtmp, const uint64_t *z, const RowMap &mv, size_t nr,
                             const CombineArgs &a, int nre, double bytes_cols, double bytes_rows, cudaStream_t st) {
    using Gm = Geo<LOGN>;
    dim3 gc(Gm::T1 / COLS, (unsigned)nr), bc(Gm::COLS_THREADS);
    dim3 gr(Gm::H / Gm::ROWS, (unsigned)nr), br(Gm::ROWS * Gm::TPR);
    kernel_begin(c, st);
    k_ntt_cols_moddown<LOGN><<<gc, bc, 0, st>>>(z, c.num_p, c.num_q, vtmp, mv, c.d_dn_phat_mont, c.d_dn_negp_mont,
                                                c.mods, c.tw);
    kernel_end(c, "ntt_moddown_cols", gc, bc, bytes_cols, st, bf_cols<LOGN>(nr));
    kernel_begin(c, st);
    k_ntt_rows_combine<LOGN><<<gr, br, 0, st>>>(vtmp, mv, a, nre, c.d_dn_Pinv, c.d_dn_Pinv_sh, c.mods, c.tw);
    kernel_end(c, "ntt_combine_rows", gr, br, bytes_rows, st, bf_rows<LOGN>(nr));
}

void launch_moddown_ntt(Context &c, uint64_t *vtmp, const uint64_t *z, const CombineArgs &a, int B, int level,
                        cudaStream_t st) {
    const int nl = level + 1, nre = nl + c.num_p, K = c.num_p;
    if (B == 0) return;
    std::vector<int> pids(nl);
    for (int i = 0; i < nl; i++) pids[i] = i;
    RowMap mv = make_map(nl, nl, pids), ms = mv;
    const uint32_t nact = set_active(ms, mv);
    const size_t blocks = (size_t)B * 2;
    const size_t chunk = 65535 / nact;
    for (size_t b0 = 0; b0 < blocks; b0 += chunk) {
        // chunks hold whole windows, so the (window, h) parity of a block is kept
        const size_t nb = std::min(chunk & ~(size_t)1, blocks - b0);
        const size_t nr = nb * nact;
        CombineArgs ab = a;
        ab.out = a.out + ((b0 * nl) << c.logn);
        ab.u = a.u + ((b0 * nre) << c.logn);
        if (ab.add0) ab.add0 += (b0 / 2) * a.add_stride;
        if (ab.add1) ab.add1 += (b0 / 2) * a.add_stride;
        if (ab.plus) ab.plus += (b0 * nl) << c.logn;
        const double row = (double)c.n * 8;
        const double bc_ = row * ((double)nr + (double)nb * K);
        const double br_ = row * ((double)nr * (3 + (ab.plus ? 1 : 0)) + (ab.add0 ? nr / 2.0 : 0) + (ab.add1 ? nr / 2.0 : 0));
#define MMFHE_MODDOWN_CALL(L)                                                                                   \
    moddown_launch_t<L>(c, vtmp + ((b0 * nl) << c.logn), z + ((b0 * K) << c.logn), mv, nr, ab, nre, bc_, br_, st)
        MMFHE_LOGN_DISPATCH(c.logn, MMFHE_MODDOWN_CALL)
#undef MMFHE_MODDOWN_CALL
    }
    CK(cudaGetLastError());
}

}  // namespace mmfhe
