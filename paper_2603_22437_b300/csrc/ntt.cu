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
#include "modarith.cuh"

namespace mmfhe {

namespace {

constexpr int COLS = 16;        // columns per CTA in the strided pass

__device__ __forceinline__ size_t row_offset(const RowMap &m, uint32_t r, int logn) {
    return ((size_t)(r / m.period) * m.block_stride + (r % m.period)) << logn;
}

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
#pragma unroll
    for (int uu = 0; uu < R; uu++) {
        const int u = FWD ? uu : R - 1 - uu;
        const int dist = 1 << (R - 1 - u);
#pragma unroll
        for (int g = 0; g < G; g++) {
#pragma unroll
            for (int j = 0; j < M; j++) {
                if (j & dist) continue;
                const int widx = twi(A + u, elem_index<LOG, A, R>(t, g, j));
                const uint64_t w = __ldg(W + widx), wp = __ldg(Wp + widx);
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

// Strided pass. FWD: stages 0..S1-1 (reads src, writes dst); inverse: stages
// S1-1..0 in place on dst, then the N^-1 factor.
template <int LOGN, bool FWD>
__global__ void __launch_bounds__(Geo<LOGN>::COLS_THREADS)
    k_ntt_cols(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst, RowMap md, ModTab mt, Twiddles tw) {
    using Gm = Geo<LOGN>;
    __shared__ uint64_t sm[Gm::H * COLS];
    const uint32_t r = blockIdx.y;
    const uint8_t pid = md.pid[r % md.period];
    if (pid == SKIP) return;
    const uint64_t *S = (FWD ? src + row_offset(ms, r, LOGN) : dst + row_offset(md, r, LOGN));
    uint64_t *D = dst + row_offset(md, r, LOGN);
    const int lo0 = blockIdx.x * COLS;
    const uint64_t q = mt.q[pid];
    for (int e = threadIdx.x; e < Gm::H * COLS; e += blockDim.x) sm[e] = S[(size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS)];
    __syncthreads();
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
    __syncthreads();
    if (FWD) {
        for (int e = threadIdx.x; e < Gm::H * COLS; e += blockDim.x) D[(size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS)] = sm[e];
    } else {
        const uint64_t ni = tw.ninv[pid], nip = tw.ninv_sh[pid];
        for (int e = threadIdx.x; e < Gm::H * COLS; e += blockDim.x)
            D[(size_t)(e / COLS) * Gm::T1 + lo0 + (e % COLS)] = mm::mul_shoup(sm[e], ni, nip, q);
    }
}

// Contiguous pass. FWD: stages S1..logN-1 in place on dst, final reduction to
// [0, q); inverse: stages logN-1..S1 (reads src, writes dst).
template <int LOGN, bool FWD>
__global__ void __launch_bounds__(256)
    k_ntt_rows(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst, RowMap md, ModTab mt, Twiddles tw) {
    using Gm = Geo<LOGN>;
    __shared__ uint64_t sm[Gm::ROWS * Gm::RS];
    const uint32_t r = blockIdx.y;
    const uint8_t pid = md.pid[r % md.period];
    if (pid == SKIP) return;
    const uint64_t *S = (FWD ? dst + row_offset(md, r, LOGN) : src + row_offset(ms, r, LOGN));
    uint64_t *D = dst + row_offset(md, r, LOGN);
    const int hi0 = blockIdx.x * Gm::ROWS;
    const uint64_t q = mt.q[pid];
    const size_t base = (size_t)hi0 * Gm::T1;
    for (int e = threadIdx.x; e < Gm::ROWS * Gm::T1; e += blockDim.x) {
        int rr = e / Gm::T1, l = e % Gm::T1;
        sm[rr * Gm::RS + l + (l >> 4)] = S[base + e];
    }
    __syncthreads();
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
    __syncthreads();
    for (int e = threadIdx.x; e < Gm::ROWS * Gm::T1; e += blockDim.x) {
        int r2 = e / Gm::T1, l = e % Gm::T1;
        uint64_t v = sm[r2 * Gm::RS + l + (l >> 4)];
        D[base + e] = FWD ? mm::reduce_4q(v, q) : v;
    }
}

__global__ void k_copy_rows(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst, RowMap md, int logn) {
    const uint32_t r = blockIdx.y;
    if (md.pid[r % md.period] == SKIP) return;
    const uint64_t *S = src + row_offset(ms, r, logn);
    uint64_t *D = dst + row_offset(md, r, logn);
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
    c.prof.push_back(Context::ProfRec{nullptr, e, nullptr, 0.0});
}

void kernel_end(Context &c, const char *name, dim3 g, dim3 b, double bytes, cudaStream_t st) {
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
        r.stop = next_event(c);
        CK(cudaEventRecord(r.stop, st));
    }
}

template <int LOGN>
static void ntt_launch_t(Context &c, const uint64_t *sb, RowMap ms, uint64_t *db, RowMap md, size_t nr, bool inverse,
                         double bytes, cudaStream_t st) {
    using Gm = Geo<LOGN>;
    dim3 gc(Gm::T1 / COLS, (unsigned)nr), bc(Gm::COLS_THREADS);
    dim3 gr(Gm::H / Gm::ROWS, (unsigned)nr), br(Gm::ROWS * Gm::TPR);
    if (!inverse) {
        kernel_begin(c, st);
        k_ntt_cols<LOGN, true><<<gc, bc, 0, st>>>(sb, ms, db, md, c.mods, c.tw);
        kernel_end(c, "ntt_fwd_cols", gc, bc, bytes, st);
        kernel_begin(c, st);
        k_ntt_rows<LOGN, true><<<gr, br, 0, st>>>(db, md, db, md, c.mods, c.tw);
        kernel_end(c, "ntt_fwd_rows", gr, br, bytes, st);
    } else {
        kernel_begin(c, st);
        k_ntt_rows<LOGN, false><<<gr, br, 0, st>>>(sb, ms, db, md, c.mods, c.tw);
        kernel_end(c, "ntt_inv_rows", gr, br, bytes, st);
        kernel_begin(c, st);
        k_ntt_cols<LOGN, false><<<gc, bc, 0, st>>>(db, md, db, md, c.mods, c.tw);
        kernel_end(c, "ntt_inv_cols", gc, bc, bytes, st);
    }
}

void launch_ntt(Context &c, const RowsView &src, const RowsView &dst, bool inverse, cudaStream_t st) {
    if (src.rows == 0) return;
    // grid.y is limited to 65535 rows per launch: split on block boundaries
    const size_t chunk = (65535 / src.map.period) * src.map.period;
    for (size_t r0 = 0; r0 < src.rows; r0 += chunk) {
        size_t nr = std::min<size_t>(chunk, src.rows - r0);
        RowMap ms = src.map, md = dst.map;
        size_t blocks0 = r0 / ms.period;
        const uint64_t *sb = src.base + ((blocks0 * ms.block_stride) << c.logn);
        uint64_t *db = dst.base + ((blocks0 * md.block_stride) << c.logn);
        size_t live = 0;   // rows actually transformed (skipped rows move no data)
        for (size_t r = 0; r < nr; r++) live += md.pid[r % md.period] != SKIP;
        const double bytes = 2.0 * (double)live * c.n * 8;   // each pass reads and writes every live row once
        switch (c.logn) {
        case 10: ntt_launch_t<10>(c, sb, ms, db, md, nr, inverse, bytes, st); break;
        case 11: ntt_launch_t<11>(c, sb, ms, db, md, nr, inverse, bytes, st); break;
        case 12: ntt_launch_t<12>(c, sb, ms, db, md, nr, inverse, bytes, st); break;
        case 13: ntt_launch_t<13>(c, sb, ms, db, md, nr, inverse, bytes, st); break;
        case 14: ntt_launch_t<14>(c, sb, ms, db, md, nr, inverse, bytes, st); break;
        case 15: ntt_launch_t<15>(c, sb, ms, db, md, nr, inverse, bytes, st); break;
        case 16: ntt_launch_t<16>(c, sb, ms, db, md, nr, inverse, bytes, st); break;
        default: throw Error(MMFHE_ERR_BAD_ARG, "unsupported ring dimension");
        }
    }
    CK(cudaGetLastError());
}

void launch_copy_rows(Context &c, const RowsView &src, const RowsView &dst, cudaStream_t st) {
    if (src.rows == 0) return;
    const size_t chunk = (65535 / src.map.period) * src.map.period;
    for (size_t r0 = 0; r0 < src.rows; r0 += chunk) {
        size_t nr = std::min<size_t>(chunk, src.rows - r0);
        size_t blocks0 = r0 / src.map.period;
        const uint64_t *sb = src.base + ((blocks0 * src.map.block_stride) << c.logn);
        uint64_t *db = dst.base + ((blocks0 * dst.map.block_stride) << c.logn);
        dim3 g(std::max(1u, c.n / 1024), (unsigned)nr), b(256);
        kernel_begin(c, st);
        k_copy_rows<<<g, b, 0, st>>>(sb, src.map, db, dst.map, c.logn);
        kernel_end(c, "copy_rows", g, b, 2.0 * (double)nr * c.n * 8, st);
    }
    CK(cudaGetLastError());
}

}  // namespace mmfhe
