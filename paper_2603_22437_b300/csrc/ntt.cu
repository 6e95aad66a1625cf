// Batched negacyclic NTT / inverse NTT over 64-bit RNS limbs.
//
// Merged (twisted) Cooley-Tukey forward transform with bit-reversed output:
// row j of the result holds a(psi^(2 brv(j) + 1)); the Gentleman-Sande inverse
// takes that order back to coefficients and multiplies by N^-1.  Stage s
// (m = 2^s butterfly groups, distance t = N / 2^(s+1)) uses twiddle
// psi^brv(m + i) for group i.
//
// Two passes per transform, each staged through shared memory:
//  * "cols": stages 0 .. s1-1 only couple elements with equal index mod
//    T1 = N / 2^s1, so each CTA loads `cols` adjacent columns of H = 2^s1
//    elements at stride T1 (128-byte row segments) and runs s1 stages;
//  * "rows": stages s1 .. logN-1 stay inside contiguous blocks of T1
//    elements, so each CTA loads whole blocks and runs the remaining stages.
// Values stay lazily reduced (forward [0, 4q), inverse [0, 2q)) until the
// last pass.  Launch: grid.y = row, grid.x = tile within the row.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "internal.h"
#include "modarith.cuh"

namespace mmfhe {

namespace {

constexpr int NTT_THREADS = 256;
constexpr int TILE_WORDS = 4096;   // 32 KiB of shared memory per CTA

struct NttShape {
    int logn, s1, T1, H, cols, rows_per_cta;
};

NttShape shape_for(int logn) {
    NttShape s;
    s.logn = logn;
    s.s1 = (logn + 1) / 2;
    s.T1 = 1 << (logn - s.s1);
    s.H = 1 << s.s1;
    s.cols = std::min(16, s.T1);
    s.rows_per_cta = std::min(s.H, TILE_WORDS / s.T1);
    return s;
}

__device__ __forceinline__ size_t row_offset(const RowMap &m, uint32_t r, int logn) {
    return ((size_t)(r / m.period) * m.block_stride + (r % m.period)) << logn;
}

__global__ void __launch_bounds__(NTT_THREADS) k_ntt_fwd_cols(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst,
                                                              RowMap md, ModTab mt, Twiddles tw, NttShape sh) {
    extern __shared__ uint64_t sm[];
    const uint32_t r = blockIdx.y;
    const uint8_t pid = md.pid[r % md.period];
    if (pid == SKIP) return;
    const uint64_t *S = src + row_offset(ms, r, sh.logn);
    uint64_t *D = dst + row_offset(md, r, sh.logn);
    const int cols = sh.cols, T1 = sh.T1, H = sh.H, s1 = sh.s1;
    const int lo0 = blockIdx.x * cols;
    const uint64_t q = mt.q[pid];
    for (int e = threadIdx.x; e < H * cols; e += blockDim.x) {
        int h = e / cols, c = e - h * cols;
        sm[e] = S[(size_t)h * T1 + lo0 + c];
    }
    __syncthreads();
    const uint64_t *W = tw.fw + ((size_t)pid << sh.logn);
    const uint64_t *Wp = tw.fw_sh + ((size_t)pid << sh.logn);
    for (int s = 0; s < s1; s++) {
        const int ltt = s1 - s - 1;
        for (int e = threadIdx.x; e < (H >> 1) * cols; e += blockDim.x) {
            int hb = e / cols, c = e - hb * cols;
            int h = ((hb >> ltt) << (ltt + 1)) + (hb & ((1 << ltt) - 1));
            int widx = (1 << s) + (h >> (s1 - s));
            uint64_t X = sm[h * cols + c], Y = sm[(h + (1 << ltt)) * cols + c];
            mm::ct_butterfly(X, Y, W[widx], Wp[widx], q);
            sm[h * cols + c] = X;
            sm[(h + (1 << ltt)) * cols + c] = Y;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < H * cols; e += blockDim.x) {
        int h = e / cols, c = e - h * cols;
        D[(size_t)h * T1 + lo0 + c] = sm[e];
    }
}

__global__ void __launch_bounds__(NTT_THREADS) k_ntt_fwd_rows(uint64_t *dst, RowMap md, ModTab mt, Twiddles tw,
                                                              NttShape sh) {
    extern __shared__ uint64_t sm[];
    const uint32_t r = blockIdx.y;
    const uint8_t pid = md.pid[r % md.period];
    if (pid == SKIP) return;
    uint64_t *D = dst + row_offset(md, r, sh.logn);
    const int T1 = sh.T1, R = sh.rows_per_cta, s1 = sh.s1, logn = sh.logn;
    const int hi0 = blockIdx.x * R;
    uint64_t *blk = D + (size_t)hi0 * T1;
    const uint64_t q = mt.q[pid];
    for (int e = threadIdx.x; e < R * T1; e += blockDim.x) sm[e] = blk[e];
    __syncthreads();
    const uint64_t *W = tw.fw + ((size_t)pid << logn);
    const uint64_t *Wp = tw.fw_sh + ((size_t)pid << logn);
    const int half = T1 >> 1;
    for (int s = s1; s < logn; s++) {
        const int lt = logn - s - 1;   // t = 2^lt
        for (int e = threadIdx.x; e < R * half; e += blockDim.x) {
            int row = e / half, k = e - row * half;
            int l = ((k >> lt) << (lt + 1)) + (k & ((1 << lt) - 1));
            int hi = hi0 + row;
            int widx = (1 << s) + (hi << (s - s1)) + (l >> (logn - s));
            uint64_t *x = sm + row * T1;
            uint64_t X = x[l], Y = x[l + (1 << lt)];
            mm::ct_butterfly(X, Y, W[widx], Wp[widx], q);
            x[l] = X;
            x[l + (1 << lt)] = Y;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < R * T1; e += blockDim.x) blk[e] = mm::reduce_4q(sm[e], q);
}

__global__ void __launch_bounds__(NTT_THREADS) k_ntt_inv_rows(const uint64_t *__restrict__ src, RowMap ms, uint64_t *dst,
                                                              RowMap md, ModTab mt, Twiddles tw, NttShape sh) {
    extern __shared__ uint64_t sm[];
    const uint32_t r = blockIdx.y;
    const uint8_t pid = md.pid[r % md.period];
    if (pid == SKIP) return;
    const uint64_t *S = src + row_offset(ms, r, sh.logn);
    uint64_t *D = dst + row_offset(md, r, sh.logn);
    const int T1 = sh.T1, R = sh.rows_per_cta, s1 = sh.s1, logn = sh.logn;
    const int hi0 = blockIdx.x * R;
    const uint64_t q = mt.q[pid];
    for (int e = threadIdx.x; e < R * T1; e += blockDim.x) sm[e] = S[(size_t)hi0 * T1 + e];
    __syncthreads();
    const uint64_t *W = tw.iw + ((size_t)pid << logn);
    const uint64_t *Wp = tw.iw_sh + ((size_t)pid << logn);
    const int half = T1 >> 1;
    for (int s = logn - 1; s >= s1; s--) {
        const int lt = logn - s - 1;
        for (int e = threadIdx.x; e < R * half; e += blockDim.x) {
            int row = e / half, k = e - row * half;
            int l = ((k >> lt) << (lt + 1)) + (k & ((1 << lt) - 1));
            int hi = hi0 + row;
            int widx = (1 << s) + (hi << (s - s1)) + (l >> (logn - s));
            uint64_t *x = sm + row * T1;
            uint64_t X = x[l], Y = x[l + (1 << lt)];
            mm::gs_butterfly(X, Y, W[widx], Wp[widx], q);
            x[l] = X;
            x[l + (1 << lt)] = Y;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < R * T1; e += blockDim.x) D[(size_t)hi0 * T1 + e] = sm[e];
}

__global__ void __launch_bounds__(NTT_THREADS) k_ntt_inv_cols(uint64_t *dst, RowMap md, ModTab mt, Twiddles tw,
                                                              NttShape sh) {
    extern __shared__ uint64_t sm[];
    const uint32_t r = blockIdx.y;
    const uint8_t pid = md.pid[r % md.period];
    if (pid == SKIP) return;
    uint64_t *D = dst + row_offset(md, r, sh.logn);
    const int cols = sh.cols, T1 = sh.T1, H = sh.H, s1 = sh.s1;
    const int lo0 = blockIdx.x * cols;
    const uint64_t q = mt.q[pid];
    for (int e = threadIdx.x; e < H * cols; e += blockDim.x) {
        int h = e / cols, c = e - h * cols;
        sm[e] = D[(size_t)h * T1 + lo0 + c];
    }
    __syncthreads();
    const uint64_t *W = tw.iw + ((size_t)pid << sh.logn);
    const uint64_t *Wp = tw.iw_sh + ((size_t)pid << sh.logn);
    for (int s = s1 - 1; s >= 0; s--) {
        const int ltt = s1 - s - 1;
        for (int e = threadIdx.x; e < (H >> 1) * cols; e += blockDim.x) {
            int hb = e / cols, c = e - hb * cols;
            int h = ((hb >> ltt) << (ltt + 1)) + (hb & ((1 << ltt) - 1));
            int widx = (1 << s) + (h >> (s1 - s));
            uint64_t X = sm[h * cols + c], Y = sm[(h + (1 << ltt)) * cols + c];
            mm::gs_butterfly(X, Y, W[widx], Wp[widx], q);
            sm[h * cols + c] = X;
            sm[(h + (1 << ltt)) * cols + c] = Y;
        }
        __syncthreads();
    }
    const uint64_t ni = tw.ninv[pid], nip = tw.ninv_sh[pid];
    for (int e = threadIdx.x; e < H * cols; e += blockDim.x) {
        int h = e / cols, c = e - h * cols;
        D[(size_t)h * T1 + lo0 + c] = mm::mul_shoup(sm[e], ni, nip, q);
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

void launch_ntt(Context &c, const RowsView &src, const RowsView &dst, bool inverse, cudaStream_t st) {
    if (src.rows == 0) return;
    const NttShape sh = shape_for(c.logn);
    const size_t smem = TILE_WORDS * sizeof(uint64_t);
    // grid.y is limited to 65535 rows per launch: split on block boundaries
    const size_t chunk = (65535 / src.map.period) * src.map.period;
    for (size_t r0 = 0; r0 < src.rows; r0 += chunk) {
        size_t nr = std::min<size_t>(chunk, src.rows - r0);
        RowMap ms = src.map, md = dst.map;
        size_t blocks0 = r0 / ms.period;
        const uint64_t *sb = src.base + ((blocks0 * ms.block_stride) << c.logn);
        uint64_t *db = dst.base + ((blocks0 * md.block_stride) << c.logn);
        dim3 gc(sh.T1 / sh.cols, (unsigned)nr), gr(sh.H / sh.rows_per_cta, (unsigned)nr), blk(NTT_THREADS);
        size_t live = 0;   // rows actually transformed (skipped rows move no data)
        for (size_t r = 0; r < nr; r++) live += md.pid[r % md.period] != SKIP;
        const double bytes = 2.0 * (double)live * c.n * 8;   // each pass reads and writes every live row once
        if (!inverse) {
            kernel_begin(c, st);
            k_ntt_fwd_cols<<<gc, blk, smem, st>>>(sb, ms, db, md, c.mods, c.tw, sh);
            kernel_end(c, "ntt_fwd_cols", gc, blk, bytes, st);
            kernel_begin(c, st);
            k_ntt_fwd_rows<<<gr, blk, smem, st>>>(db, md, c.mods, c.tw, sh);
            kernel_end(c, "ntt_fwd_rows", gr, blk, bytes, st);
        } else {
            kernel_begin(c, st);
            k_ntt_inv_rows<<<gr, blk, smem, st>>>(sb, ms, db, md, c.mods, c.tw, sh);
            kernel_end(c, "ntt_inv_rows", gr, blk, bytes, st);
            kernel_begin(c, st);
            k_ntt_inv_cols<<<gc, blk, smem, st>>>(db, md, c.mods, c.tw, sh);
            kernel_end(c, "ntt_inv_cols", gc, blk, bytes, st);
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
