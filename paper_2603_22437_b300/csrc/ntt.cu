// Row maps, launch bookkeeping (launch count, trace, event profile) and the
// dispatch of the NTT passes to their per-ring-dimension entry points
// (ntt_launch.h); the kernels are in ntt_impl.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "internal.h"
#include "kernels.h"
#include "ntt_impl.cuh"
#include "ntt_launch.h"

namespace mmfhe {

namespace {

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

// Consecutive active rows that read the same conversion source, in groups of
// at most rg: rows p, p' share it when p / src_rows == p' / src_rows (one
// ModUp digit), or always when src_rows == 0 (every ModDown row).
static RowGroups make_groups(const RowMap &m, int rg, int src_rows) {
    RowGroups g{};
    for (uint32_t k = 0; k < m.nact; k++) {
        const bool same = g.n > 0 && g.count[g.n - 1] < rg &&
                          (src_rows == 0 || m.act[k] / src_rows == m.act[g.start[g.n - 1]] / src_rows);
        if (same) {
            g.count[g.n - 1]++;
        } else {
            g.start[g.n] = (uint8_t)k;
            g.count[g.n] = 1;
            g.n++;
        }
    }
    return g;
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
    c.prof.push_back(Context::ProfRec{nullptr, e, nullptr, 0.0, 0.0, 0.0});
}

void kernel_end(Context &c, const char *name, dim3 g, dim3 b, double bytes, cudaStream_t st, double butterflies,
                double macs) {
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
        r.macs = macs;
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
#define MMFHE_NTT_CALL(L) ntt_launch_##L(c, sb, ms, db, md, nr, inverse, bytes, oscale, oscale_sh, st)
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
        const RowGroups gr = make_groups(md, c.tune.conv_rows, nre);
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
            // conversion work: every converted word of digit j sums |D_j| products
            double macs = 0.0;
            for (int jj = 0; jj < nj; jj++) {
                const double dj = (double)lc.digits[j0 + jj].size();
                macs += (double)nb * (double)(nre - (int)dj) * dj * (double)c.n;
            }
#define MMFHE_MODUP_CALL(L) modup_launch_##L(c, db, yb, md, gr, nb, nl, nre, j0, lc.d_up_mm, bc_, br_, macs, st)
            MMFHE_LOGN_DISPATCH(c.logn, MMFHE_MODUP_CALL)
#undef MMFHE_MODUP_CALL
        }
    }
    CK(cudaGetLastError());
}

void launch_keyip_p_inv(Context &c, uint64_t *z, const KeyipArgs &ka, int B, int level, cudaStream_t st) {
    const int K = c.num_p;
    if (B == 0) return;
    std::vector<int> pids(K);
    for (int k = 0; k < K; k++) pids[k] = c.num_q + k;
    RowMap mz = make_map(K, K, pids), ms = mz;
    set_active(ms, mz);
    const size_t chunk = 65535 / (2 * (size_t)K);   // windows per launch
    const double row = (double)c.n * 8;
    for (size_t w0 = 0; w0 < (size_t)B; w0 += chunk) {
        const size_t nw = std::min(chunk, (size_t)B - w0);
        const size_t nr = nw * 2 * K;
        KeyipArgs kc = ka;
        kc.w0 = ka.w0 + (int)w0;
        // reads each window's beta digit rows of the P primes and the keys' rows (once per
        // launch when shared), writes every z row; the strided pass reads and writes z
        const double kn = ka.key.n == 1 ? 1.0 : (double)nw;
        const double br_ = row * ((double)nr + (double)nw * ka.beta * K + kn * ka.beta * 2.0 * K);
        const double bc_ = 2.0 * row * (double)nr;
#define MMFHE_KPI_CALL(L)                                                                                         \
    keyip_p_inv_launch_##L(c, z + ((w0 * 2 * K) << c.logn), kc, mz, nr, br_, bc_, c.lv[level].d_ks_scale,         \
                           c.lv[level].d_ks_scale_sh, st)
        MMFHE_LOGN_DISPATCH(c.logn, MMFHE_KPI_CALL)
#undef MMFHE_KPI_CALL
    }
    CK(cudaGetLastError());
}

static void moddown_ntt_impl(Context &c, uint64_t *vtmp, const uint64_t *z, const CombineArgs &a, size_t blocks,
                             int level, cudaStream_t st, const KeyipArgs *ka);

void launch_moddown_ntt_blocks(Context &c, uint64_t *vtmp, const uint64_t *z, const CombineArgs &a, size_t blocks,
                               int level, cudaStream_t st) {
    if (a.add0 || a.add1) throw Error(MMFHE_ERR_BAD_ARG, "moddown of single blocks takes no window addends");
    moddown_ntt_impl(c, vtmp, z, a, blocks, level, st, nullptr);
}

void launch_moddown_ntt(Context &c, uint64_t *vtmp, const uint64_t *z, const CombineArgs &a, int B, int level,
                        cudaStream_t st, const KeyipArgs *ka) {
    moddown_ntt_impl(c, vtmp, z, a, (size_t)B * 2, level, st, ka);
}

static void moddown_ntt_impl(Context &c, uint64_t *vtmp, const uint64_t *z, const CombineArgs &a, size_t blocks,
                             int level, cudaStream_t st, const KeyipArgs *ka) {
    const int nl = level + 1, nre = nl + c.num_p, K = c.num_p;
    if (blocks == 0) return;
    const size_t ustride = a.u_stride ? a.u_stride : (size_t)nre;
    std::vector<int> pids(nl);
    for (int i = 0; i < nl; i++) pids[i] = i;
    RowMap mv = make_map(nl, nl, pids), ms = mv;
    const uint32_t nact = set_active(ms, mv);
    const RowGroups gr = make_groups(mv, c.tune.conv_rows, 0);
    const size_t chunk = 65535 / nact;
    for (size_t b0 = 0; b0 < blocks; b0 += chunk) {
        // chunks hold whole windows, so the (window, h) parity of a block is kept
        const size_t nb = std::min(chunk & ~(size_t)1, blocks - b0);
        const size_t nr = nb * nact;
        CombineArgs ab = a;
        ab.out = a.out + ((b0 * nl) << c.logn);
        if (ab.u) ab.u = a.u + ((b0 * ustride) << c.logn);
        if (ab.add0) ab.add0 += (b0 / 2) * a.add_stride;
        if (ab.add1) ab.add1 += (b0 / 2) * a.add_stride;
        if (ab.plus) ab.plus += (b0 * nl) << c.logn;
        KeyipArgs kc{};
        if (ka) {
            kc = *ka;
            kc.w0 = ka->w0 + (int)(b0 / 2);
        }
        const double row = (double)c.n * 8;
        const double bc_ = row * ((double)nr + (double)nb * K);
        // v read and out written per row; u read, or the key inner product's digit rows
        // (once per window) and key rows (once per launch when shared)
        double ub = (double)nr;
        if (ka) ub = (double)(nb / 2) * ka->beta * nl + (ka->key.n == 1 ? 1.0 : nb / 2.0) * ka->beta * 2.0 * nl;
        const double br_ = row * ((double)nr * (2 + (ab.plus ? 1 : 0)) + ub + (ab.add0 ? nr / 2.0 : 0) + (ab.add1 ? nr / 2.0 : 0));
#define MMFHE_MODDOWN_CALL(L)                                                                                   \
    moddown_launch_##L(c, vtmp + ((b0 * nl) << c.logn), z + ((b0 * K) << c.logn), mv, gr, nb, ab, nre, bc_, br_,   \
                       (double)nr * c.n * (K + 1), ka ? &kc : nullptr, st)
        MMFHE_LOGN_DISPATCH(c.logn, MMFHE_MODDOWN_CALL)
#undef MMFHE_MODDOWN_CALL
    }
    CK(cudaGetLastError());
}

}  // namespace mmfhe
