// Internal structures of the mmfhe library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "mmfhe.h"

namespace mmfhe {

constexpr int MAXPRIMES = MMFHE_MAX_Q + MMFHE_MAX_P;   // prime ids: 0..num_q-1 = q_i, num_q.. = p_k
constexpr int MAXROWMAP = 64;
constexpr uint8_t SKIP = 0xFF;

// Error carrying an ABI status code; caught at the ABI boundary.
struct Error : std::runtime_error {
    mmfhe_status code;
    Error(mmfhe_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

void cuda_check(cudaError_t e, const char *what);
#define CK(x) ::mmfhe::cuda_check((x), #x)

// Moduli passed by value to kernels (constant-bank resident).
struct ModTab {
    uint64_t q[MAXPRIMES];
    uint64_t mu[MAXPRIMES];     // Barrett constant floor(2^(2k) / q)
    uint64_t qinv[MAXPRIMES];   // q^-1 mod 2^64 (Montgomery reduction)
    uint64_t r64[MAXPRIMES];    // 2^64 mod q (conversion into Montgomery form)
    uint32_t k[MAXPRIMES];
};

// Row addressing of a launch over blocks of `period` rows: period row p of
// block b lives at base + (b * block_stride + p - row0) * N and is reduced mod
// prime pid[p] (SKIP = untouched).  The launcher fills act[0..nact) with the
// non-SKIP period rows, so a grid covers only the rows it transforms.
struct RowMap {
    uint32_t period;
    uint32_t block_stride;   // in rows
    uint32_t row0;           // first stored period row (0 unless the buffer holds a tail of each block)
    uint32_t nact;
    uint8_t pid[MAXROWMAP];
    uint8_t act[MAXROWMAP];
};

// Groups of rows of one launch that share a base-conversion source: group g
// holds the active rows act[start[g]] .. act[start[g] + count[g] - 1] of the
// launch's row map (consecutive, same source rows).
struct RowGroups {
    uint32_t n;
    uint8_t start[MAXROWMAP];
    uint8_t count[MAXROWMAP];
};

// Twiddle tables (device): [prime id][N], forward psi^brv(i) and inverse
// psi^-brv(i) with Shoup companions; n_inv per prime with companion.
struct Twiddles {
    const uint64_t *fw, *fw_sh, *iw, *iw_sh;
    const uint64_t *ninv, *ninv_sh;
};

// ---------------------------------------------------------------------------
// device memory pool (caching, by exact size; stream-ordered reuse)
// ---------------------------------------------------------------------------
class Pool {
public:
    explicit Pool(int device) : device_(device) {}
    ~Pool();
    uint64_t *get(size_t words);
    void put(uint64_t *p, size_t words);
    size_t bytes_held() const { return held_; }
    size_t bytes_free() const { return free_bytes_; }
    void trim();

private:
    int device_;
    std::multimap<size_t, uint64_t *> free_;
    size_t held_ = 0;
    size_t free_bytes_ = 0;
};

// Every device allocation of the evaluator goes through dev_alloc / dev_free,
// which keep per-device totals (current bytes, high-water mark, number of
// cudaMalloc calls).  dev_alloc returns nullptr when cudaMalloc fails and
// throws OUT_OF_MEMORY while the failure hook (set_fail_after) is armed:
// after n more successful allocations, every later one fails without calling
// cudaMalloc until the hook is disarmed (n < 0).
void *dev_alloc(int device, size_t bytes);
void dev_free(int device, void *p, size_t bytes);
void mem_stats(int device, uint64_t *bytes, uint64_t *peak, uint64_t *allocs);
void mem_peak_reset(int device);
void set_fail_after(int64_t n);

// Pooled device buffer (RAII).
class Buf {
public:
    Buf() = default;
    Buf(Pool *pool, size_t words) : pool_(pool), words_(words), p_(words ? pool->get(words) : nullptr) {}
    ~Buf() { release(); }
    Buf(Buf &&o) noexcept { *this = std::move(o); }
    Buf &operator=(Buf &&o) noexcept {
        if (this != &o) {
            release();
            pool_ = o.pool_; words_ = o.words_; p_ = o.p_;
            o.p_ = nullptr; o.words_ = 0;
        }
        return *this;
    }
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    uint64_t *get() const { return p_; }
    size_t words() const { return words_; }
    void release() {
        if (p_ && pool_) pool_->put(p_, words_);
        p_ = nullptr; words_ = 0;
    }

private:
    Pool *pool_ = nullptr;
    size_t words_ = 0;
    uint64_t *p_ = nullptr;
};

// Per-level basis-conversion constants (device).
struct LevelConsts {
    int level;
    int beta;                        // digits at this level
    std::vector<std::vector<int>> digits;
    // ModUp: for digit j, source u (< alpha), target row t (< level+1+K):
    //  inv[j][u] = (Qhat_{j,u})^-1 mod q_{D_j[u]} (+ Shoup),
    //  m[j][u][t] = Qhat_{j,u} mod prime(t) (+ Shoup)
    uint64_t *d_up_inv = nullptr, *d_up_inv_sh = nullptr;
    uint64_t *d_up_m = nullptr, *d_up_m_sh = nullptr;
    // fused ModUp (Montgomery form): m_mont[j][u][t] = Qhat_{j,u} * 2^64 mod prime(t)
    uint64_t *d_up_mm = nullptr;
    // last multiply of the key switch's inverse NTTs, by prime id: N^-1 (Qhat_{j,u})^-1
    // for q_i (ModUp input rows) and N^-1 Phat_k^-1 for p_k (ModDown P rows) (+ Shoup)
    uint64_t *d_ks_scale = nullptr, *d_ks_scale_sh = nullptr;
    // rescale by q_level: qinv[i] = q_level^-1 mod q_i, qmod[i] = q_level mod q_i
    uint64_t *d_rs_qinv = nullptr, *d_rs_qinv_sh = nullptr, *d_rs_qmod = nullptr;
};

// Tile shapes and work split picked by the autotuner (tune.cu).
struct Tune {
    int cols_w = 16;     // columns per CTA of the strided NTT pass (8 or 16)
    int rows_t = 256;    // threads per CTA of the contiguous NTT pass (128 or 256)
    int keyip_wg = 4;    // windows per thread of the key inner product (1, 2, 4 or 8)
    int conv_rows = 1;   // converted rows per CTA of the fused ModUp / ModDown strided passes (1, 2 or 4)
    int keyip_fused = 0; // key inner product stored by its own kernel (0) or formed inside the ModDown passes (1)
    int keyip_pipe = 0;  // shared-key inner product with the window walk pipelined through shared memory (1)
    float ntt_ms[4] = {};     // last autotune: NTT pair per (cols_w, rows_t) in {8,16} x {128,256}
    float keyip_ms[4] = {};   // last autotune: key inner product per window group 1, 2, 4, 8
    float keyip_pipe_ms[4] = {};   // the same, pipelined
    int combine_pipe = 0;          // the ModDown combine walks its tiles with the next tile's load in flight (1)
    float combine_pipe_ms[3] = {};    // last autotune: fused ModUp + ModDown with the pipelined combine, rows 1, 2, 4
    float conv_ms[3] = {};    // last autotune: fused ModUp + ModDown per rows per CTA 1, 2, 4
};


struct Context {
    int device = 0;
    int sm_count = 148;   // streaming multiprocessors of the device (persistent grids)
    Tune tune;
    mmfhe_params params{};
    int logn = 0;
    uint32_t n = 0;
    int num_q = 0, num_p = 0, dnum = 0, alpha = 0;
    int L = 0;
    std::vector<uint64_t> primes;    // by prime id
    ModTab mods{};
    uint64_t *d_tw = nullptr;        // 4 * np * N words
    uint64_t *d_ninv = nullptr;      // 2 * np words
    Twiddles tw{};
    // ModDown constants: pinv[k] = Phat_k^-1 mod p_k, phat[k][i] = Phat_k mod q_i,
    // pmod[i] = P mod q_i, Pinv[i] = P^-1 mod q_i (with Shoup companions)
    uint64_t *d_dn_pinv = nullptr, *d_dn_pinv_sh = nullptr;
    uint64_t *d_dn_phat = nullptr, *d_dn_phat_sh = nullptr;
    uint64_t *d_dn_pmod = nullptr, *d_dn_pmod_sh = nullptr, *d_dn_Pinv = nullptr, *d_dn_Pinv_sh = nullptr;
    // Montgomery forms for the fused ModDown: phat_mont[k][i] = Phat_k 2^64 mod q_i,
    // negp_mont[i] = (-P) 2^64 mod q_i
    uint64_t *d_dn_phat_mont = nullptr, *d_dn_negp_mont = nullptr;
    std::vector<LevelConsts> lv;     // per level 0..L
    int sum_terms_max = 8;           // products one Montgomery reduction may absorb: n*q_max < 2^64
    int sum_terms_max_qp = 8;        // the same over every prime of Q * P (extended-basis sums)
    std::unique_ptr<Pool> pool;
    uint64_t launches = 0;
    std::string last_error;
    std::vector<std::pair<void *, size_t>> owned;   // device tables (pointer, bytes)
    uint64_t *noalloc_scratch = nullptr;              // device address of the no-allocation scratch array
    // optional launch trace (kernel name + shape) for the data-obliviousness test
    bool tracing = false;
    std::vector<std::string> trace;
    // optional per-launch CUDA-event profile: (name, start, stop, algorithmic bytes)
    bool profiling = false;
    struct ProfRec {
        const char *name;
        cudaEvent_t start, stop;
        double bytes;
        double butterflies;
        double macs;   // multiply-accumulates of fused base conversions
    };
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> event_pool;
    size_t event_next = 0;

    size_t ct_words(int level) const { return 2ull * (level + 1) * n; }
};

// ---------------------------------------------------------------------------
// device ciphertext batch (evaluation domain), layout [B][2][level+1][N]
// ---------------------------------------------------------------------------
struct CtB {
    Buf buf;
    int B = 0;
    int level = -1;
    double scale = 0.0;
    uint64_t *ptr() const { return buf.get(); }
};

// Degree-2 tensor batch: [B][3][level+1][N] (d0, d1, d2).
struct TensorB {
    Buf buf;
    int B = 0;
    int level = -1;
    double scale = 0.0;
};

// ModUp digits [B][beta][level+1+K][N], evaluation domain.  Row t of digit j
// for t inside digit j's own primes is not stored: it equals the input row,
// read from `own` (window b at own + b * own_stride, row t at + t * N), which
// must outlive the digits.
struct DigitsB {
    Buf buf;
    int B = 0;
    int level = -1;
    int beta = 0;
    const uint64_t *own = nullptr;
    size_t own_stride = 0;   // words
};

// Plaintext on device (evaluation domain), [level+1][N].
struct PtDev {
    Buf buf;
    int level = -1;
    double scale = 0.0;
    bool mont = false;   // words stored as x * 2^64 mod q (Montgomery form)
    bool qp = false;     // rows over the extended basis: q_0..q_level, then p_0..p_{K-1}
};

struct Keys {
    Context *ctx = nullptr;
    uint64_t user = 0;
    Buf rlk;                                   // [dnum][2][L+1+K][N] eval
    std::map<int32_t, Buf> gk;                 // rotation (mod N/2) -> key
    // A batch mixing users: the key set of every window, in window order
    // (rlk and gk are then unused).
    std::vector<const Keys *> windows;
};

// Switching-key words of one key switch: one key for every window (n == 1)
// or one per window (n == B, a batch mixing users), passed by value to the
// key inner product.
constexpr int MAX_KEY_WINDOWS = 64;
struct KeyPtrs {
    const uint64_t *k[MAX_KEY_WINDOWS];
    int n = 0;
};

// ---------------------------------------------------------------------------
// launchers (ntt.cu)
// ---------------------------------------------------------------------------
struct RowsView {
    uint64_t *base;
    RowMap map;
    size_t rows;
};

RowMap make_map(uint32_t period, uint32_t block_stride, const std::vector<int> &pids);

// Forward or inverse NTT of the rows of src into dst (same period and active
// rows).  An inverse NTT ends with a multiply by N^-1 mod q, or, when oscale is
// given, by oscale[pid] (with its Shoup companion oscale_sh[pid]).
void launch_ntt(Context &c, const RowsView &src, const RowsView &dst, bool inverse, cudaStream_t s,
                const uint64_t *oscale = nullptr, const uint64_t *oscale_sh = nullptr);
void launch_copy_rows(Context &c, const RowsView &src, const RowsView &dst, cudaStream_t s);

// Time the tile-shape variants on a batch of `batch` ciphertexts at `level`
// and keep the fastest in c.tune (tune.cu).
void autotune(Context &c, int batch, int level);

// Butterflies per second of register-resident 64-bit and 32-bit butterfly loops (peaks.cu).
void measure_butterfly_peak(Context &c, double *bf64, double *bf32);
// Products per second of a register-resident loop of the base conversion's
// Montgomery multiply-accumulate (four products per reduction) (peaks.cu).
double measure_mac_peak(Context &c);

// Launch bookkeeping: kernel_begin before a launch, kernel_end after it
// (launch count, optional trace line, optional event pair + algorithmic bytes).
void kernel_begin(Context &c, cudaStream_t st);
void kernel_end(Context &c, const char *name, dim3 g, dim3 b, double bytes, cudaStream_t st,
                double butterflies = 0.0, double macs = 0.0);

}  // namespace mmfhe
