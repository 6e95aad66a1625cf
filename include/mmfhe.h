/*
 * mmfhe.h -- C ABI of the B300 (sm_103a) homomorphic evaluation library for
 * the mmFHE cloud side: CKKS (RNS, hybrid key switching) evaluation of the
 * paper's data-oblivious radar DSP kernel chains on batches of ciphertext
 * windows.
 *
 * Problem statement followed (paper Sec. "System Design"): the cloud receives
 * ciphertexts plus the public evaluation keys (rlk, gk), chains the fixed
 * kernels K1..K7 over the ciphertexts, and returns encrypted results; the
 * client alone decrypts.  The calls below are exactly that: create a context
 * for a parameter set, load evaluation keys, load a plan (the public
 * constants of a circuit), evaluate a batch of windows, synchronise.
 *
 * Conventions (apply to every call unless stated otherwise)
 * ---------------------------------------------------------
 *  - Status: every call returns MMFHE_OK (0) or a negative MMFHE_ERR_* code;
 *    no C++ exception crosses the ABI.  mmfhe_last_error() gives a message.
 *  - Rings: R_q = Z_q[X]/(X^N + 1), N = 2^log_n.  Q = q_0 ... q_L ("level l"
 *    uses q_0..q_l, i.e. l+1 limbs), P = p_0 ... p_{K-1} (special primes).
 *  - Boundary form: every polynomial crossing the ABI is in COEFFICIENT form,
 *    limb-major, little-endian uint64, limb i holding residues in [0, q_i).
 *    A ciphertext at level l is uint64[2][l+1][N] (c0 then c1; decrypts as
 *    c0 + c1*s).  A batch of B ciphertexts is uint64[B][2][l+1][N].
 *    A plaintext at level l is uint64[l+1][N].
 *    A switching key is uint64[dnum][2][L+1+K][N]: digit j holds (b_j, a_j)
 *    over q_0..q_L then p_0..p_{K-1}, with b_j = -a_j*s + e_j + P*Qt_j*s'.
 *  - Memory: pointers may be host or device memory of the context's device
 *    (detected with cudaPointerGetAttributes).  The caller owns all buffers
 *    it passes; inputs are not modified unless stated.  The library owns
 *    contexts, keys and plans until the matching destroy/unload call; it
 *    copies every blob it is given, so the caller may free them on return.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *    Calls that take a stream only enqueue work, except that host buffers are
 *    copied synchronously with respect to the call (the call returns after
 *    host outputs are written).  Calls on one context must use one stream at
 *    a time (the context's scratch pool is stream-ordered); synchronise
 *    before switching streams.  Use mmfhe_sync for a bounded wait.
 *  - Alignment: device pointers must be 16-byte aligned.
 *  - Thread safety: one context may be used by one host thread at a time.
 */
#ifndef MMFHE_H
#define MMFHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mmfhe_status;

#define MMFHE_OK 0
#define MMFHE_ERR_BAD_ARG (-1)        /* null pointer, size or value out of range */
#define MMFHE_ERR_BAD_BLOB (-2)       /* malformed parameter set / key / constant */
#define MMFHE_ERR_PARAM_MISMATCH (-3) /* object built for another context */
#define MMFHE_ERR_LEVEL_MISMATCH (-4) /* operand levels do not fit the operation */
#define MMFHE_ERR_OUT_OF_MEMORY (-5)  /* device allocation failed */
#define MMFHE_ERR_CUDA (-6)           /* a CUDA runtime call failed (no device, launch error) */
#define MMFHE_ERR_TIMEOUT (-7)        /* bounded wait expired; work is still queued */
#define MMFHE_ERR_NOT_FOUND (-8)      /* missing Galois key / constant */
#define MMFHE_ERR_BUSY (-9)           /* object in use */
#define MMFHE_ERR_CANCELLED (-10)     /* a queued serving request was cancelled */

#define MMFHE_MAX_Q 32
#define MMFHE_MAX_P 8

/* ------------------------------------------------------------------------
 * Parameters (paper Table 7: CKKS, N = 32768, depth 11, 128-bit classical
 * security per the HE Standard; Delta = 2^40 vital, 2^50 gesture).
 * ---------------------------------------------------------------------- */
typedef struct mmfhe_params {
    uint32_t log_n;            /* ring dimension N = 2^log_n, 10 <= log_n <= 16 */
    uint32_t num_q;            /* L + 1, 1..MMFHE_MAX_Q */
    uint32_t num_p;            /* K, 1..MMFHE_MAX_P */
    uint32_t dnum;             /* key-switching digits; alpha = ceil(num_q/dnum) <= num_p required */
    uint64_t q[MMFHE_MAX_Q];   /* q_0..q_L: distinct primes = 1 mod 2N, 2^20 < q < 2^61 */
    uint64_t p[MMFHE_MAX_P];   /* p_0..p_{K-1}: same conditions, distinct from q */
} mmfhe_params;

/* Deterministic prime selection (host only, needs no GPU):
 * q_0 = largest prime < 2^q0_bits with q = 1 mod 2N; q_1..q_L alternate
 * largest-unused-below / smallest-unused-above 2^q_bits (below first);
 * p_k = largest unused primes < 2^p_bits.  Errors: BAD_ARG. */
mmfhe_status mmfhe_params_select(uint32_t log_n, uint32_t num_q, uint32_t q0_bits, uint32_t q_bits,
                                 uint32_t num_p, uint32_t p_bits, uint32_t dnum, mmfhe_params *out);

/* ------------------------------------------------------------------------
 * Context: one parameter set on one device.  Builds the NTT twiddle tables,
 * basis-conversion and rescale constants in device memory.
 * params_size must be sizeof(mmfhe_params).  Errors: BAD_ARG, BAD_BLOB
 * (non-prime / not 1 mod 2N / duplicate / out of range), CUDA (no device),
 * OUT_OF_MEMORY.
 * ---------------------------------------------------------------------- */
typedef struct mmfhe_ctx mmfhe_ctx;
mmfhe_status mmfhe_ctx_create(const mmfhe_params *params, size_t params_size, int device, mmfhe_ctx **out);
mmfhe_status mmfhe_ctx_destroy(mmfhe_ctx *ctx);
/* Message of the last failing call on ctx (ctx may be NULL: last failure of
 * the calling thread).  The string stays valid until the next call. */
const char *mmfhe_last_error(const mmfhe_ctx *ctx);
/* Bounded wait for all work on `stream`: polls, returns TIMEOUT after
 * timeout_ms without blocking further (the work stays queued). */
mmfhe_status mmfhe_sync(mmfhe_ctx *ctx, void *stream, uint32_t timeout_ms);
/* Number of kernels this library has launched on ctx since creation. */
mmfhe_status mmfhe_launch_count(const mmfhe_ctx *ctx, uint64_t *out);
/* Device memory held by this library on the context's device (no
 * counterpart in the paper beyond its Table 5 "peak GPU memory"): every
 * context, key set, plan, scratch pool, graph and staging buffer of the
 * library on that device, summed over all contexts there.  peak_bytes is the
 * high-water mark since the last mmfhe_mem_peak_reset (or since the library
 * was loaded); allocations counts the library's cudaMalloc calls on the
 * device; pool_bytes / pool_free_bytes are ctx's own scratch pool (cached
 * blocks included) and the part of it not in use.  Errors: BAD_ARG. */
typedef struct mmfhe_mem_stats {
    uint64_t device_bytes;
    uint64_t peak_bytes;
    uint64_t allocations;
    uint64_t pool_bytes;
    uint64_t pool_free_bytes;
} mmfhe_mem_stats;
mmfhe_status mmfhe_mem_stats_get(const mmfhe_ctx *ctx, mmfhe_mem_stats *out);
/* Restart the high-water mark at the current device_bytes. */
mmfhe_status mmfhe_mem_peak_reset(mmfhe_ctx *ctx);
/* Host-side fault injection for tests of the failure paths (no GPU fault is
 * involved): after `after` more successful device allocations, every device
 * allocation of the library's evaluator (pools, context tables, batcher
 * staging) fails with OUT_OF_MEMORY without calling cudaMalloc, until the
 * hook is disarmed with after < 0.  Process-wide; needs no device. */
mmfhe_status mmfhe_debug_fail_allocations(int64_t after);
/* Launch trace for auditing data obliviousness (Theorem 2: the execution
 * trace depends only on public parameters).  enable != 0 clears the trace and
 * starts recording one line "kernel grid(x,y,z) block(x,y,z)" per launch;
 * enable == 0 stops.  mmfhe_trace_get copies up to capacity-1 bytes of the
 * newline-separated trace into buf (NUL-terminated) and sets *length to the
 * full length. */
mmfhe_status mmfhe_trace_enable(mmfhe_ctx *ctx, int enable);
mmfhe_status mmfhe_trace_get(const mmfhe_ctx *ctx, char *buf, size_t capacity, size_t *length);
/* Per-kernel CUDA-event profile.  enable != 0 clears the profile and records
 * a start/stop event pair around every subsequent launch (on the launch's
 * stream); enable == 0 stops recording.  mmfhe_profile_get synchronises the
 * recorded events and aggregates them by kernel name: up to `capacity`
 * entries are written (names NUL-terminated, truncated to 31 chars);
 * *count is the number of distinct kernels.  bytes = the launches'
 * algorithmic bytes (every distinct word a launch must read or write once);
 * butterflies = the NTT butterflies the launches perform (N/2 per stage per
 * transformed row; 0 for kernels without NTT stages). */
typedef struct mmfhe_kernel_stat {
    char name[32];
    uint64_t launches;
    double total_ms;
    double bytes;
    double butterflies;
    double macs;        /* multiply-accumulates of fused base conversions (ModUp, ModDown strided passes) */
} mmfhe_kernel_stat;
mmfhe_status mmfhe_profile_enable(mmfhe_ctx *ctx, int enable);
mmfhe_status mmfhe_profile_get(mmfhe_ctx *ctx, mmfhe_kernel_stat *out, uint32_t capacity, uint32_t *count);
/* Integer-pipe ceiling of the NTT arithmetic on this device (no counterpart in
 * the paper: a measurement helper for the roofline).  Runs a register-resident
 * loop of the library's forward butterfly (64-bit words, Harvey lazy reduction
 * with a Shoup product) on every SM, and the same butterfly on 32-bit words,
 * and returns butterflies per second for each (CUDA-event timed, after one
 * warm-up launch).  No memory traffic beyond one word per thread.  Errors:
 * BAD_ARG (null output), CUDA. */
mmfhe_status mmfhe_measure_butterfly_peak(mmfhe_ctx *ctx, double *bf64_per_s, double *bf32_per_s);
/* The same for the base conversion's arithmetic: a register-resident loop of
 * Montgomery multiply-accumulates (four 64-bit products summed in 128 bits,
 * one reduction) on every SM; returns products per second. */
mmfhe_status mmfhe_measure_mac_peak(mmfhe_ctx *ctx, double *mac64_per_s);

/* ------------------------------------------------------------------------
 * Evaluation keys (paper: rlk after every ct x ct product, one Galois key
 * per rotation amount).  Keys are converted to the library's evaluation
 * domain and stay resident in device memory until unloaded.
 * ---------------------------------------------------------------------- */
typedef struct mmfhe_keys mmfhe_keys;
mmfhe_status mmfhe_keys_create(mmfhe_ctx *ctx, uint64_t user_id, mmfhe_keys **out);
/* words: switching key from s^2 to s, layout above.  Errors: BAD_ARG. */
mmfhe_status mmfhe_keys_set_relin(mmfhe_keys *keys, const uint64_t *words);
/* Galois key for the left rotation Rot(x, k)[j] = x[(j + k) mod N/2], i.e.
 * the automorphism X -> X^g, g = 5^(k mod N/2) mod 2N; switches s(X^g) to s.
 * rotation = MMFHE_ROT_CONJ: the key of the conjugation g = 2N - 1 (every
 * slot to its complex conjugate). */
#define MMFHE_ROT_CONJ ((int32_t)0x80000000)
mmfhe_status mmfhe_keys_set_galois(mmfhe_keys *keys, int32_t rotation, const uint64_t *words);
mmfhe_status mmfhe_keys_unload(mmfhe_keys *keys);

/* ------------------------------------------------------------------------
 * Primitive operations (for composition and testing).  All take and return
 * coefficient-form buffers, batched over `batch` ciphertexts of one level.
 * Each call converts to the evaluation domain, runs, and converts back.
 * Level errors: LEVEL_MISMATCH.  Missing key: NOT_FOUND.
 * ---------------------------------------------------------------------- */
/* Negacyclic NTT of `rows` rows of N words in place; row r is reduced mod the
 * prime with index prime_idx[r] (0..num_q-1 = q_i, num_q..num_q+K-1 = p_k;
 * prime_idx is a host array).  Forward output order is the library's
 * evaluation order (row j holds a(psi^(2 brv(j) + 1))); inverse takes that
 * order back to coefficients. */
mmfhe_status mmfhe_ntt(mmfhe_ctx *ctx, uint64_t *rows, const uint32_t *prime_idx, size_t num_rows, int inverse, void *stream);
/* The batched transform the evaluator runs on ciphertexts: blocks x limbs
 * rows of N words in DEVICE memory (16-byte aligned), row (b, i) reduced mod
 * q_i, limbs 1..num_q; asynchronous on `stream` (two launches: the strided
 * and the contiguous pass over every row).  BAD_ARG for host memory. */
mmfhe_status mmfhe_ntt_batch(mmfhe_ctx *ctx, uint64_t *rows, size_t blocks, uint32_t limbs, int inverse, void *stream);
/* out[r] = a[r] * b[r] in Z_q[X]/(X^N+1), coefficient form (at most 64 rows). */
mmfhe_status mmfhe_poly_mul(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b,
                            const uint32_t *prime_idx, size_t num_rows, void *stream);
/* out = a + b (slot-wise add, depth free). */
mmfhe_status mmfhe_ct_add(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b, size_t batch,
                          uint32_t level, void *stream);
/* out = ct * pt (pt shared by the batch), not rescaled. */
mmfhe_status mmfhe_ct_mul_plain(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *ct, const uint64_t *pt, size_t batch,
                                uint32_t level, void *stream);
/* out = relinearize(a (x) b): tensor product + key switch with rlk; not rescaled. */
mmfhe_status mmfhe_ct_mul_relin(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *a,
                                const uint64_t *b, size_t batch, uint32_t level, void *stream);
/* out (level-1) = rescale(in): c_i <- (c_i - [c]_{q_l}^centered) * q_l^-1. */
mmfhe_status mmfhe_ct_rescale(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *in, size_t batch, uint32_t level,
                              void *stream);
/* out = Rot(in, k). */
mmfhe_status mmfhe_ct_rotate(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *in, size_t batch,
                             uint32_t level, int32_t k, void *stream);
/* outs[i] = Rot(in, ks[i]) sharing one ModUp (hoisting); k = 0 copies. */
mmfhe_status mmfhe_ct_rotate_hoisted(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *const *outs,
                                     const uint64_t *in, size_t batch, uint32_t level, const int32_t *ks,
                                     size_t num_k, void *stream);
/* Digit decomposition + ModUp of d (uint64[batch][level+1][N]):
 * out uint64[batch][beta][level+1+K][N] (coefficient form), beta = number of
 * digits at this level; row order q_0..q_level, p_0..p_{K-1}. */
mmfhe_status mmfhe_modup(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *d, size_t batch, uint32_t level, void *stream);
/* Key switch of d (uint64[batch][level+1][N]): out = uint64[batch][2][level+1][N]
 * = ModDown(ModUp(d) . key).  which = 0: relinearization key; which = 1:
 * Galois key of `rotation` (no automorphism applied). */
mmfhe_status mmfhe_keyswitch(mmfhe_ctx *ctx, const mmfhe_keys *keys, int which, int32_t rotation, uint64_t *out,
                             const uint64_t *d, size_t batch, uint32_t level, void *stream);
/* Key switch that allocates nothing (the paper has no counterpart; this is a
 * library-level convenience).  Same result, word for word, as
 * mmfhe_keyswitch, for callers that must not allocate device memory during
 * a call: code running where cudaMalloc/cudaFree are not allowed (host
 * callbacks, paths that may not take the allocator's lock, runtimes that hand
 * all device memory to their own allocator at start-up).  d and out must be
 * 16-byte aligned DEVICE pointers (d uint64[batch][level+1][N] and out
 * uint64[batch][2][level+1][N], coefficient form); work is only enqueued on
 * `stream`.  Every intermediate lives in one fixed device array of
 * MMFHE_NOALLOC_SCRATCH_BYTES that the library holds on each GPU it runs on
 * until the process exits; a call that needs more (batch x rows of
 * (level+1) + beta (level+1+K) + 2 (level+1+K) + 4 (level+1), N words each)
 * returns BAD_ARG -- at N = 2^15, top level 11, K = 4, dnum = 3 that is one
 * ciphertext per call.  d and out must be memory of the context's own
 * device (BAD_ARG otherwise).  The first call on a context looks up the
 * array's device address (cudaGetSymbolAddress) with the context's device
 * current and keeps it in the context; make that first call before any
 * stream capture.  The address belongs to the device's primary CUDA context:
 * a device reset (cudaDeviceReset) invalidates it together with every other
 * device object of the mmfhe context, so destroy mmfhe contexts before a
 * reset and create new ones after it.  All calls share the array and it
 * keeps the last call's contents (no region needs clearing: every word read
 * is written earlier in the same call); calls that overlap on the GPU, on
 * any stream or context of the same device, race on it -- serialise them. */
#define MMFHE_NOALLOC_SCRATCH_BYTES (64u << 20)
mmfhe_status mmfhe_keyswitch_noalloc(mmfhe_ctx *ctx, const mmfhe_keys *keys, int which, int32_t rotation,
                                     uint64_t *out, const uint64_t *d, size_t batch, uint32_t level, void *stream);
/* Rotate-and-sum: x <- x + Rot(x, stride * 2^i) for i < log2(span). */
mmfhe_status mmfhe_ct_rotsum(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *in, size_t batch,
                             uint32_t level, int32_t stride, uint32_t span, void *stream);
/* BSGS diagonal product: out = sum_g Rot(sum_b D'_{g,b} (.) Rot(in, b*stride), g*n1*stride)
 * over the given diagonals delta = g*n1 + b (deltas[i], diags[i] = encoded
 * pre-rotated diagonal uint64[level+1][N]); baby steps hoisted; not rescaled. */
mmfhe_status mmfhe_ct_bsgs(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *in, size_t batch,
                           uint32_t level, int32_t stride, uint32_t n1, const uint32_t *deltas,
                           const uint64_t *const *diags, size_t num_diags, void *stream);

/* Double-hoisted BSGS product (Bossuat, Mouchet, Troncoso-Pastoriza and
 * Hubaux, Eurocrypt 2021, Sec. 4; the paper's hoisting of rotations, Sec.
 * "Discussion"): out = sum_g Rot( sum_{s, b} D'_{s,g,b} (.) Rot(in, b*stride
 * + offsets[s]), g*n1*stride ) over num_sets baby sets of the same input.
 * Diagonal i belongs to set set_of[i], delta = deltas[i] = g*n1 + b, diags[i]
 * = its pre-rotated encoding over Q_level (uint64[level+1][N], coefficient
 * form; the library extends it to the special primes from the centered
 * residues mod q_0, so coefficients must be below q_0 / 2 in magnitude,
 * BAD_ARG otherwise).  The baby rotations share one ModUp and stay in the
 * extended basis Q_level * P with their inner sums; a giant step brings only
 * the c1 of its inner sum down to Q_level for its key switch; one ModDown
 * ends the product.  The words differ from mmfhe_ct_bsgs's (other rounding).
 * Not rescaled.  Errors: BAD_ARG, LEVEL_MISMATCH, NOT_FOUND. */
mmfhe_status mmfhe_ct_bsgs_dh(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *in, size_t batch,
                              uint32_t level, int32_t stride, uint32_t n1, uint32_t num_sets, const int32_t *offsets,
                              const uint32_t *set_of, const uint32_t *deltas, const uint64_t *const *diags,
                              size_t num_diags, void *stream);

/* ------------------------------------------------------------------------
 * Circuits (plans).  A plan holds a circuit's public configuration
 * (Sec. "Leakage Profile": R, F, filter order, Taylor order, ...) and its
 * encoded public constants (FIR taps, DFT rows, masks) resident on device.
 * ---------------------------------------------------------------------- */
#define MMFHE_CIRCUIT_FIR_DFT 1 /* 64-tap bandpass FIR + windowed fftshifted DFT on every bin */
#define MMFHE_CIRCUIT_VITAL 2   /* vital-sign chain K1->K2 | K4->K5->K7->K3->|X|^2->sharpen->avg */
#define MMFHE_CIRCUIT_FC 3      /* polynomial network: dense layers with a square after each but the last */
/* The vital chain with per-frame packing (the paper's slow baseline, Sec.
 * "Packing"): one ciphertext per frame and part, range bin r in slot r.
 * Inputs per window: stream 1 frames t = 0..F-1 as (Re, Im), then stream 2
 * alike (4F ciphertexts at the top level).  Same formulas, level schedule and
 * outputs as MMFHE_CIRCUIT_VITAL (third order only), values in slot 0. */
#define MMFHE_CIRCUIT_VITAL_PER_FRAME 4
/* The gesture chain (paper Sec. "Example Pipelines", Encrypted Dynamic Radar
 * Classification; depth 11 per Table 1): per frame K3 windowed fftshifted
 * Doppler DFT over the D chirps (Eq. K3, block-diagonal BSGS), K1 power, K6
 * notch (zero on Doppler bins floor(D/2)..ceil(D/2)), soft power w = p^4,
 * feature p w; sum over frames; FC1 (reads every feature slot) + bias +
 * square, FC2 + square, FC3.  Slot of antenna a, range bin r, chirp c within
 * a frame: a R D + r D + c; ARD_pad = 2^ceil(log2(A R D)); k = (N/2) /
 * ARD_pad frames per ciphertext, frame f in pair f / k at offset
 * (f mod k) ARD_pad.  Window input: pairs = ceil(F / k) ciphertext pairs,
 * (Re, Im) of pair 0, then pair 1, ... at the top level (2 pairs inputs);
 * with complex_slots one ciphertext of Re + i Im per pair (pairs inputs).
 * Output: one ciphertext at level top - 11, logits in slots 0..classes-1 of
 * every fc_width-slot period.  Fields: bins = R, frames = F, antennas = A,
 * chirps = D, fc_width = the FC slot period (a power of two <= ARD_pad,
 * above every FC width), fc_dims = {A R D, d_1, d_2, classes}, input_scale =
 * the encryption scale (sets the scale of FC1's bias vector). */
#define MMFHE_CIRCUIT_GESTURE 5

typedef struct mmfhe_circuit_config {
    uint32_t kind;             /* MMFHE_CIRCUIT_* */
    uint32_t bins;             /* R range bins */
    uint32_t frames;           /* F frames per window */
    uint32_t fs_mhz;           /* frame rate in mHz */
    uint32_t taps;             /* FIR taps */
    uint32_t taylor_order;     /* 1 or 3 (VITAL) */
    uint32_t num_bands;        /* FIR_DFT: 1; VITAL: 2 (respiration, heart) */
    uint32_t band_lo_mhz[2];
    uint32_t band_hi_mhz[2];
    double dft_gain[2];        /* VITAL: public per-band DFT gains (both 0: defaults
                                  30, 1 for third order; 1.5, 0.2 for first order) */
    /* FC (the paper's fully connected network with square activations):
     * bins = D, the slot period of every layer (a power of two), taps = the
     * number of layers L (1..8), fc_dims[0..L] = the widths d_0 (inputs) ..
     * d_L (outputs), all below D.  Slot D-1 of every period holds the
     * constant 1 (biases = column D-1; row D-1 keeps the constant).  Input:
     * one ciphertext at the top level holding the inputs in slots 0..d_0-1
     * and 1 in slot D-1 of every period; output at level top - 2L + 1. */
    uint32_t fc_dims[9];
    /* GESTURE only (zero otherwise) */
    uint32_t antennas;         /* A virtual antennas */
    uint32_t chirps;           /* D chirps per frame = Doppler bins */
    uint32_t fc_width;         /* slot period of the FC layers */
    uint32_t complex_slots;    /* GESTURE and VITAL: 1 = Re + i Im in one ciphertext of complex slots
                                  (half the inputs; |z|^2 as z conj(z), so the conjugation key
                                  MMFHE_ROT_CONJ is needed).  GESTURE: one input per pair, K3 one
                                  complex product.  VITAL: stream 1 then stream 2, one ciphertext
                                  per group; K4 gives I + i Q, one FIR product per band, K7 from
                                  w = Z conj(Z at t-1), the phase from w^3 - conj(w^3) = 2i Im(w^3) */
    double input_scale;        /* encryption scale Delta of the inputs */
    /* GESTURE: the feature map between the notch and the frame accumulation.
     * MMFHE_FEATURE_POWER (0): the paper's soft power gamma = 4 and feature
     * weighting, f = p w with w = p^4 (degree 5, three levels; Table 1).
     * MMFHE_FEATURE_LEARNED (1): f = a p + b p^2 with (a, b) = feature_coef,
     * learned together with the network (one level): the chain needs two
     * levels less, so its parameter set has two Q primes less.  Output level
     * top - 11 (power) or top - 9 (learned). */
    uint32_t feature_map;
    double feature_coef[2];
} mmfhe_circuit_config;
#define MMFHE_FEATURE_POWER 0
#define MMFHE_FEATURE_LEARNED 1

/* Constant tags of mmfhe_const_key.tag */
#define MMFHE_CONST_IDX 1   /* VITAL side branch: bin index of group g's bins at the start of its packed
                               frame block (-g mod G'); VITAL_PER_FRAME: bin r in slot r */
#define MMFHE_CONST_ONE 2   /* the same positions holding 1 */
#define MMFHE_CONST_FIR 3   /* FIR diagonal delta=`index` of band `band` (pre-rotated) */
#define MMFHE_CONST_DRE 4   /* VITAL DFT rows of band `band`, diagonal `index`: Re X_k in row k, Im X_k in
                               row k + F_pad/2 (both bands run in one BSGS product) */
#define MMFHE_CONST_DIM 5   /* reserved (no current plan uses it) */
#define MMFHE_CONST_FW 6    /* frequency weights f_k (Hz) of band `band` */
#define MMFHE_CONST_FONE 7  /* band indicator of band `band` */
#define MMFHE_CONST_DFT_C 8  /* FIR_DFT: C = Re W diagonal `index` */
#define MMFHE_CONST_DFT_S 9  /* FIR_DFT: S = Im W */
#define MMFHE_CONST_DFT_MS 10 /* FIR_DFT: -S */
#define MMFHE_CONST_FCW 11   /* FC: diagonal `index` of layer `band` (pre-rotated); GESTURE layer 0:
                                extended diagonal `index` (0..fc_width-1) of FC1 */
#define MMFHE_CONST_GDFT_C 12  /* GESTURE: Re W Doppler diagonal delta = index - D (pre-rotated) */
#define MMFHE_CONST_GDFT_S 13  /* GESTURE: Im W */
#define MMFHE_CONST_GDFT_MS 14 /* GESTURE: -Im W */
#define MMFHE_CONST_NOTCH 15   /* GESTURE: notch mask m[c] on every active slot */
#define MMFHE_CONST_FCB 16     /* GESTURE: FC1 bias b[s mod fc_width], 1 in slot fc_width-1, encoded at
                                  the scale of FC1's rescaled output */
#define MMFHE_CONST_GDFT_W 17  /* GESTURE with complex slots: the complex W Doppler diagonal delta =
                                  index - D (pre-rotated), encoded as complex slots */
#define MMFHE_CONST_NOTCH_B 18 /* GESTURE, learned feature map: b times the notch mask */
#define MMFHE_CONST_FEAT_A 19  /* GESTURE, learned feature map: a on every active slot, encoded at the
                                  scale of the notched power (one level below the notch) */
#define MMFHE_CONST_PMASK 20   /* VITAL side branch: 1 on the first F_pad / G' frames of every bin slot
                                  (G' = groups rounded up to a power of two), the block each group's
                                  frame sums are kept in before the groups are packed */

typedef struct mmfhe_const_key {
    uint32_t tag, band, index, level;
} mmfhe_const_key;

typedef struct mmfhe_plan mmfhe_plan;
mmfhe_status mmfhe_plan_create(mmfhe_ctx *ctx, const mmfhe_circuit_config *cfg, size_t cfg_size, mmfhe_plan **out);
mmfhe_status mmfhe_plan_destroy(mmfhe_plan *plan);
/* The constants the circuit needs, in a fixed order (index 0..count-1). */
mmfhe_status mmfhe_plan_num_consts(const mmfhe_plan *plan, uint32_t *count);
mmfhe_status mmfhe_plan_const_key(const mmfhe_plan *plan, uint32_t i, mmfhe_const_key *out);
/* Install pre-encoded constant i (coefficient form, uint64[level+1][N]). */
mmfhe_status mmfhe_plan_set_const(mmfhe_plan *plan, uint32_t i, const uint64_t *words);
/* Copy constant i back in coefficient form (uint64[level+1][N]); NOT_FOUND if unset. */
mmfhe_status mmfhe_plan_get_const(const mmfhe_plan *plan, uint32_t i, uint64_t *words);
/* Design and encode every constant with the library's own FP64 design
 * (Hamming-windowed-sinc taps, Hann-windowed DFT rows) and encoder. */
mmfhe_status mmfhe_plan_encode_consts(mmfhe_plan *plan);
/* FC plans: encode layer `layer` from its D x D matrix W (row-major,
 * y = W v on every period; only the structurally present diagonals are
 * stored).  The constants of an FC plan are learned, so
 * mmfhe_plan_encode_consts returns BAD_ARG for it.  GESTURE plans: layer 0
 * is fc_width x (A R D + 1) (column j < A R D weighs feature slot j, the
 * last column is the bias; row fc_width-1 is ignored: that slot becomes the
 * constant 1), layers 1 and 2 are fc_width x fc_width as for FC plans;
 * mmfhe_plan_encode_consts encodes the Doppler DFT and notch constants. */
mmfhe_status mmfhe_plan_set_fc_layer(mmfhe_plan *plan, uint32_t layer, const double *W);
/* Per-frame plans: the public scalar constants (count from
 * mmfhe_plan_num_scalars), in this order: per band the FIR taps h[0..taps);
 * per band, per DFT bin k, the coefficients g w[t] cos(2 pi k t / F) for
 * t = 1..F-1 then -g w[t] sin(2 pi k t / F) (g = the band gain / 3, w =
 * Hann); per band, per bin k, the frequency k fs / F in Hz.  A scalar c
 * multiplies as the constant polynomial round(q_l c) at level l.  The plan
 * starts with the library's FP64 design; set_scalars replaces it. */
mmfhe_status mmfhe_plan_num_scalars(const mmfhe_plan *plan, uint32_t *count);
mmfhe_status mmfhe_plan_get_scalars(const mmfhe_plan *plan, double *out, uint32_t capacity);
mmfhe_status mmfhe_plan_set_scalars(mmfhe_plan *plan, const double *values, uint32_t count);
/* Rotation amounts whose Galois keys the plan needs (ascending, in [0, N/2);
 * MMFHE_ROT_CONJ first when the circuit conjugates). */
mmfhe_status mmfhe_plan_rotations(const mmfhe_plan *plan, int32_t *out, uint32_t capacity, uint32_t *count);
/* Input/output shape: ciphertexts per window in and out, and the level of
 * every output ciphertext (levels capacity 16).  Window input layout:
 * uint64[n_in][2][L+1][N]; output: the n_out ciphertexts back to back, each
 * uint64[2][level_i+1][N]. */
mmfhe_status mmfhe_plan_io(const mmfhe_plan *plan, uint32_t *n_in, uint32_t *n_out, uint32_t *out_levels);
/* Where the client reads a vital plan's results after decryption: for
 * num_r, den_r, num_RR, den_RR, num_HR, den_HR (the target bin's weighted
 * average and each band's, Sec. "Example Pipelines"), the output ciphertext
 * index and the slot.  The three outputs are the side branch (num_r in slot
 * 0, den_r in slot r_c) and one ciphertext per band (num_b in slot b, den_b
 * in slot span_b r_c + b, span_b the band's power-of-two bin span), so each
 * band's sums stay apart from the other band's.  *count = 6 for VITAL plans,
 * 0 for the others; BAD_ARG when capacity is below the count. */
mmfhe_status mmfhe_plan_readout(const mmfhe_plan *plan, uint32_t *out_index, uint32_t *slot, uint32_t capacity,
                                uint32_t *count);

/* Evaluate the plan's circuit on `batch` windows.  keys[w], in_cts[w] and
 * out_cts[w] belong to window w; windows with the same keys object are
 * evaluated together, every launch covering all of them.  Errors: BAD_ARG,
 * NOT_FOUND (missing key/constant), CUDA, OUT_OF_MEMORY.  batch = 0 is a
 * no-op. */
mmfhe_status mmfhe_eval(mmfhe_ctx *ctx, const mmfhe_plan *plan, mmfhe_keys *const *keys,
                        const uint64_t *const *in_cts, size_t batch, uint64_t *const *out_cts, void *stream);
/* mmfhe_eval restricted to MMFHE_CIRCUIT_VITAL (and _PER_FRAME) plans (paper Sec. "Example
 * Pipelines", Encrypted Vital Signs; depth per Table 1).  Window inputs:
 * stream 1 (K1) G groups x (Re, Im), then stream 2 (K4) G x (Re, Im), at the
 * top level.  VITAL outputs: three ciphertexts holding num_r, den_r (target
 * bin), num_RR, den_RR, num_HR, den_HR (frequency-weighted sums in Hz; BPM =
 * 60 num/den) at the slots mmfhe_plan_readout gives; VITAL_PER_FRAME: six
 * ciphertexts, those values in slot 0 in that order. */
mmfhe_status mmfhe_eval_vital(mmfhe_ctx *ctx, const mmfhe_plan *plan, mmfhe_keys *const *keys,
                              const uint64_t *const *in_cts, size_t batch, uint64_t *const *out_cts, void *stream);

/* ------------------------------------------------------------------------
 * What crosses the trust boundary, serialized and checked (paper Sec.
 * "System Design": the client uploads its ciphertexts and its public
 * evaluation keys rlk and gk once at enrollment; the cloud returns
 * ciphertexts).  Blobs and headers carry the fingerprint of the parameter
 * set they were made for, so an object made for another parameter set is
 * refused (PARAM_MISMATCH) instead of being evaluated into garbage.
 * ---------------------------------------------------------------------- */
/* Parameter-set fingerprint: word-wise FNV-1a (h = offset basis
 * 0xcbf29ce484222325; for every 64-bit word w: h = (h xor w) *
 * 0x100000001b3 mod 2^64) over the words log_n, num_q, num_p, dnum,
 * q_0..q_L, p_0..p_{K-1}.  Host only.  Errors: BAD_ARG. */
mmfhe_status mmfhe_params_hash(const mmfhe_params *params, uint64_t *out);

/* 32-byte header of one ciphertext: its level, log2 of its scale and the
 * fingerprint of its parameter set. */
#define MMFHE_CT_MAGIC 0x54434D4Du   /* bytes "MMCT" */
typedef struct mmfhe_ct_header {
    uint32_t magic;        /* MMFHE_CT_MAGIC */
    uint16_t version;      /* 1 */
    uint16_t reserved0;
    uint32_t level;        /* l: the ciphertext has l+1 limbs */
    uint32_t reserved1;
    double log2_scale;     /* log2 of the scale Delta the message is multiplied by */
    uint64_t params_hash;  /* mmfhe_params_hash of its parameter set */
} mmfhe_ct_header;
/* Fill a header (host only; what a client attaches to each ciphertext it
 * encrypts at `level` and `scale`).  Errors: BAD_ARG, LEVEL_MISMATCH. */
mmfhe_status mmfhe_ct_header_make(const mmfhe_params *params, uint32_t level, double scale, mmfhe_ct_header *out);

/* mmfhe_eval with a header per ciphertext.  in_hdrs[w] holds the n_in
 * headers of window w's inputs (mmfhe_plan_io), out_hdrs[w] receives the
 * n_out headers of its outputs (level, tracked log2 scale, fingerprint).
 * Checked before any work is queued: BAD_BLOB (not a header), PARAM_MISMATCH
 * (another parameter set; keys or plan of another context; GESTURE plans:
 * a scale other than the plan's input_scale), LEVEL_MISMATCH (an input not
 * at the top level), BAD_ARG (inputs of one call at different scales).
 * Otherwise as mmfhe_eval; the words computed do not depend on the scale. */
mmfhe_status mmfhe_eval_checked(mmfhe_ctx *ctx, const mmfhe_plan *plan, mmfhe_keys *const *keys,
                                const mmfhe_ct_header *const *in_hdrs, const uint64_t *const *in_cts, size_t batch,
                                mmfhe_ct_header *const *out_hdrs, uint64_t *const *out_cts, void *stream);

/* Blobs: little-endian 64-bit words in host memory, 8-byte aligned.
 *   word 0  magic 0x424C424548464D4D (bytes "MMFHEBLB")
 *   word 1  version (1) in the low 32 bits, kind in the high 32 bits
 *   word 2  mmfhe_params_hash of the parameter set
 *   word 3  body length in words (W)
 *   words 4 .. 4+W-1  body
 *   word 4+W  checksum: word-wise FNV-1a (as in mmfhe_params_hash) of words 0 .. 3+W
 * MMFHE_BLOB_KEYS body: count C (the relinearization key, then C-1 Galois
 * keys), the words per key dnum*2*(L+1+K)*N, C key ids (0 for the
 * relinearization key, then a rotation in [1, N/2) or MMFHE_ROT_CONJ, as
 * signed 64-bit words), then the C keys, each in the layout of
 * mmfhe_keys_set_relin.
 * MMFHE_BLOB_PLAN body: sizeof(mmfhe_circuit_config), the configuration's
 * bytes zero-padded to whole words, the constant count C, C levels, then the
 * C constants in the plan's order (mmfhe_plan_const_key), constant i as
 * uint64[level_i+1][N] in coefficient form. */
#define MMFHE_BLOB_KEYS 1u
#define MMFHE_BLOB_PLAN 2u
/* Serialize a user's evaluation keys (host only): the relinearization key and
 * n_rot Galois keys (layouts as mmfhe_keys_set_*).  out == NULL: *size gets
 * the blob's size in bytes and nothing is written.  Errors: BAD_ARG (null
 * key, rotation 0, capacity too small), BAD_BLOB (a residue not below its
 * prime). */
mmfhe_status mmfhe_keys_blob_write(const mmfhe_params *params, const uint64_t *relin, uint32_t n_rot,
                                   const int32_t *rotations, const uint64_t *const *galois, void *out, size_t capacity,
                                   size_t *size);
/* Serialize a plan: its configuration and `count` encoded constants at the
 * given levels (host only; out == NULL: size only).  Errors: BAD_ARG,
 * LEVEL_MISMATCH, BAD_BLOB (a residue not below its prime). */
mmfhe_status mmfhe_plan_blob_write(const mmfhe_params *params, const mmfhe_circuit_config *cfg, size_t cfg_size,
                                   uint32_t count, const uint32_t *levels, const uint64_t *const *consts, void *out,
                                   size_t capacity, size_t *size);
/* Validate a blob against a parameter set without a GPU (what mmfhe_keys_load
 * and mmfhe_plan_load check before they upload anything): BAD_BLOB for a
 * wrong magic, version or kind, a truncated or oversized blob, inconsistent
 * counts or sizes, a bad key id, a residue not below its prime, or a
 * checksum mismatch; PARAM_MISMATCH for another parameter set; BAD_ARG for a
 * null, unaligned or device pointer.  *kind (nullable) gets the blob's kind. */
mmfhe_status mmfhe_blob_check(const mmfhe_params *params, const void *blob, size_t size, uint32_t *kind);
/* Make a serialized key set resident (enrollment, paper Sec. "System
 * Design"): validated as mmfhe_blob_check against the context's parameters,
 * then uploaded; the blob is not referenced after the call.  Errors as
 * mmfhe_blob_check, plus BAD_BLOB (a rotation key twice), OUT_OF_MEMORY,
 * CUDA.  Release with mmfhe_keys_unload. */
mmfhe_status mmfhe_keys_load(mmfhe_ctx *ctx, uint64_t user_id, const void *blob, size_t size, mmfhe_keys **out);
/* Create a plan from a serialized configuration and its encoded constants:
 * validated as mmfhe_blob_check, then BAD_BLOB if the configuration is
 * invalid or its plan has another constant count or levels.  Release with
 * mmfhe_plan_destroy. */
mmfhe_status mmfhe_plan_load(mmfhe_ctx *ctx, const void *blob, size_t size, mmfhe_plan **out);

/* ------------------------------------------------------------------------
 * Autotuner (no counterpart in the paper).  The NTT passes and the key inner
 * product come in tile-shape variants: columns per CTA of the strided pass
 * (8 or 16), threads per CTA of the contiguous pass (128 or 256), windows per
 * thread of the key inner product (1, 2, 4, 8) and converted rows per CTA of
 * the fused ModUp / ModDown strided passes (1, 2, 4).  mmfhe_autotune times
 * every variant on `batch` ciphertexts at `level` (NTT: forward + inverse of
 * all their rows; key inner product: a rotation's digits and key) and keeps
 * the fastest for every later call on the context.  Every variant computes
 * the same words.  Errors: BAD_ARG (batch 0 or level above the top), CUDA.
 * ---------------------------------------------------------------------- */
typedef struct mmfhe_tuning {
    uint32_t ntt_cols_width;     /* 8 or 16 */
    uint32_t ntt_rows_threads;   /* 128 or 256 */
    uint32_t keyip_windows;      /* 1, 2, 4 or 8 */
    uint32_t conv_rows;          /* rows per CTA of the fused ModUp / ModDown conversions: 1, 2 or 4 */
    float ntt_ms[4];             /* last autotune, ms: (8,128), (8,256), (16,128), (16,256) */
    float keyip_ms[4];           /* last autotune, ms: window groups 1, 2, 4, 8 */
    float conv_ms[3];            /* last autotune, ms: ModUp + ModDown with 1, 2, 4 rows per CTA */
    uint32_t keyip_fused;        /* 0 (default): a key switch's inner-product words are stored by their own
                                    kernel; 1: formed inside the ModDown passes that consume them (P rows in
                                    the inverse NTT's load, Q rows in the combine) and never stored, which
                                    measures slower on B300.  Same words either way.  The autotuner leaves
                                    it unchanged. */
    uint32_t keyip_pipe;         /* 1: the key inner product of a batch sharing one key walks its windows
                                    with the next group's digit words copied into shared memory while
                                    the current group's products run (key switches with at most 4
                                    digits); same words.  Picked by the autotuner. */
    float keyip_pipe_ms[4];      /* last autotune, ms: pipelined, window groups 1, 2, 4, 8 */
    uint32_t combine_pipe;       /* 1: the ModDown combine runs on persistent CTAs that load the next tile
                                    while the current one is transformed and combined; same words.
                                    Picked by the autotuner. */
    float combine_pipe_ms[3];    /* last autotune, ms: ModUp + ModDown with the pipelined combine, rows
                                    1, 2, 4 */
} mmfhe_tuning;
mmfhe_status mmfhe_autotune(mmfhe_ctx *ctx, uint32_t batch, uint32_t level, mmfhe_tuning *out);
mmfhe_status mmfhe_tuning_get(const mmfhe_ctx *ctx, mmfhe_tuning *out);
/* Set the variants explicitly (timings ignored); BAD_ARG for other values. */
mmfhe_status mmfhe_tuning_set(mmfhe_ctx *ctx, const mmfhe_tuning *in);

/* ------------------------------------------------------------------------
 * Polynomial network training (plaintext, FP32, on the GPU; no counterpart
 * in the paper beyond its learned FC weights).  Trains z_l = W_l [a_{l-1}; 1],
 * a_l = z_l + alpha z_l^2 after every layer but the last, softmax
 * cross-entropy, momentum SGD (0.9) on mini-batches of `batch` rows, inputs
 * standardised (spread floored at 5 % of the largest input's; folded back,
 * so the weights act on raw inputs).  X: host
 * float [n][dims[0]]; labels: host int32 in [0, dims[layers]); weights out:
 * host float, W_0 [d_1][d_0 + 1], W_1 [d_2][d_1 + 1], ... back to back (last
 * column = bias).  *train_accuracy (nullable): argmax accuracy on X. */
mmfhe_status mmfhe_train_poly_net(mmfhe_ctx *ctx, const float *X, const int32_t *labels, uint64_t n,
                                  const uint32_t *dims, uint32_t layers, float alpha, uint32_t epochs,
                                  uint32_t batch, float lr, uint64_t seed, float *weights, float *train_accuracy);
/* Host only.  The same network with pure squares (the form of
 * MMFHE_CIRCUIT_FC): z + alpha z^2 = alpha (z + 1/(2 alpha))^2 - 1/(4 alpha),
 * the shift folded into each hidden layer's bias and alpha, -1/(4 alpha) into
 * the next layer.  mats out: layers x width x width doubles, row-major, bias
 * in column width-1, mats[l][width-1][width-1] = 1.  BAD_ARG if a width is
 * not below `width` or `width` is not a power of two. */
mmfhe_status mmfhe_fold_poly_net(const uint32_t *dims, uint32_t layers, float alpha, const float *weights,
                                 uint32_t width, double *mats);
/* Host only.  The same folding for a network whose input width d_0 may reach
 * or exceed `width` (a GESTURE plan's FC1 reads every feature slot): layer 0
 * out: first = width x (d_0 + 1) doubles (bias in column d_0, entry
 * [width-1][d_0] = 1); layers 1.. out: mats = (layers-1) x width x width as
 * in mmfhe_fold_poly_net.  BAD_ARG as there, for d_1.. only. */
mmfhe_status mmfhe_fold_poly_net_wide(const uint32_t *dims, uint32_t layers, float alpha, const float *weights,
                                      uint32_t width, double *first, double *mats);

/* ------------------------------------------------------------------------
 * Word-size ablation (no counterpart in the paper, whose CKKS library fixes
 * the word size): the same negacyclic NTT on 32-bit RNS words, primes below
 * 2^30, one shared-memory pass per row (a 32-bit row of N <= 2^15 words fits
 * in shared memory).  Output order and convention as mmfhe_ntt (bit-reversed
 * evaluation order; the inverse takes it back and multiplies by N^-1).
 * ---------------------------------------------------------------------- */
typedef struct mmfhe_ntt32 mmfhe_ntt32;
/* Host only: the `count` largest primes below 2^bits that are 1 mod 2N,
 * descending.  BAD_ARG: log_n outside 10..15, bits outside log_n+2..30, or
 * too few such primes. */
mmfhe_status mmfhe_ntt32_select_primes(uint32_t log_n, uint32_t bits, uint32_t count, uint32_t *out);
/* Twiddle tables for num_primes (1..64) primes on `device`.  BAD_BLOB: a
 * prime not below 2^30, not 1 mod 2N or not prime. */
mmfhe_status mmfhe_ntt32_create(uint32_t log_n, const uint32_t *primes, uint32_t num_primes, int device,
                                mmfhe_ntt32 **out);
/* In place on num_rows rows of N words, row r under prime r mod num_primes,
 * inputs reduced mod their prime.  rows: device (16-byte aligned) or host
 * memory (staged through the device; the call then waits for the stream). */
mmfhe_status mmfhe_ntt32_run(mmfhe_ntt32 *p, uint32_t *rows, size_t num_rows, int inverse, void *stream);
mmfhe_status mmfhe_ntt32_destroy(mmfhe_ntt32 *p);

/* ------------------------------------------------------------------------
 * Batching runtime.  The paper evaluates windows one call at a time (its
 * batched packing fills the slots of one window's ciphertexts); these calls
 * add a runtime around mmfhe_eval for many uneven windows: CUDA-graph replay
 * of a whole evaluation, and a batcher that groups windows by frame count and
 * key set.  Not thread-safe per context: one host thread drives a context.
 * ---------------------------------------------------------------------- */
/* CUDA graph of one mmfhe_eval call on fixed DEVICE buffers (in_cts[w],
 * out_cts[w], 16-byte aligned).  The graph owns a private pool for every
 * intermediate, so a replay shares no scratch with other work; keys, plan and
 * the buffers must outlive the graph.  Capture runs the evaluation once
 * (filling the pool; its outputs are written) on an internal stream, waits
 * for it, then records a second run.  Replay: mmfhe_graph_launch on any
 * stream; one replay of a graph at a time.  Errors: BAD_ARG (host buffer,
 * batch 0), NOT_FOUND, CUDA, OUT_OF_MEMORY. */
typedef struct mmfhe_graph mmfhe_graph;
mmfhe_status mmfhe_graph_capture(mmfhe_ctx *ctx, const mmfhe_plan *plan, mmfhe_keys *const *keys,
                                 const uint64_t *const *in_cts, size_t batch, uint64_t *const *out_cts,
                                 mmfhe_graph **out);
mmfhe_status mmfhe_graph_launch(mmfhe_graph *graph, void *stream);
/* Kernels one replay launches, and device bytes the graph holds. */
mmfhe_status mmfhe_graph_info(const mmfhe_graph *graph, uint64_t *kernels, uint64_t *bytes);
mmfhe_status mmfhe_graph_destroy(mmfhe_graph *graph);

typedef struct mmfhe_batcher_config {
    uint32_t max_batch;           /* windows per launch, 1..256 */
    uint32_t use_graphs;          /* nonzero: one captured graph per (frames, keys, batch size), replayed */
    uint64_t plan_budget_bytes;   /* device bytes of cached plans (least recently used evicted); 0: no limit */
    uint64_t graph_budget_bytes;  /* device bytes of cached graphs and their staging; 0: no limit */
} mmfhe_batcher_config;
typedef struct mmfhe_batcher_stats {
    uint64_t windows;             /* windows evaluated */
    uint64_t batches;             /* evaluations (graph replays or mmfhe_eval batches) */
    uint64_t graph_replays;
    uint64_t graphs_captured, graphs_evicted;
    uint64_t plans_created, plans_evicted;
    uint64_t plan_bytes, graph_bytes;   /* currently held */
} mmfhe_batcher_stats;
typedef struct mmfhe_batcher mmfhe_batcher;
/* base: the circuit every window runs (size = sizeof(mmfhe_circuit_config));
 * a window of F frames runs it with frames = F (its own plan, created and
 * encoded with mmfhe_plan_encode_consts on first use). */
mmfhe_status mmfhe_batcher_create(mmfhe_ctx *ctx, const mmfhe_circuit_config *base, size_t base_size,
                                  const mmfhe_batcher_config *cfg, mmfhe_batcher **out);
/* The plan for `frames` (created on first use).  Owned by the batcher: valid
 * until the batcher is destroyed or the plan is evicted by a later call. */
mmfhe_status mmfhe_batcher_plan(mmfhe_batcher *b, uint32_t frames, const mmfhe_plan **out);
/* Queue one window: input [n_in][2][L+1][N] coefficient form, output as for
 * mmfhe_eval, host or device memory.  Nothing runs until mmfhe_batcher_flush. */
mmfhe_status mmfhe_batcher_submit(mmfhe_batcher *b, mmfhe_keys *keys, uint32_t frames, const uint64_t *in,
                                  uint64_t *out);
/* Evaluate every queued window: windows with equal (frames, keys) are split
 * into batches of at most max_batch in submission order.  Outputs in host
 * memory are complete on return; device outputs are ordered on `stream`. */
mmfhe_status mmfhe_batcher_flush(mmfhe_batcher *b, void *stream);
/* Drop every graph that uses `keys` (call before mmfhe_keys_unload). */
mmfhe_status mmfhe_batcher_forget_keys(mmfhe_batcher *b, const mmfhe_keys *keys);
mmfhe_status mmfhe_batcher_stats_get(const mmfhe_batcher *b, mmfhe_batcher_stats *out);
mmfhe_status mmfhe_batcher_destroy(mmfhe_batcher *b);

/* ------------------------------------------------------------------------
 * Serving loop (no counterpart in the paper's text: a multi-user runtime
 * around the evaluator).  Windows from many users arrive at any time
 * (mmfhe_server_submit, thread-safe); a worker thread admits them into
 * batches of equal frame count (users mixed: each window is key-switched with
 * its own user's keys) as soon as one of `streams` slots is free
 * (continuous batching: windows that arrive while others run join the next
 * batch), runs each batch on its slot's CUDA stream with the slot's private
 * memory pool (batches on different slots overlap on the device), and keeps
 * users' evaluation keys resident under key_budget_bytes, reloading an
 * evicted user's keys from the words registered with mmfhe_server_add_user
 * (least recently used first; keys of a running batch are never evicted).
 * While a server exists, its worker thread is the only user of the context.
 * ---------------------------------------------------------------------- */
typedef struct mmfhe_server_config {
    uint32_t max_batch;           /* windows per batch, 1..256 */
    uint32_t streams;             /* concurrent batches, 1..8 */
    uint64_t key_budget_bytes;    /* device bytes of resident key sets; 0: no limit */
    uint32_t batch_wait_us;       /* a free slot waits up to this long for a batch to fill (0: dispatch at once) */
} mmfhe_server_config;
typedef struct mmfhe_server_stats {
    uint64_t submitted, completed, failed;
    uint64_t batches;             /* dispatched batches */
    uint64_t key_loads, key_evictions;
    uint64_t keys_resident, key_bytes;
    double mean_batch;            /* windows per batch */
    double p50_ms, p99_ms;        /* submit -> output written, completed windows */
    double windows_per_s;         /* completed / (last completion - first submission) */
    uint64_t cancelled;           /* requests cancelled while queued */
} mmfhe_server_stats;
typedef struct mmfhe_server mmfhe_server;
/* base: the circuit every window runs (one plan per frame count, created on
 * first use).  The worker thread starts here. */
mmfhe_status mmfhe_server_create(mmfhe_ctx *ctx, const mmfhe_circuit_config *base, size_t base_size,
                                 const mmfhe_server_config *cfg, mmfhe_server **out);
/* Register a user's evaluation keys: the relinearization key and n_rot
 * Galois keys (layouts as mmfhe_keys_set_*), host or device words that the
 * caller keeps unchanged until mmfhe_server_destroy.  Nothing is uploaded
 * until the user's first window runs.  BAD_ARG if user_id is registered. */
mmfhe_status mmfhe_server_add_user(mmfhe_server *s, uint64_t user_id, const uint64_t *relin, const int32_t *rotations,
                                   const uint64_t *const *galois, uint32_t n_rot);
/* Learned layers (FC and GESTURE servers): layer `layer` as for
 * mmfhe_plan_set_fc_layer, `count` doubles (FC: D x D; GESTURE: layer 0
 * fc_width x (A R D + 1), layers 1-2 fc_width x fc_width), copied and applied
 * to every plan the server creates.  Call before the first submit (BUSY
 * after); BAD_ARG for another circuit, layer or size. */
mmfhe_status mmfhe_server_set_fc_layer(mmfhe_server *s, uint32_t layer, const double *W, size_t count);
/* Caller-encoded public constants: `count` words (coefficient form,
 * uint64[level+1][N], the plan's constant `index` as listed by
 * mmfhe_plan_const_key for a plan of `frames` frames) replace the library's
 * own encoding of that constant in the plan the server creates for that
 * frame count (for a client that designs its constants itself, and for
 * parity tests that install an independent encoding).  Copied; call before
 * the first submit (BUSY after).  A wrong index or size makes the windows of
 * that frame count fail with BAD_ARG. */
mmfhe_status mmfhe_server_set_const(mmfhe_server *s, uint32_t frames, uint32_t index, const uint64_t *words,
                                    size_t count);
/* Queue one window (input and output as for mmfhe_eval; host buffers should
 * be pinned for the copies to overlap).  *ticket identifies it.  NOT_FOUND
 * for an unknown user. */
mmfhe_status mmfhe_server_submit(mmfhe_server *s, uint64_t user_id, uint32_t frames, const uint64_t *in,
                                 uint64_t *out, uint64_t *ticket);
/* Cancel a window that is still queued: it is never dispatched, its output
 * is not written, and its wait returns CANCELLED.  A window already running on
 * the GPU (or complete) is not interrupted: BUSY.  NOT_FOUND for an unknown
 * ticket. */
mmfhe_status mmfhe_server_cancel(mmfhe_server *s, uint64_t ticket);
/* Wait up to timeout_ms for a window: OK (output written; *latency_ms =
 * submit -> completion), TIMEOUT, CANCELLED, or the status its batch failed
 * with. */
mmfhe_status mmfhe_server_wait(mmfhe_server *s, uint64_t ticket, uint32_t timeout_ms, double *latency_ms);
/* Wait up to timeout_ms until every submitted window has completed, failed
 * or been cancelled. */
mmfhe_status mmfhe_server_drain(mmfhe_server *s, uint32_t timeout_ms);
mmfhe_status mmfhe_server_stats_get(mmfhe_server *s, mmfhe_server_stats *out);
/* Stop the worker after the queued windows complete, free everything. */
mmfhe_status mmfhe_server_destroy(mmfhe_server *s);

/* ------------------------------------------------------------------------
 * Host-side helpers (no GPU needed).
 * ---------------------------------------------------------------------- */
/* Batched-packing layout (Sec. "Packing", batched): values[F][R] (real) ->
 * G slot vectors of N/2 doubles, slot(t, r) = t*R_c + r, F_pad = 2^ceil(log2 F),
 * R_c = (N/2)/F_pad, G = ceil(R/R_c).  out must hold G*N/2 doubles. */
mmfhe_status mmfhe_pack_window(uint32_t log_n, uint32_t frames, uint32_t bins, const double *values, double *out);
/* Encode a real slot vector (N/2 doubles) at `scale` into uint64[level+1][N]
 * (m = round(scale * tau^-1(z)), slot j <-> zeta^(5^j)). */
mmfhe_status mmfhe_encode(const mmfhe_params *params, const double *slots, double scale, uint32_t level, uint64_t *out);

#ifdef __cplusplus
}
#endif
#endif /* MMFHE_H */
