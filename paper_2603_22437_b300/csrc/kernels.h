// Kernel parameter structs and launcher declarations (kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mmfhe {

constexpr int MAX_ALPHA = 8;   // primes per key-switching digit
constexpr int MAX_DNUM = 8;    // key-switching digits

// Prime id of each row within a period (elementwise kernels).
struct PidList {
    uint8_t pid[MAXROWMAP];
};

// ModUp constants of one level (device pointers):
//   inv[j*MAX_ALPHA + u]     = (Qhat_{j,u})^-1 mod q_{j*alpha+u}   (+ Shoup)
//   m[(j*MAX_ALPHA + u)*MAXROWMAP + t] = Qhat_{j,u} mod prime(t)   (+ Shoup)
struct ModUpConsts {
    const uint64_t *inv, *inv_sh, *m, *m_sh;
    int pid_p0;
};

// ModDown constants (device pointers):
//   pinv[k] = Phat_k^-1 mod p_k; phat[k*MAX_Q + i] = Phat_k mod q_i;
//   pmod[i] = P mod q_i; Pinv[i] = P^-1 mod q_i  (all with Shoup companions)
struct ModDownConsts {
    const uint64_t *pinv, *pinv_sh, *phat, *phat_sh, *pmod, *pmod_sh, *Pinv, *Pinv_sh;
    int pid_p0;
};

// Rescale-by-q_l constants: qinv[i] = q_l^-1 mod q_i (+ Shoup), qmod[i] = q_l mod q_i.
struct RescaleConsts {
    const uint64_t *qinv, *qinv_sh, *qmod;
};

void k_launch_addsub(Context &c, uint64_t *out, const uint64_t *a, const uint64_t *b, size_t rows, const PidList &pl,
                     uint32_t period, bool sub, cudaStream_t st);
void k_launch_mul_int(Context &c, uint64_t *out, const uint64_t *a, size_t rows, const PidList &pl, uint32_t period,
                      long long k, cudaStream_t st);
void k_launch_mul_plain(Context &c, uint64_t *out, const uint64_t *a, const uint64_t *pt, size_t rows,
                        const PidList &pl, uint32_t period, bool acc, cudaStream_t st, bool mont = false);
// Convert rows of a view into (to) or out of Montgomery form, in place.
void k_launch_mont_convert(Context &c, const RowsView &v, bool to, cudaStream_t st);
// c0 rows of B ciphertexts at `level` += pt (Montgomery form, level+1 rows).
void k_launch_add_plain(Context &c, uint64_t *ct, const uint64_t *pt, int B, int level, cudaStream_t st);
// out[b] = sum_{g < G} in[b G + g], B output ciphertexts at `level`.
void k_launch_group_sum(Context &c, uint64_t *out, const uint64_t *in, int B, int G, int level, cudaStream_t st);
void k_launch_tensor(Context &c, uint64_t *d, const uint64_t *a, const uint64_t *b, int B, int level, long long coef,
                     bool acc, cudaStream_t st);
void k_launch_modup_bconv(Context &c, uint64_t *out, const uint64_t *coef, const uint64_t *deval, size_t deval_stride,
                          int B, int level, const ModUpConsts &mc, cudaStream_t st);
// u_h[b][t] = sum_j digit_j[b][t] (after the Galois permutation) * key_b[j][h][t]
// (key_b = key.k[0] for every window, or key.k[b] when key.n == B);
// rows of a digit inside its own primes come from `own` (window b, digit j,
// row t at own + b * own_stride + j * own_jstride + t * N).
void k_launch_keyip(Context &c, uint64_t *u, const uint64_t *digits, const uint64_t *own, size_t own_stride,
                    size_t own_jstride, const KeyPtrs &key, int B, int level, int beta, uint32_t galois,
                    cudaStream_t st);
void k_launch_moddown_bconv(Context &c, uint64_t *v, const uint64_t *u, int B, int level, const ModDownConsts &dc,
                            cudaStream_t st);
void k_launch_moddown_combine(Context &c, uint64_t *out, const uint64_t *u, const uint64_t *v, const uint64_t *add0,
                              const uint64_t *add1, size_t add_stride, uint32_t add_galois, int B, int level,
                              const ModDownConsts &dc, cudaStream_t st, const uint64_t *plus = nullptr);
void k_launch_rescale_spread(Context &c, uint64_t *tmp, const uint64_t *last, int B, int level,
                             const RescaleConsts &rc, cudaStream_t st);
void k_launch_rescale_combine(Context &c, uint64_t *out, const uint64_t *cc, const uint64_t *tmp, int B, int level,
                              const RescaleConsts &rc, cudaStream_t st);
void k_launch_permute(Context &c, uint64_t *out, const uint64_t *in, size_t rows, uint32_t galois, cudaStream_t st);

// Fused ModUp tail (ntt.cu): y[b][i] = [x_{b,i} (Qhat_{j,u})^-1]_{q_i} in
// coefficient form ([B][level+1][N]).  For every stored digit row (window b,
// digit j, target t outside digit j's primes) the strided pass of the forward
// NTT forms sum_u y[b][j*alpha+u] * Qhat_{j,u} mod prime(t) on the fly; both
// forward passes then run in place on digits [B][beta][level+1+K][N].
void launch_modup_ntt(Context &c, uint64_t *digits, const uint64_t *y, int B, int level, cudaStream_t st);

// Fused ModDown tail (ntt.cu).  z[bh][k] = [u_{p_k} Phat_k^-1]_{p_k} in
// coefficient form ([B*2][K][N]).  The strided pass of v's forward NTT forms
// v_i = sum_k z_k Phat_k - c P mod q_i (c = number of z_k > p_k / 2) on the
// fly into vtmp ([B*2][level+1][N]); the contiguous pass writes
//   out[b][h][i][x] = (u[b][h][i][x] - v[b][h][i][x]) P^-1 + add_h[b][i][perm(x)] + plus[b][h][i][x]
// (add_h and plus optional; perm = the Galois map of `galois`).
struct CombineArgs {
    uint64_t *out;
    const uint64_t *u;            // [B][2][level+1+K][N]; null: computed in place from KeyipArgs
    const uint64_t *add0, *add1;  // window stride add_stride words
    size_t add_stride;
    uint32_t galois;
    const uint64_t *plus;         // [B][2][level+1][N]
    size_t u_stride = 0;          // rows between consecutive blocks of u (0: level+1+K)
};

// Operands of the key inner product when its output words are formed inside
// the ModDown passes that consume them, instead of being stored: word (b, h,
// t, x) = redc(sum_j digit_j[b][t][perm(x)] * key_b[j][h][t][x]), the same
// 128-bit sum and single Montgomery reduction as k_launch_keyip, so the words
// are identical.  Window b's digits sit at digits + b * beta * nre * N, its
// own-prime rows at own + b * own_stride; w0 is the batch index of the
// launch's first window (key lookup and digit offsets).
struct KeyipArgs {
    const uint64_t *digits;
    const uint64_t *own;
    size_t own_stride;
    KeyPtrs key;
    int beta, alpha, nre, level, key_rows, L1;
    int w0;
    uint32_t galois;
};
void launch_moddown_ntt(Context &c, uint64_t *vtmp, const uint64_t *z, const CombineArgs &a, int B, int level,
                        cudaStream_t st, const KeyipArgs *ka = nullptr);
// The same over `blocks` single blocks (no window/part structure: add0, add1
// and the key-inner-product operands unused), block k of u at
// u + k * u_stride rows, out [blocks][level+1][N].
void launch_moddown_ntt_blocks(Context &c, uint64_t *vtmp, const uint64_t *z, const CombineArgs &a, size_t blocks,
                               int level, cudaStream_t st);
// The P rows of the key inner product, formed in the load of the inverse
// NTT's contiguous pass, then the strided pass: z[bh][k] =
// [u_{p_k} Phat_k^-1]_{p_k} in coefficient form ([B*2][K][N]).
void launch_keyip_p_inv(Context &c, uint64_t *z, const KeyipArgs &ka, int B, int level, cudaStream_t st);

// Fused sum of products: out (+)= sum_k ct_k (.) pt_k over a batch of
// ciphertexts at one level (each ct_k [B][2][l+1][N], each pt_k [l+1][N] in
// Montgomery form); at most Context::sum_terms_max terms per launch.
constexpr int MAX_SUM_TERMS = 16;
struct SumTerms {
    const uint64_t *ct[MAX_SUM_TERMS];
    const uint64_t *pt[MAX_SUM_TERMS];
    int n;
};
void k_launch_mul_plain_sum(Context &c, uint64_t *out, const SumTerms &terms, int B, int level, bool acc,
                            cudaStream_t st);

// Every giant step of a BSGS product in one pass over its baby steps:
// out_g (+)= sum_t ct_t * pt_{g,t} for g < ng (pt_{g,t} = nullptr: absent),
// ng <= MULTI_SUM_GROUPS, nt <= min(MAX_SUM_TERMS, Context::sum_terms_max).
constexpr int MULTI_SUM_GROUPS = 4;
struct MultiSumTerms {
    const uint64_t *ct[MAX_SUM_TERMS];
    const uint64_t *pt[MULTI_SUM_GROUPS][MAX_SUM_TERMS];
    uint64_t *out[MULTI_SUM_GROUPS];
    int nt, ng;
};
// qp: every operand and output is over the extended basis Q_l * P
// ([B][2][l+1+K][N], constants [l+1+K][N]).
void k_launch_mul_plain_sum_multi(Context &c, const MultiSumTerms &terms, int B, int level, bool acc,
                                  cudaStream_t st, bool qp = false);

// Extended-basis helpers of the double-hoisted BSGS product (batches
// [B][2][l+1+K][N], rows q_0..q_l then p_0..p_{K-1}, evaluation domain):
// out = (P c0, P c1) from a ciphertext over Q_l ([B][2][l+1][N]);
void k_launch_qp_times_p(Context &c, uint64_t *out, const uint64_t *in, int B, int level, const ModDownConsts &dc,
                         cudaStream_t st);
// u_0 rows mod q_i += P * c0[perm(x)] (c0 of ct [B][2][l+1][N], perm = the Galois map);
void k_launch_qp_add_pc0(Context &c, uint64_t *u, const uint64_t *ct, int B, int level, uint32_t galois,
                         const ModDownConsts &dc, cudaStream_t st);
// acc (+)= (in_0[perm(x)] + w_0, w_1), or acc (+)= in when w is null;
void k_launch_qp_giant_acc(Context &c, uint64_t *acc, const uint64_t *in, const uint64_t *w, int B, int level,
                           uint32_t galois, bool accumulate, cudaStream_t st);
// rows l+1.. of pt ([l+1+K][N], coefficient form) from its row 0, checked against row 1 (*err |= 1).
void k_launch_qp_extend(Context &c, uint64_t *pt, int level, int *err, cudaStream_t st);

// Linear combination with scalar constants: out (+)= sum_k s_k * ct_k over a
// batch at one level, s_k[i] = the scalar's residue mod q_i in Montgomery
// form; at most Context::sum_terms_max terms per launch.
struct LincombTerms {
    const uint64_t *ct[MAX_SUM_TERMS];
    uint64_t s[MAX_SUM_TERMS][MMFHE_MAX_Q];
    int n;
};
void k_launch_lincomb(Context &c, uint64_t *out, const LincombTerms &terms, int B, int level, bool acc,
                      cudaStream_t st);

}  // namespace mmfhe
