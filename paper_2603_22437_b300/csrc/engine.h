// Homomorphic operations on device ciphertext batches (evaluation domain).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"
#include "kernels.h"

namespace mmfhe {

ModUpConsts modup_consts(const Context &c, int level);
ModDownConsts moddown_consts(const Context &c);
RescaleConsts rescale_consts(const Context &c, int level);

PidList pids_q(int nl);
uint32_t galois_elt(const Context &c, int32_t k);
int32_t norm_rot(const Context &c, int32_t k);

CtB ct_new(Context &c, int B, int level, double scale);
PtDev pt_new(Context &c, int level, double scale);
// in-place NTT (inverse=false) / iNTT of `blocks` contiguous blocks of nl Q-limbs
void ntt_q_blocks(Context &c, uint64_t *base, size_t blocks, int nl, bool inverse, cudaStream_t st);

void ct_addsub(Context &c, CtB &out, const CtB &a, const CtB &b, bool sub, cudaStream_t st);
void ct_mul_plain(Context &c, CtB &out, const CtB &a, const PtDev &pt, bool acc, cudaStream_t st);
void ct_mul_int(Context &c, CtB &out, const CtB &a, long long k, cudaStream_t st);
// Convert a plaintext (evaluation domain) into Montgomery form, in place.
void pt_to_mont(Context &c, PtDev &pt, cudaStream_t st);
// A plaintext over the extended basis Q_level * P from its coefficient-form Q
// rows (host or device words, uint64[level+1][N]): the integer coefficients
// (centered residues mod q_0, which must be below q_0 / 2 in magnitude:
// checked against q_1, BAD_ARG otherwise) reduced mod every p_k; evaluation
// domain, Montgomery form.
PtDev pt_qp_from_coeffs(Context &c, const uint64_t *words, int level, double scale, cudaStream_t st);
CtB ct_copy(Context &c, const CtB &a, cudaStream_t st);
CtB ct_drop(Context &c, const CtB &a, int level, cudaStream_t st);
// Ciphertexts b0 .. b0+nb-1 of a batch (a copy), and the reverse: src copied
// into dst starting at ciphertext b0 (same level).
CtB ct_slice(Context &c, const CtB &a, int b0, int nb, cudaStream_t st);
void ct_place(Context &c, CtB &dst, int b0, const CtB &src, cudaStream_t st);

TensorB tensor_new(Context &c, int B, int level);
// t (+)= coef * (a (x) b); first call with init = true
void tensor_acc(Context &c, TensorB &t, const CtB &a, const CtB &b, long long coef, bool init, cudaStream_t st);
CtB relin(Context &c, const Keys &k, const TensorB &t, cudaStream_t st);
CtB rescale(Context &c, const CtB &a, cudaStream_t st);

// ModUp of d (B windows, rows q_0..q_level, window stride block_stride_rows):
// digits in the evaluation domain.
DigitsB modup(Context &c, const uint64_t *d_eval, size_t block_stride_rows, int B, int level, cudaStream_t st);
// Write the digits' own rows (copies of the input rows) into the digit buffer.
void digits_fill_own(Context &c, DigitsB &dg, cudaStream_t st);
// ModDown(digits . key); `key` = device key in evaluation domain; galois != 1
// applies the automorphism to the digits; add0/add1 optional addends (add0
// read through the same automorphism).
CtB keyswitch_moddown(Context &c, const DigitsB &dg, const KeyPtrs &key, uint32_t galois, const uint64_t *add0,
                      const uint64_t *add1, size_t add_stride_words, double scale, cudaStream_t st,
                      const CtB *plus = nullptr);
// Switching keys of a rotation / of relinearization (per window for a batch
// mixing users); NOT_FOUND when a key is not loaded.
KeyPtrs galois_key(const Keys &k, int32_t rot);
KeyPtrs relin_key(const Keys &k);

CtB rotate(Context &c, const Keys &k, const CtB &a, int32_t rot, cudaStream_t st);
// Rot(a, rot) + plus, the addition fused into the key switch's last kernel.
CtB rotate_add(Context &c, const Keys &k, const CtB &a, int32_t rot, const CtB &plus, cudaStream_t st);
std::vector<CtB> rotate_hoisted(Context &c, const Keys &k, const CtB &a, const std::vector<int32_t> &rots,
                                cudaStream_t st);
CtB rotsum(Context &c, const Keys &k, const CtB &a, int32_t stride, uint32_t span, cudaStream_t st);

// a + pt (pt at a's level, Montgomery form, encoded at a's scale): joins c0.
CtB add_plain(Context &c, const CtB &a, const PtDev &pt, cudaStream_t st);

// Sums consecutive groups of G ciphertexts of a batch: out[b] = sum_g a[b G + g].
CtB group_sum(Context &c, const CtB &a, int G, cudaStream_t st);

// sum_i c_i * x_i for real constants c_i, each encoded at `scale` as the
// constant polynomial round(scale c_i) (an exact integer multiply); all x_i
// at one level and batch; not rescaled; result scale x.scale * scale.
CtB lincomb(Context &c, const std::vector<std::pair<const CtB *, double>> &terms, double scale, cudaStream_t st);

// One BSGS operand: baby rotations of an input (baby[i] = Rot(x, baby_idx[i] * stride))
// and the diagonals it is multiplied with, keyed by delta = g*n1 + b.
struct BsgsTerm {
    const std::vector<CtB> *baby = nullptr;
    std::vector<int> baby_idx;
    std::vector<std::pair<int, const PtDev *>> diags;   // (delta, pre-rotated diagonal)
};
CtB bsgs(Context &c, const Keys &k, const std::vector<BsgsTerm> &terms, int n1, int32_t stride, cudaStream_t st);

// One baby set of a double-hoisted BSGS product: baby b is Rot(x, b * stride
// + offset), kept over the extended basis; diags = (delta, pre-rotated
// diagonal D'_{g,b} encoded over Q_l * P), delta = g * n1 + b.
struct BsgsSet {
    const CtB *x = nullptr;
    int32_t offset = 0;
    std::vector<std::pair<int, const PtDev *>> diags;
};
// Double-hoisted BSGS product (Bossuat, Mouchet, Troncoso-Pastoriza and
// Hubaux, Eurocrypt 2021, Sec. 4): one ModUp per distinct input; every baby
// (P sigma_b(c0) + u0, u1), inner sum and giant-step term over Q_l * P; a
// giant step brings only the c1 of its inner sum down to Q (ModDown, ModUp,
// key inner product w) and adds (sigma_g(inner_0) + w_0, w_1); one ModDown of
// both parts ends the product.  Not rescaled.
CtB bsgs_dh(Context &c, const Keys &k, const std::vector<BsgsSet> &sets, int n1, int32_t stride, cudaStream_t st);

}  // namespace mmfhe
