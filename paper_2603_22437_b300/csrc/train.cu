// Plaintext training of the polynomial network (FP32 on the GPU) and its
// folding into the pure-square form the encrypted circuit evaluates.
//
// The network: z_l = W_l [a_{l-1}; 1] (W_l is d_{l+1} x (d_l + 1), the last
// column the bias), a_l = z_l + alpha z_l^2 after every layer but the last,
// softmax cross-entropy on the last layer's outputs.  Any quadratic
// activation is a shifted, scaled square,
//   z + alpha z^2 = alpha (z + beta)^2 - gamma,  beta = 1 / (2 alpha), gamma = 1 / (4 alpha),
// so the trained network equals one with pure squares whose affine parts are
// folded into the neighbouring layers (mmfhe_fold_poly_net): the form the
// paper's FC network with square activations takes, at the same depth.
// Inputs are standardised for training; the standardisation is folded back
// into the first layer, so the returned weights act on raw inputs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <vector>

#include "handles.h"
#include "internal.h"

using namespace mmfhe;

namespace {

constexpr int TT = 256;

// C[m][n] = sum_k A[m*sam + k*sak] * B[k*sbk + n*sbn]  (+ C when acc)
__global__ void k_gemm(int M, int N, int K, const float *A, int sam, int sak, const float *B, int sbk, int sbn,
                       float *C, int ldc, int acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * N) return;
    const int m = i / N, n = i % N;
    float s = 0.f;
    for (int k = 0; k < K; k++) s += A[(size_t)m * sam + (size_t)k * sak] * B[(size_t)k * sbk + (size_t)n * sbn];
    C[(size_t)m * ldc + n] = acc ? C[(size_t)m * ldc + n] + s : s;
}

// Next layer's input [a; 1]: a = z + alpha z^2 (rows of width d, ld d + 1).
__global__ void k_act(const float *z, float *anext, int M, int d, float alpha) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * (d + 1)) return;
    const int m = i / (d + 1), j = i % (d + 1);
    const float v = j < d ? z[(size_t)m * d + j] : 0.f;
    anext[i] = j < d ? v + alpha * v * v : 1.f;
}

// dz = da * (1 + 2 alpha z), da read from the first d columns of rows of width ld.
__global__ void k_act_back(const float *da, int ld, const float *z, float *dz, int M, int d, float alpha) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * d) return;
    const int m = i / d, j = i % d;
    dz[i] = da[(size_t)m * ld + j] * (1.f + 2.f * alpha * z[i]);
}

// dz = (softmax(z) - onehot(y)) / M for rows of width C.
__global__ void k_softmax_grad(const float *z, const int *y, float *dz, int M, int C) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const float *zr = z + (size_t)m * C;
    float mx = zr[0];
    for (int c = 1; c < C; c++) mx = fmaxf(mx, zr[c]);
    float s = 0.f;
    for (int c = 0; c < C; c++) s += expf(zr[c] - mx);
    for (int c = 0; c < C; c++) dz[(size_t)m * C + c] = (expf(zr[c] - mx) / s - (c == y[m] ? 1.f : 0.f)) / (float)M;
}

// Gather rows idx[0..M) of X (width d) into [x; 1] rows (width d + 1) and their labels.
__global__ void k_gather(const float *X, const int *labels, const int *idx, float *A0, int *y, int M, int d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * (d + 1)) return;
    const int m = i / (d + 1), j = i % (d + 1);
    A0[i] = j < d ? X[(size_t)idx[m] * d + j] : 1.f;
    if (j == 0) y[m] = labels[idx[m]];
}

// Momentum SGD: v = mu v + g; w -= lr v.
__global__ void k_sgd(float *w, float *v, const float *g, int n, float lr, float mu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    v[i] = mu * v[i] + g[i];
    w[i] -= lr * v[i];
}

inline unsigned blocks(size_t n) { return (unsigned)((n + TT - 1) / TT); }

struct DevBuf {
    float *p = nullptr;
    explicit DevBuf(size_t n) { CK(cudaMalloc(&p, std::max<size_t>(1, n) * sizeof(float))); }
    ~DevBuf() { cudaFree(p); }
};

}  // namespace

// Fold the quadratic activations into pure squares.  Layer l's matrix is
// D x D (bias in column D-1, M[D-1][D-1] = 1); with `wide`, layer 0 goes to
// `first` as D x (d_0 + 1) (bias in column d_0) and layers 1.. to mats.
static mmfhe_status fold(const uint32_t *dims, uint32_t layers, float alpha, const float *weights, uint32_t width,
                         bool wide, double *first, double *mats) {
    if (!dims || !weights || (!mats && !wide) || layers < 1 || layers > 8 || alpha <= 0.f || width < 2 ||
        (width & (width - 1)))
        return MMFHE_ERR_BAD_ARG;
    const int L = (int)layers, D = (int)width;
    for (int l = wide ? 1 : 0; l <= L; l++)
        if (dims[l] < 1 || (int)dims[l] >= D) return MMFHE_ERR_BAD_ARG;
    if (dims[0] < 1) return MMFHE_ERR_BAD_ARG;
    const double a = alpha, beta = 1.0 / (2.0 * a), gamma = 1.0 / (4.0 * a);
    size_t off = 0;
    for (int l = 0; l < L; l++) {
        const int din = (int)dims[l], dout = (int)dims[l + 1];
        const bool w0 = wide && l == 0;
        const int cols = w0 ? din + 1 : D, bcol = w0 ? din : D - 1;
        double *M = w0 ? first : mats + (size_t)(wide ? l - 1 : l) * D * D;
        std::fill(M, M + (size_t)D * cols, 0.0);
        for (int o = 0; o < dout; o++) {
            const float *row = weights + off + (size_t)o * (din + 1);
            double bias = row[din];
            for (int j = 0; j < din; j++) {
                // the input of a layer after the first is a = alpha s - gamma (s = the previous square)
                M[(size_t)o * cols + j] = l > 0 ? a * row[j] : row[j];
                if (l > 0) bias -= gamma * row[j];
            }
            // a hidden layer's square takes (z + beta)^2
            M[(size_t)o * cols + bcol] = bias + (l < L - 1 ? beta : 0.0);
        }
        M[(size_t)(D - 1) * cols + bcol] = 1.0;
        off += (size_t)dout * (din + 1);
    }
    return MMFHE_OK;
}

extern "C" {

mmfhe_status mmfhe_train_poly_net(mmfhe_ctx *ctx, const float *X, const int32_t *labels, uint64_t n,
                                  const uint32_t *dims, uint32_t layers, float alpha, uint32_t epochs,
                                  uint32_t batch, float lr, uint64_t seed, float *weights, float *train_accuracy) {
    Context *c = nullptr;
    try {
        if (!ctx || !ctx->c) throw Error(MMFHE_ERR_BAD_ARG, "null context");
        c = ctx->c;
        if (!X || !labels || !dims || !weights || n == 0 || layers < 1 || layers > 8 || batch < 1 || alpha <= 0.f)
            throw Error(MMFHE_ERR_BAD_ARG, "bad training arguments");
        CK(cudaSetDevice(c->device));
        const int L = (int)layers, d0 = (int)dims[0], C = (int)dims[L];
        for (int l = 0; l <= L; l++)
            if (dims[l] < 1 || dims[l] > 4096) throw Error(MMFHE_ERR_BAD_ARG, "layer widths 1..4096");
        for (uint64_t i = 0; i < n; i++)
            if (labels[i] < 0 || labels[i] >= C) throw Error(MMFHE_ERR_BAD_ARG, "label out of range");
        // standardise the inputs (folded back into the first layer at the end)
        std::vector<double> mu(d0, 0.0), sd(d0, 0.0);
        for (uint64_t i = 0; i < n; i++)
            for (int j = 0; j < d0; j++) mu[j] += X[i * d0 + j];
        for (int j = 0; j < d0; j++) mu[j] /= (double)n;
        for (uint64_t i = 0; i < n; i++)
            for (int j = 0; j < d0; j++) sd[j] += (X[i * d0 + j] - mu[j]) * (X[i * d0 + j] - mu[j]);
        // a floor of 5 % of the largest spread keeps near-constant inputs
        // from inflating their folded weights (encoded at scale q_l later)
        double sd_max = 0.0;
        for (int j = 0; j < d0; j++) sd_max = std::max(sd_max, sd[j] = std::sqrt(sd[j] / (double)n));
        for (int j = 0; j < d0; j++) sd[j] = std::max(sd[j], 0.05 * sd_max) + 1e-12;
        std::vector<float> Xs(n * d0);
        for (uint64_t i = 0; i < n; i++)
            for (int j = 0; j < d0; j++) Xs[i * d0 + j] = (float)((X[i * d0 + j] - mu[j]) / sd[j]);
        // parameters: W_l [d_{l+1}][d_l + 1], He-style initialisation
        std::mt19937_64 rng(seed);
        std::vector<size_t> off(L + 1, 0);
        for (int l = 0; l < L; l++) off[l + 1] = off[l] + (size_t)dims[l + 1] * (dims[l] + 1);
        std::vector<float> w(off[L], 0.f);
        for (int l = 0; l < L; l++) {
            std::normal_distribution<float> nd(0.f, 1.f / std::sqrt((float)dims[l]));
            for (uint32_t o = 0; o < dims[l + 1]; o++)
                for (uint32_t i = 0; i < dims[l]; i++) w[off[l] + (size_t)o * (dims[l] + 1) + i] = nd(rng);
        }
        const int Bm = (int)std::min<uint64_t>(batch, n);
        DevBuf dX(n * d0), dW(off[L]), dV(off[L]), dG(off[L]);
        int *dlab = nullptr, *didx = nullptr, *dy = nullptr;
        CK(cudaMalloc(&dlab, n * sizeof(int)));
        CK(cudaMalloc(&didx, std::max<uint64_t>(n, 1) * sizeof(int)));
        CK(cudaMalloc(&dy, std::max<uint64_t>(n, 1) * sizeof(int)));
        struct IntFree {
            int *a, *b, *c;
            ~IntFree() { cudaFree(a); cudaFree(b); cudaFree(c); }
        } int_free{dlab, didx, dy};
        CK(cudaMemcpy(dX.p, Xs.data(), Xs.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dlab, labels, n * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dW.p, w.data(), w.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemset(dV.p, 0, off[L] * 4));
        // activations: A_l = [a_{l-1}; 1] (rows d_l + 1), Z_l (rows d_{l+1}), gradients alike
        const int Mmax = (int)n;   // the final pass runs the whole set at once
        std::vector<std::unique_ptr<DevBuf>> A(L), Z(L), dZ(L), dA(L);
        for (int l = 0; l < L; l++) {
            A[l].reset(new DevBuf((size_t)Mmax * (dims[l] + 1)));
            Z[l].reset(new DevBuf((size_t)Mmax * dims[l + 1]));
            dZ[l].reset(new DevBuf((size_t)Mmax * dims[l + 1]));
            dA[l].reset(new DevBuf((size_t)Mmax * (dims[l] + 1)));
        }
        auto forward = [&](int M) {
            for (int l = 0; l < L; l++) {
                const int din = (int)dims[l] + 1, dout = (int)dims[l + 1];
                // Z = A W^T
                k_gemm<<<blocks((size_t)M * dout), TT>>>(M, dout, din, A[l]->p, din, 1, dW.p + off[l], 1, din,
                                                         Z[l]->p, dout, 0);
                if (l + 1 < L) k_act<<<blocks((size_t)M * (dout + 1)), TT>>>(Z[l]->p, A[l + 1]->p, M, dout, alpha);
            }
        };
        std::vector<int> order(n);
        std::iota(order.begin(), order.end(), 0);
        for (uint32_t ep = 0; ep < epochs; ep++) {
            std::shuffle(order.begin(), order.end(), rng);
            for (uint64_t s0 = 0; s0 + Bm <= n; s0 += Bm) {
                const int M = Bm;
                CK(cudaMemcpy(didx, order.data() + s0, M * sizeof(int), cudaMemcpyHostToDevice));
                k_gather<<<blocks((size_t)M * (d0 + 1)), TT>>>(dX.p, dlab, didx, A[0]->p, dy, M, d0);
                forward(M);
                k_softmax_grad<<<blocks(M), TT>>>(Z[L - 1]->p, dy, dZ[L - 1]->p, M, C);
                for (int l = L - 1; l >= 0; l--) {
                    const int din = (int)dims[l] + 1, dout = (int)dims[l + 1];
                    // G_l = dZ^T A  (dout x din)
                    k_gemm<<<blocks((size_t)dout * din), TT>>>(dout, din, M, dZ[l]->p, 1, dout, A[l]->p, din, 1,
                                                               dG.p + off[l], din, 0);
                    if (l > 0) {
                        // dA = dZ W  (M x din), then dZ_{l-1} = dA (1 + 2 alpha z)
                        k_gemm<<<blocks((size_t)M * din), TT>>>(M, din, dout, dZ[l]->p, dout, 1, dW.p + off[l], din, 1,
                                                                dA[l]->p, din, 0);
                        k_act_back<<<blocks((size_t)M * dims[l]), TT>>>(dA[l]->p, din, Z[l - 1]->p, dZ[l - 1]->p, M,
                                                                       (int)dims[l], alpha);
                    }
                }
                k_sgd<<<blocks(off[L]), TT>>>(dW.p, dV.p, dG.p, (int)off[L], lr, 0.9f);
            }
            CK(cudaGetLastError());
        }
        CK(cudaMemcpy(w.data(), dW.p, w.size() * 4, cudaMemcpyDeviceToHost));
        if (train_accuracy) {
            std::vector<int> all(n);
            std::iota(all.begin(), all.end(), 0);
            CK(cudaMemcpy(didx, all.data(), n * sizeof(int), cudaMemcpyHostToDevice));
            k_gather<<<blocks((size_t)n * (d0 + 1)), TT>>>(dX.p, dlab, didx, A[0]->p, dy, (int)n, d0);
            forward((int)n);
            std::vector<float> z((size_t)n * C);
            CK(cudaMemcpy(z.data(), Z[L - 1]->p, z.size() * 4, cudaMemcpyDeviceToHost));
            uint64_t ok = 0;
            for (uint64_t i = 0; i < n; i++)
                ok += (uint64_t)(std::max_element(z.begin() + i * C, z.begin() + (i + 1) * C) - (z.begin() + i * C)) ==
                      (uint64_t)labels[i];
            *train_accuracy = (float)ok / (float)n;
        }
        // fold the standardisation into layer 0: W x_s + b = (W / sd) x + (b - W mu / sd)
        for (uint32_t o = 0; o < dims[1]; o++) {
            float *row = &w[off[0] + (size_t)o * (d0 + 1)];
            double b = row[d0];
            for (int j = 0; j < d0; j++) {
                b -= row[j] * mu[j] / sd[j];
                row[j] = (float)(row[j] / sd[j]);
            }
            row[d0] = (float)b;
        }
        std::copy(w.begin(), w.end(), weights);
    } catch (const Error &e) {
        if (c) c->last_error = e.what();
        return e.code;
    } catch (const std::exception &e) {
        if (c) c->last_error = e.what();
        return MMFHE_ERR_CUDA;
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_fold_poly_net(const uint32_t *dims, uint32_t layers, float alpha, const float *weights,
                                 uint32_t width, double *mats) {
    return fold(dims, layers, alpha, weights, width, false, nullptr, mats);
}

mmfhe_status mmfhe_fold_poly_net_wide(const uint32_t *dims, uint32_t layers, float alpha, const float *weights,
                                      uint32_t width, double *first, double *mats) {
    if (!first || (layers > 1 && !mats)) return MMFHE_ERR_BAD_ARG;
    return fold(dims, layers, alpha, weights, width, true, first, mats);
}

}  // extern "C"
