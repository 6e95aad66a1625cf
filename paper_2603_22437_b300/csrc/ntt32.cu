// Word-size ablation: the negacyclic NTT on 32-bit RNS words (primes below
// 2^30), for comparing transform throughput per modulus bit with the 64-bit
// path the chains run on.
//
// Same transform as the 64-bit kernels (merged Cooley-Tukey forward with
// bit-reversed output: stage s, group i uses psi^brv(2^s + i); Gentleman-Sande
// inverse, then N^-1), but one pass: a 32-bit row of N <= 2^15 words fits in
// shared memory (128 KB), so a CTA owns a whole row, reads it from HBM once
// and writes it once.  Inside, every thread holds 16 words per round in
// registers and applies up to four stages per shared-memory round trip.
// Shoup products with 32-bit companions; values stay in [0, 4q) (forward) or
// [0, 2q) (inverse) until the final reduction (q < 2^30 keeps 4q < 2^32).
#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "handles.h"
#include "hostmath.h"
#include "internal.h"

using namespace mmfhe;

struct mmfhe_ntt32 {
    int device = 0, logn = 0, np = 0;
    std::vector<uint32_t> primes;
    uint32_t *d_tw = nullptr;     // [4][np][N]: W, W', Winv, Winv' (brv order)
    uint32_t *d_q = nullptr;      // [np] primes, then [np] N^-1, then [np] Shoup(N^-1)
    std::string last_error;
};

namespace {

constexpr int NT32_MAX_THREADS = 1024;

__device__ __forceinline__ uint32_t shoup32(uint32_t a, uint32_t w, uint32_t wp, uint32_t q) {
    return a * w - __umulhi(a, wp) * q;   // in [0, 2q) for any a < 2^32
}

__device__ __forceinline__ uint32_t pad32(uint32_t i) { return i + (i >> 5); }

// Element (group g, index j) of a round over global stages [A, A+R) of the
// size-2^LOG transform, for 16-word unit u: j fills bits [POS, POS+R).
template <int LOG, int A, int R>
__device__ __forceinline__ uint32_t idx32(uint32_t u, int g, int j) {
    constexpr int POS = LOG - A - R;
    const uint32_t o = u * (16 >> R) + g;
    return ((o >> POS) << (POS + R)) | ((uint32_t)j << POS) | (o & ((1u << POS) - 1));
}

template <int LOG, int A, int R, bool FWD>
__device__ __forceinline__ void round32(uint32_t *sm, uint32_t u, uint32_t q, const uint32_t *__restrict__ W,
                                        const uint32_t *__restrict__ Wp) {
    constexpr int G = 16 >> R, M = 1 << R;
    uint32_t x[16];
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int j = 0; j < M; j++) x[g * M + j] = sm[pad32(idx32<LOG, A, R>(u, g, j))];
    const uint32_t q2 = 2 * q;
#pragma unroll
    for (int uu = 0; uu < R; uu++) {
        const int s = FWD ? uu : R - 1 - uu;   // local stage
        const int dist = 1 << (R - 1 - s);
#pragma unroll
        for (int g = 0; g < G; g++) {
            uint32_t w = 0, wp = 0;
#pragma unroll
            for (int j = 0; j < M; j++) {
                if (j & dist) continue;
                if ((j & (dist - 1)) == 0) {   // the pairs of a run share one twiddle
                    const uint32_t h = idx32<LOG, A, R>(u, g, j);
                    const uint32_t widx = (1u << (A + s)) + (h >> (LOG - A - s));
                    w = __ldg(W + widx);
                    wp = __ldg(Wp + widx);
                }
                uint32_t &a = x[g * M + j], &b = x[g * M + j + dist];
                if (FWD) {
                    if (a >= q2) a -= q2;
                    const uint32_t t = shoup32(b, w, wp, q);
                    b = a - t + q2;
                    a = a + t;
                } else {
                    uint32_t t = a + b;
                    if (t >= q2) t -= q2;
                    b = shoup32(a - b + q2, w, wp, q);
                    a = t;
                }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int j = 0; j < M; j++) sm[pad32(idx32<LOG, A, R>(u, g, j))] = x[g * M + j];
}

template <int LOG>
struct Geo32 {
    static constexpr int N = 1 << LOG;
    static constexpr int UNITS = N / 16;
    static constexpr int THREADS = UNITS < NT32_MAX_THREADS ? UNITS : NT32_MAX_THREADS;
    static constexpr int UPT = UNITS / THREADS;   // 16-word units per thread and round
    static constexpr int SMEM = (N + N / 32) * 4;
};

// Rounds of at most four stages: [0,4), [4,8), ... ; the last may be shorter.
template <int LOG, int A, bool FWD>
__device__ __forceinline__ void rounds_fwd(uint32_t *sm, uint32_t q, const uint32_t *W, const uint32_t *Wp) {
    if constexpr (A < LOG) {
        constexpr int R = (LOG - A) < 4 ? (LOG - A) : 4;
#pragma unroll
        for (int k = 0; k < Geo32<LOG>::UPT; k++) round32<LOG, A, R, true>(sm, threadIdx.x + k * Geo32<LOG>::THREADS, q, W, Wp);
        __syncthreads();
        rounds_fwd<LOG, A + R, FWD>(sm, q, W, Wp);
    }
}

// Inverse rounds, last stages first: A is the first stage of the round.
template <int LOG, int A>
__device__ __forceinline__ void rounds_inv(uint32_t *sm, uint32_t q, const uint32_t *W, const uint32_t *Wp) {
    if constexpr (A >= 0) {
        constexpr int R = (LOG - A) < 4 ? (LOG - A) : 4;
#pragma unroll
        for (int k = 0; k < Geo32<LOG>::UPT; k++) round32<LOG, A, R, false>(sm, threadIdx.x + k * Geo32<LOG>::THREADS, q, W, Wp);
        __syncthreads();
        rounds_inv<LOG, A - 4>(sm, q, W, Wp);
    }
}


template <int LOG, bool FWD>
__global__ void __launch_bounds__(Geo32<LOG>::THREADS, 1)
    k_ntt32(uint32_t *data, int np, const uint32_t *__restrict__ tw, const uint32_t *__restrict__ qs) {
    using Gm = Geo32<LOG>;
    extern __shared__ uint32_t sm[];
    const int pi = (int)(blockIdx.x % (uint32_t)np);
    const uint32_t q = qs[pi];
    const size_t N = Gm::N;
    uint32_t *row = data + (size_t)blockIdx.x * N;
    const uint32_t *W = tw + ((size_t)(FWD ? 0 : 2) * np + pi) * N;
    const uint32_t *Wp = tw + ((size_t)(FWD ? 1 : 3) * np + pi) * N;
    for (uint32_t i = threadIdx.x * 4; i < N; i += Gm::THREADS * 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(row + i);
        sm[pad32(i)] = v.x;
        sm[pad32(i + 1)] = v.y;
        sm[pad32(i + 2)] = v.z;
        sm[pad32(i + 3)] = v.w;
    }
    __syncthreads();
    if (FWD)
        rounds_fwd<LOG, 0, true>(sm, q, W, Wp);
    else
        rounds_inv<LOG, ((LOG - 1) / 4) * 4>(sm, q, W, Wp);   // the first stage of the last forward round
    const uint32_t ninv = qs[np + pi], ninvp = qs[2 * np + pi];
    for (uint32_t i = threadIdx.x * 4; i < N; i += Gm::THREADS * 4) {
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            uint32_t a = sm[pad32(i + k)];
            if (FWD) {
                if (a >= 2 * q) a -= 2 * q;
            } else {
                a = shoup32(a, ninv, ninvp, q);
            }
            v[k] = a >= q ? a - q : a;
        }
        *reinterpret_cast<uint4 *>(row + i) = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

template <int LOG>
void launch32(mmfhe_ntt32 &p, uint32_t *d, size_t rows, bool inverse, cudaStream_t st) {
    using Gm = Geo32<LOG>;
    auto kern = inverse ? k_ntt32<LOG, false> : k_ntt32<LOG, true>;
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM));
    kern<<<(unsigned)rows, Gm::THREADS, Gm::SMEM, st>>>(d, p.np, p.d_tw, p.d_q);
    CK(cudaGetLastError());
}

mmfhe_status fail32(mmfhe_ntt32 *p, mmfhe_status code, const char *msg) {
    if (p) p->last_error = msg;
    return code;
}

}  // namespace

extern "C" {

mmfhe_status mmfhe_ntt32_select_primes(uint32_t log_n, uint32_t bits, uint32_t count, uint32_t *out) {
    if (!out || log_n < 10 || log_n > 15 || bits < log_n + 2 || bits > 30 || count < 1) return MMFHE_ERR_BAD_ARG;
    const uint64_t m = 2ull << log_n;
    uint64_t x = ((1ull << bits) - 1) / m * m + 1;   // largest value below 2^bits that is 1 mod 2N
    for (uint32_t k = 0; k < count; x -= m) {
        if (x < m) return MMFHE_ERR_BAD_ARG;           // not enough primes of this size
        if (x < (1ull << bits) && hm::is_prime(x)) out[k++] = (uint32_t)x;
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_ntt32_create(uint32_t log_n, const uint32_t *primes, uint32_t num_primes, int device,
                                mmfhe_ntt32 **out) {
    if (!out || !primes || log_n < 10 || log_n > 15 || num_primes < 1 || num_primes > 64) return MMFHE_ERR_BAD_ARG;
    std::unique_ptr<mmfhe_ntt32> p(new mmfhe_ntt32());
    const uint64_t N = 1ull << log_n;
    for (uint32_t i = 0; i < num_primes; i++) {
        const uint64_t q = primes[i];
        if (q >= (1u << 30) || q % (2 * N) != 1 || !hm::is_prime(q)) return MMFHE_ERR_BAD_BLOB;
    }
    try {
        CK(cudaSetDevice(device));
        p->device = device;
        p->logn = (int)log_n;
        p->np = (int)num_primes;
        p->primes.assign(primes, primes + num_primes);
        const int np = (int)num_primes;
        std::vector<uint32_t> tw((size_t)4 * np * N), qs((size_t)3 * np);
        for (int i = 0; i < np; i++) {
            const uint64_t q = primes[i], psi = hm::primitive_root_2n(q, N), psi_inv = hm::invmod(psi, q);
            for (uint64_t k = 0; k < N; k++) {
                const uint32_t e = hm::bitrev((uint32_t)k, (int)log_n);
                const uint64_t w = hm::powmod(psi, e, q), wi = hm::powmod(psi_inv, e, q);
                tw[((size_t)0 * np + i) * N + k] = (uint32_t)w;
                tw[((size_t)1 * np + i) * N + k] = (uint32_t)((w << 32) / q);
                tw[((size_t)2 * np + i) * N + k] = (uint32_t)wi;
                tw[((size_t)3 * np + i) * N + k] = (uint32_t)((wi << 32) / q);
            }
            const uint64_t ninv = hm::invmod(N % q, q);
            qs[i] = (uint32_t)q;
            qs[np + i] = (uint32_t)ninv;
            qs[2 * np + i] = (uint32_t)((ninv << 32) / q);
        }
        CK(cudaMalloc(&p->d_tw, tw.size() * 4));
        CK(cudaMalloc(&p->d_q, qs.size() * 4));
        CK(cudaMemcpy(p->d_tw, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->d_q, qs.data(), qs.size() * 4, cudaMemcpyHostToDevice));
    } catch (const Error &e) {
        if (p->d_tw) cudaFree(p->d_tw);
        if (p->d_q) cudaFree(p->d_q);
        return e.code;
    }
    *out = p.release();
    return MMFHE_OK;
}

mmfhe_status mmfhe_ntt32_run(mmfhe_ntt32 *p, uint32_t *rows, size_t num_rows, int inverse, void *stream) {
    if (!p || !rows) return fail32(p, MMFHE_ERR_BAD_ARG, "null argument");
    if (num_rows == 0) return MMFHE_OK;
    if (num_rows > (1u << 31)) return fail32(p, MMFHE_ERR_BAD_ARG, "too many rows");
    if ((uintptr_t)rows & 15) return fail32(p, MMFHE_ERR_BAD_ARG, "rows not 16-byte aligned");
    try {
        CK(cudaSetDevice(p->device));
        cudaStream_t st = (cudaStream_t)stream;
        const size_t bytes = num_rows * ((size_t)4 << p->logn);
        cudaPointerAttributes at{};
        const bool host = cudaPointerGetAttributes(&at, rows) != cudaSuccess || at.type != cudaMemoryTypeDevice;
        cudaGetLastError();
        uint32_t *d = rows;
        if (host) {
            CK(cudaMalloc(&d, bytes));
            CK(cudaMemcpyAsync(d, rows, bytes, cudaMemcpyHostToDevice, st));
        }
        switch (p->logn) {
        case 10: launch32<10>(*p, d, num_rows, inverse != 0, st); break;
        case 11: launch32<11>(*p, d, num_rows, inverse != 0, st); break;
        case 12: launch32<12>(*p, d, num_rows, inverse != 0, st); break;
        case 13: launch32<13>(*p, d, num_rows, inverse != 0, st); break;
        case 14: launch32<14>(*p, d, num_rows, inverse != 0, st); break;
        default: launch32<15>(*p, d, num_rows, inverse != 0, st); break;
        }
        if (host) {
            CK(cudaMemcpyAsync(rows, d, bytes, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            CK(cudaFree(d));
        }
    } catch (const Error &e) {
        return fail32(p, e.code, e.what());
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_ntt32_destroy(mmfhe_ntt32 *p) {
    if (!p) return MMFHE_OK;
    cudaSetDevice(p->device);
    if (p->d_tw) cudaFree(p->d_tw);
    if (p->d_q) cudaFree(p->d_q);
    delete p;
    return MMFHE_OK;
}

}  // extern "C"
