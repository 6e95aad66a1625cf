// Integer-pipe ceiling of the NTT arithmetic: register-resident loops of the
// forward (Harvey) butterfly on 64-bit words, exactly as the NTT passes run
// it, and of the same butterfly on 32-bit words (primes below 2^30) for the
// word-size comparison.  Each thread keeps 16 words in registers and applies
// two stages of 8 butterflies per iteration with per-pair twiddles, so
// nothing but the butterfly arithmetic is timed.
#include <cuda_runtime.h>

#include "internal.h"
#include "modarith.cuh"

namespace mmfhe {

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_ITERS = 2048;

// 32-bit Harvey butterfly: X, Y in [0, 4q), q < 2^30, Shoup w' = floor(w 2^32 / q).
__device__ __forceinline__ void ct_butterfly32(uint32_t &X, uint32_t &Y, uint32_t w, uint32_t wp, uint32_t q) {
    const uint32_t q2 = q << 1;
    const uint32_t x = X >= q2 ? X - q2 : X;
    const uint32_t t = Y * w - __umulhi(Y, wp) * q;
    X = x + t;
    Y = x - t + q2;
}

__global__ void __launch_bounds__(PEAK_THREADS)
    k_peak_bf64(uint64_t *sink, uint64_t q, const uint64_t *__restrict__ tw, int iters) {
    uint64_t x[16], w[8], wp[8];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = (threadIdx.x * 16u + i) % q;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        w[i] = tw[2 * i];
        wp[i] = tw[2 * i + 1];
    }
    for (int it = 0; it < iters; it++) {   // two stages per iteration, different pairings
#pragma unroll
        for (int i = 0; i < 8; i++) mm::ct_butterfly(x[i], x[i + 8], w[i], wp[i], q);
#pragma unroll
        for (int i = 0; i < 8; i++) mm::ct_butterfly(x[2 * i], x[2 * i + 1], w[i], wp[i], q);
    }
    uint64_t acc = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) acc ^= x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void __launch_bounds__(PEAK_THREADS)
    k_peak_bf32(uint64_t *sink, uint32_t q, const uint32_t *__restrict__ tw, int iters) {
    uint32_t x[16], w[8], wp[8];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = (threadIdx.x * 16u + i) % q;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        w[i] = tw[2 * i];
        wp[i] = tw[2 * i + 1];
    }
    for (int it = 0; it < iters; it++) {   // two stages per iteration, different pairings
#pragma unroll
        for (int i = 0; i < 8; i++) ct_butterfly32(x[i], x[i + 8], w[i], wp[i], q);
#pragma unroll
        for (int i = 0; i < 8; i++) ct_butterfly32(x[2 * i], x[2 * i + 1], w[i], wp[i], q);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) acc ^= x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// The base conversion's arithmetic: four Montgomery products summed in 128
// bits and reduced once, as the fused ModUp / ModDown passes run it.  Each
// iteration forms four outputs from the thread's 16 words (16 products) and
// feeds them back, so nothing is hoisted out of the loop.
__global__ void __launch_bounds__(PEAK_THREADS)
    k_peak_mac64(uint64_t *sink, uint64_t q, uint64_t qinv, const uint64_t *__restrict__ f, int iters) {
    uint64_t x[16], fm[4];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = (threadIdx.x * 16u + i * 977u) % q;
#pragma unroll
    for (int u = 0; u < 4; u++) fm[u] = f[u];
    for (int it = 0; it < iters; it++) {
        uint64_t r[4];
#pragma unroll
        for (int o = 0; o < 4; o++) {
            uint64_t hi = 0, lo = 0;
#pragma unroll
            for (int u = 0; u < 4; u++) mm::mac128(hi, lo, x[4 * o + u], fm[u]);
            r[o] = mm::redc(hi, lo, q, qinv);
        }
#pragma unroll
        for (int o = 0; o < 4; o++) x[4 * o + (o + it) % 4] = r[o];
    }
    uint64_t acc = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) acc ^= x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

double measure_mac_peak(Context &c) {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    const unsigned blocks = (unsigned)sms * 8;
    const size_t threads = (size_t)blocks * PEAK_THREADS;
    const uint64_t q = c.primes[0], qinv = c.mods.qinv[0];
    uint64_t h[4];
    for (int u = 0; u < 4; u++) h[u] = (q / 5 + 104729ull * (uint64_t)(u + 1)) % q;
    Buf sink(c.pool.get(), threads);
    Buf fb(c.pool.get(), 4);
    CK(cudaMemcpy(fb.get(), h, sizeof h, cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float ms = 0.f;
    k_peak_mac64<<<blocks, PEAK_THREADS>>>(sink.get(), q, qinv, fb.get(), PEAK_ITERS);   // warm-up
    CK(cudaEventRecord(e0));
    k_peak_mac64<<<blocks, PEAK_THREADS>>>(sink.get(), q, qinv, fb.get(), PEAK_ITERS);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    CK(cudaGetLastError());
    return (double)threads * PEAK_ITERS * 16 / (ms * 1e-3);
}

// Returns butterflies per second of the 64-bit and 32-bit loops on this device.
void measure_butterfly_peak(Context &c, double *bf64, double *bf32) {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    const unsigned blocks = (unsigned)sms * 8;   // 8 resident CTAs of 256 threads per SM
    const size_t threads = (size_t)blocks * PEAK_THREADS;
    // twiddle pairs of the first q prime (64-bit) and of a 30-bit prime 1 mod 2^16 (32-bit)
    const uint64_t q64 = c.primes[0];
    const uint32_t q32 = 1073479681u;   // 2^30 - 2^18 + 1, prime
    uint64_t h64[16];
    uint32_t h32[16];
    for (int i = 0; i < 8; i++) {
        const uint64_t w = (q64 / 3 + 7919ull * (uint64_t)(i + 1)) % q64;
        h64[2 * i] = w;
        h64[2 * i + 1] = (uint64_t)(((unsigned __int128)w << 64) / q64);
        const uint32_t w32 = (uint32_t)((q32 / 3u + 7919u * (uint32_t)(i + 1)) % q32);
        h32[2 * i] = w32;
        h32[2 * i + 1] = (uint32_t)(((uint64_t)w32 << 32) / q32);
    }
    Buf sink(c.pool.get(), threads);
    Buf tw(c.pool.get(), 16 + 8);
    uint32_t *tw32 = reinterpret_cast<uint32_t *>(tw.get() + 16);
    CK(cudaMemcpy(tw.get(), h64, sizeof h64, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(tw32, h32, sizeof h32, cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const double bfs = (double)threads * PEAK_ITERS * 16;
    float ms = 0.f;
    k_peak_bf64<<<blocks, PEAK_THREADS>>>(sink.get(), q64, tw.get(), PEAK_ITERS);   // warm-up
    CK(cudaEventRecord(e0));
    k_peak_bf64<<<blocks, PEAK_THREADS>>>(sink.get(), q64, tw.get(), PEAK_ITERS);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    *bf64 = bfs / (ms * 1e-3);
    k_peak_bf32<<<blocks, PEAK_THREADS>>>(sink.get(), q32, tw32, PEAK_ITERS);
    CK(cudaEventRecord(e0));
    k_peak_bf32<<<blocks, PEAK_THREADS>>>(sink.get(), q32, tw32, PEAK_ITERS);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    *bf32 = bfs / (ms * 1e-3);
    CK(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

}  // namespace mmfhe
