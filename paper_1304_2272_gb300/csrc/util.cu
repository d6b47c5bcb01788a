// Small device utilities of the engine.
#include <algorithm>

#include "../../include/gwas.h"
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace gwas {

// Deterministic pseudo-random dosages in {0, 1, 2} (splitmix64 of the index), used by
// the autotuner when the caller gives no dosages: kernel timing does not depend on them.
__global__ void k_fill_dosages(int8_t* __restrict__ X, int64_t count, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        X[i] = (int8_t)(z % 3);
    }
}

cudaError_t launch_fill_dosages(int8_t* X, int64_t count, uint64_t seed, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_fill_dosages<<<1024, 256, 0, s>>>(X, count, seed);
    return cudaGetLastError();
}

// Exercises the bounded-wait path every pipeline kernel relies on: one thread waits for
// phase 0 of an mbarrier that nothing ever arrives on. The wait must give up after
// limit_ns and report it, leaving the context usable.
__global__ void k_wait_selftest(uint64_t limit_ns, int* code, unsigned long long* waited_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = tc::globaltimer();
        const bool completed = tc::mbar_wait(&bar, 0, limit_ns);
        *waited_ns = tc::globaltimer() - t0;
        *code = completed ? 0 : 1;
    }
}

// FP64 multiply-add throughput probe: every thread runs CHAINS independent chains
// a <- a * beta + gamma (beta = 1 - 2^-20, gamma = 2^-20, so a stays near 1: no overflow,
// no subnormals) for iters x 16 steps, then stores its sum so no chain is dead code.
template <int CHAINS>
__global__ void __launch_bounds__(256) k_dfma_rate(int iters, double beta, double gamma,
                                                   double* __restrict__ out) {
    double a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = 1.0 + 1e-3 * (double)((threadIdx.x + i) & 7);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], beta, gamma);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CHAINS>
static cudaError_t time_dfma(int blocks, int iters, double* out, cudaEvent_t e0, cudaEvent_t e1,
                             double* tflops) {
    const double beta = 1.0 - 1.0 / 1048576.0, gamma = 1.0 / 1048576.0;
    k_dfma_rate<CHAINS><<<blocks, 256>>>(iters, beta, gamma, out);  // warm-up
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double best = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        k_dfma_rate<CHAINS><<<blocks, 256>>>(iters, beta, gamma, out);
        cudaEventRecord(e1);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
        const double flops = 2.0 * 16.0 * CHAINS * (double)iters * blocks * 256.0;
        if (ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    *tflops = best;
    return cudaGetLastError();
}

}  // namespace gwas

extern "C" gwas_status gwas_fp64_fma_rate(int device, double* tflops) {
    if (!tflops) return GWAS_ERR_ARG;
    *tflops = 0.0;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return GWAS_ERR_CUDA;
    int sms = 0;
    gwas_status st = GWAS_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* out = nullptr;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        cudaMalloc(&out, sizeof(double) * 256 * 8 * (size_t)sms) == cudaSuccess) {
        // a few shapes (chains per thread x CTAs per SM), each launch ~0.1-0.2 s at
        // 1.25 TFLOP/s; the best rate is the FP64 FMA peak this device sustains
        const int shapes[4][2] = {{8, 2}, {8, 4}, {16, 2}, {4, 8}};
        double best = 0.0;
        bool ok = true;
        for (const auto& sh : shapes) {
            const int chains = sh[0], blocks = sh[1] * sms;
            const int iters = (int)(1.5e11 / (2.0 * 16.0 * chains * blocks * 256.0));
            double r = 0.0;
            cudaError_t e = chains == 4    ? gwas::time_dfma<4>(blocks, iters, out, e0, e1, &r)
                            : chains == 8  ? gwas::time_dfma<8>(blocks, iters, out, e0, e1, &r)
                                           : gwas::time_dfma<16>(blocks, iters, out, e0, e1, &r);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ok = false;
                break;
            }
            best = std::max(best, r);
        }
        if (ok) {
            *tflops = best;
            st = GWAS_OK;
        }
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

extern "C" gwas_status gwas_selftest_wait(int device, int timeout_ms, double* waited_ms) {
    if (timeout_ms < 1 || timeout_ms > 10000) return GWAS_ERR_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return GWAS_ERR_CUDA;
    void* buf = nullptr;
    gwas_status st = GWAS_ERR_CUDA;
    if (cudaMalloc(&buf, 16) == cudaSuccess) {
        int* code = static_cast<int*>(buf);
        auto* waited = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + 8);
        gwas::k_wait_selftest<<<1, 32>>>((uint64_t)timeout_ms * 1000000ull, code, waited);
        int h_code = -1;
        unsigned long long h_waited = 0;
        if (cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
            cudaMemcpy(&h_code, code, sizeof h_code, cudaMemcpyDeviceToHost) == cudaSuccess &&
            cudaMemcpy(&h_waited, waited, sizeof h_waited, cudaMemcpyDeviceToHost) == cudaSuccess) {
            if (waited_ms) *waited_ms = h_waited / 1e6;
            st = h_code == 1 ? GWAS_ERR_TIMEOUT : GWAS_OK;
        }
        cudaFree(buf);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}
