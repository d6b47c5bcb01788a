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

// FP64 multiply-add throughput probe with the FP64 block kernel's inner loop: 256
// threads, each a 4 x 4 register tile acc[a][b] += As[k][a] Bs[k][b] over 16-deep chunks
// re-read from shared memory after a barrier (dependent chains of fma on shared
// constants run slower on this part, so they would not bound the block kernel).
// Operands are near 1 (no overflow, no subnormals); each thread stores its sum.
__global__ void __launch_bounds__(256) k_dfma_rate(int iters, double beta, double gamma,
                                                   double* __restrict__ out) {
    __shared__ double As[KC64][T64 + 1];
    __shared__ double Bs[KC64][T64 + 1];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    for (int e = tid; e < KC64 * T64; e += blockDim.x) {
        As[e / T64][e % T64] = beta * (1.0 + 1e-6 * (double)(e & 31));
        Bs[e / T64][e % T64] = gamma * (1.0 - 1e-6 * (double)(e & 15));
    }
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int it = 0; it < iters; ++it) {
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC64; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) s += acc[a][b];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// fma per thread and iteration of k_dfma_rate
constexpr double kFmaPerIter = 16.0 * KC64;

static cudaError_t time_dfma(int blocks, int iters, double* out, cudaEvent_t e0, cudaEvent_t e1,
                             double* tflops) {
    const double beta = 1.0 - 1.0 / 1048576.0, gamma = 1.0 / 1048576.0;
    k_dfma_rate<<<blocks, 256>>>(iters, beta, gamma, out);  // warm-up
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double best = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        k_dfma_rate<<<blocks, 256>>>(iters, beta, gamma, out);
        cudaEventRecord(e1);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
        const double flops = 2.0 * kFmaPerIter * (double)iters * blocks * 256.0;
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
        // 2, 4 and 8 CTAs per SM, each launch ~0.12 s at 1.25 TFLOP/s; the best rate is
        // the FP64 FMA rate this device sustains
        const int per_sm[3] = {2, 4, 8};
        double best = 0.0;
        bool ok = true;
        for (int ps : per_sm) {
            const int blocks = ps * sms;
            const int iters = (int)(1.5e11 / (2.0 * gwas::kFmaPerIter * blocks * 256.0));
            double r = 0.0;
            cudaError_t e = gwas::time_dfma(blocks, iters, out, e0, e1, &r);
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
