// Small device utilities of the engine.
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

}  // namespace gwas

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
