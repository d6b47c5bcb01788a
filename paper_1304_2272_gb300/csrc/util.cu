// Small device utilities of the engine.
#include "common.cuh"
#include "kernels.h"

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

}  // namespace gwas
