// Shared device/host helpers of the GWAS engine (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define GWAS_DEV __device__ __forceinline__

namespace gwas {

constexpr int WARP = 32;

// Tile edge of the FP64 SIMT kernels (rows x columns per CTA) and their k-chunk.
constexpr int T64 = 64;
constexpr int KC64 = 16;

// Largest number of per-SNP reduction values: (p-1) covariates + 1 + t phenotypes.
constexpr int MAX_P = 20;
constexpr int MAX_T = 64;

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Exact int8 dosage -> double with integer operations only (no FP64 conversion
// instruction): 0 -> +0.0, 1 -> 1.0, 2 -> 2.0. Values outside {0,1,2} map to NaN so
// that a bad dosage can never pass silently through the arithmetic.
GWAS_DEV double dosage_to_f64(int v) {
    unsigned long long bits;
    if (v == 0) bits = 0ull;
    else if (v == 1) bits = 0x3FF0000000000000ull;
    else if (v == 2) bits = 0x4000000000000000ull;
    else bits = 0x7FF8000000000000ull;
    return __longlong_as_double((long long)bits);
}

}  // namespace gwas
