// 2-bit packed genotype calls -> int8 dosages (the input format of the block kernels).
// The paper streams FP64 genotype matrices; four 2-bit calls per byte cut the host ->
// device stream of a block to a quarter of the int8 dosages (n/4 bytes per SNP).
#include "common.cuh"
#include "kernels.h"

namespace gwas {

// Each SNP column of Xp holds ldp = ceil(n/4) bytes; individual k sits in bits
// 2(k%4), 2(k%4)+1 of byte k/4. The four codes index the bytes of `table` (byte c =
// the dosage of code c), so one byte perm turns a packed byte into four dosages.
__global__ void __launch_bounds__(256)
k_unpack_2bit(const uint8_t* __restrict__ Xp, int64_t ldp, int64_t n, int64_t mb,
              uint32_t table, int8_t* __restrict__ X) {
    for (int64_t j = blockIdx.x; j < mb; j += gridDim.x) {
        const uint8_t* src = Xp + j * ldp;
        int8_t* dst = X + j * n;
        const bool aligned = ((reinterpret_cast<uintptr_t>(dst) & 3) == 0);
        for (int64_t kb = threadIdx.x; kb < ldp; kb += blockDim.x) {
            const uint32_t v = src[kb];
            const uint32_t sel = (v & 0x3u) | ((v << 2) & 0x30u) | ((v << 4) & 0x300u) |
                                 ((v << 6) & 0x3000u);
            const uint32_t out = __byte_perm(table, 0u, sel);
            const int64_t k0 = 4 * kb;
            if (aligned && k0 + 3 < n) {
                *reinterpret_cast<uint32_t*>(dst + k0) = out;
            } else {
                for (int e = 0; e < 4 && k0 + e < n; ++e) dst[k0 + e] = (int8_t)(out >> (8 * e));
            }
        }
    }
}

cudaError_t launch_unpack_2bit(const uint8_t* Xp, int64_t n, int64_t mb, const int8_t code[4],
                               int8_t* X, cudaStream_t s) {
    if (mb <= 0) return cudaSuccess;
    uint32_t table = 0;
    for (int c = 0; c < 4; ++c) table |= (uint32_t)(uint8_t)code[c] << (8 * c);
    const unsigned grid = (unsigned)min64(mb, 1 << 20);
    k_unpack_2bit<<<grid, 256, 0, s>>>(Xp, ceil_div(n, 4), n, mb, table, X);
    return cudaGetLastError();
}

}  // namespace gwas
