// Helpers of the mixed-precision path that run outside its dominant kernel: the int8
// dosage -> BF16 conversion of each block, and the once-per-cohort split of L^{-1} (row
// tiles) and Z = M^-1 [X_L | Y] (linear rows) into BF16 integer limbs with one power-of-two
// exponent per tile (the limb representation used by k_block_mixed).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gwas {

// ----------------------------------------------------------------------------
// Dosages -> BF16 rows (one SNP per row, k contiguous), flags for bad dosages.
// ----------------------------------------------------------------------------
// One warp converts one SNP row: n dosages -> BF16 (0 -> 0x0000, 1 -> 0x3F80, 2 -> 0x4000),
// returns the row's flags (warp-wide): FLAG_BAD_DOSAGE if a dosage is not in {0,1,2},
// FLAG_CONSTANT if every dosage equals the first. A row that starts on a 16-byte
// boundary is read 16 dosages per lane (coalesced 512-byte warp loads); the remainder,
// or a whole unaligned row, one dosage per lane.
__device__ __forceinline__ uint32_t bf16_pair(uint32_t v) {
    // v holds two 16-bit lanes with values in {0,1,2}: each becomes v * 0x80 + (v != 0) * 0x3F00
    const uint32_t nz = (v | (v >> 1)) & 0x00010001u;
    return v * 0x80u + nz * 0x3F00u;
}

__device__ __forceinline__ uint32_t bad_bytes(uint32_t w) {
    // nonzero iff a byte of w is >= 3: some bit above bit 1 set, or bits 0 and 1 both set
    return (w & 0xFCFCFCFCu) | (w & (w >> 1) & 0x01010101u);
}

// 16 dosages -> flags and 32 bytes of BF16 at dst (32-byte aligned).
__device__ __forceinline__ void geno_chunk16(const uint32_t (&in)[4], uint32_t first4,
                                             uint32_t& flag, uint32_t& differ, uint4* d) {
    uint32_t o[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        flag |= bad_bytes(in[e]);
        differ |= in[e] ^ first4;
        o[2 * e] = bf16_pair(__byte_perm(in[e], 0u, 0x4140));
        o[2 * e + 1] = bf16_pair(__byte_perm(in[e], 0u, 0x4342));
    }
    d[0] = make_uint4(o[0], o[1], o[2], o[3]);
    d[1] = make_uint4(o[4], o[5], o[6], o[7]);
}

__device__ __forceinline__ int geno_row_warp(const int8_t* __restrict__ src, int64_t n,
                                             uint16_t* __restrict__ dst) {
    const int lane = threadIdx.x % 32;
    const uint32_t first = (uint32_t)(uint8_t)src[0];
    const uint32_t first4 = first * 0x01010101u;
    uint32_t flag = 0, differ = 0;
    uint4* d4 = reinterpret_cast<uint4*>(dst);  // BF16 rows start on 128-byte boundaries
    // dosages [head, body) go through 16-dosage chunks, the rest one per lane
    int64_t head = 0, body = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        body = (n / 16) * 16;
        for (int64_t v = lane; v < n / 16; v += 32) {
            const uint4 w = __ldg(s4 + v);
            const uint32_t in[4] = {w.x, w.y, w.z, w.w};
            geno_chunk16(in, first4, flag, differ, d4 + 2 * v);
        }
    } else {
        // A row off a 16-byte boundary (n not a multiple of 16): chunk v >= 1 is assembled
        // from the five aligned 32-bit words around it with byte perms. Those words hold
        // row bytes 16v - 3 .. 16v + 19 at most, so chunk v is taken while 16v + 19 < n
        // (chunk 0 and the tail go one dosage per lane).
        const int mis = (int)(reinterpret_cast<uintptr_t>(src) & 3);
        const uint32_t* wb = reinterpret_cast<const uint32_t*>(src - mis);
        const uint32_t sel = (uint32_t)mis | ((uint32_t)(mis + 1) << 4) |
                             ((uint32_t)(mis + 2) << 8) | ((uint32_t)(mis + 3) << 12);
        const int64_t vmax = n >= 20 ? (n - 20) / 16 + 1 : 1;
        head = n < 16 ? n : 16;
        body = 16 * vmax;
        for (int64_t v = 1 + lane; v < vmax; v += 32) {
            uint32_t a[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) a[k] = __ldg(wb + 4 * v + k);
            uint32_t in[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) in[k] = __byte_perm(a[k], a[k + 1], sel);
            geno_chunk16(in, first4, flag, differ, d4 + 2 * v);
        }
    }
    auto one = [&](int64_t k) {
        const uint32_t v = (uint32_t)(uint8_t)src[k];
        flag |= v > 2u ? 1u : 0u;
        differ |= v ^ first;
        dst[k] = (uint16_t)bf16_pair(v);
    };
    if (head > 0) {
        for (int64_t k = lane; k < head; k += 32) one(k);
        for (int64_t k = (body > head ? body : head) + lane; k < n; k += 32) one(k);
    } else {
        for (int64_t k = body + lane; k < n; k += 32) one(k);
    }
    const bool bad = __any_sync(0xffffffffu, flag != 0);
    const bool varies = __any_sync(0xffffffffu, differ != 0);
    return (bad ? FLAG_BAD_DOSAGE : 0) | (varies ? 0 : FLAG_CONSTANT);
}

constexpr int GENO_WARPS = 8;

__global__ void __launch_bounds__(GENO_WARPS * 32)
k_geno_bf16(const int8_t* __restrict__ X, int64_t ldx, int64_t n, int64_t mb,
            uint16_t* __restrict__ Xb, int64_t n_pad, uint8_t* __restrict__ bad) {
    const int64_t w0 = (int64_t)blockIdx.x * GENO_WARPS + threadIdx.x / 32;
    for (int64_t j = w0; j < mb; j += (int64_t)gridDim.x * GENO_WARPS) {
        const int flags = geno_row_warp(X + j * ldx, n, Xb + j * n_pad);
        if (threadIdx.x % 32 == 0) bad[j] = (uint8_t)flags;
    }
}

// Batched cohorts: one warp per SNP of every cohort that owns its BF16 rows.
__global__ void __launch_bounds__(GENO_WARPS * 32)
k_geno_bf16_batch(const BatchJob* __restrict__ jobs, int n_jobs, int64_t n_snps) {
    const int64_t w0 = (int64_t)blockIdx.x * GENO_WARPS + threadIdx.x / 32;
    for (int64_t g = w0; g < n_snps; g += (int64_t)gridDim.x * GENO_WARPS) {
        int lo = 0, hi = n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (jobs[mid].snp_base <= g) lo = mid;
            else hi = mid - 1;
        }
        const BatchJob& jb = jobs[lo];
        const int64_t j = g - jb.snp_base;
        if (j >= jb.mb || !jb.convert) continue;  // uniform across the warp
        const int flags = geno_row_warp(jb.X + j * jb.c.n, jb.c.n, jb.Xb + j * jb.n_pad);
        if (threadIdx.x % 32 == 0) jb.bad[j] = (uint8_t)flags;
    }
}

// ----------------------------------------------------------------------------
// Exponents and limb split of L^{-1} (row tiles) and of Z (linear rows).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_absmax_w(const double* __restrict__ W, int64_t ldw, int64_t n, int R, int off,
           unsigned long long* bits) {
    // grid: x = k chunks of 256, y = row tile of R rows (tile rt holds rows rt R - off ..,
    // so the first tile is the short one); elements (i, k) of the tile's lower part, i
    // fastest (coalesced along the column-major rows)
    const int rt = blockIdx.y;
    const int64_t r0 = (int64_t)rt * R - off, k0 = (int64_t)blockIdx.x * 256;
    double m = 0.0;
    for (int e = threadIdx.x; e < R * 256; e += blockDim.x) {
        const int64_t r = r0 + e % R, k = k0 + e / R;
        if (r >= 0 && r < n && k <= r) m = fmax(m, fabs(W[r + k * ldw]));
    }
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && red[0] > 0.0)
        atomicMax(&bits[rt], (unsigned long long)__double_as_longlong(red[0]));
}

__global__ void __launch_bounds__(256)
k_absmax_z(const double* __restrict__ Z, int64_t n, unsigned long long* bits) {
    const int j = blockIdx.y;
    double m = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(Z[k + (int64_t)j * n]));
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && red[0] > 0.0)
        atomicMax(&bits[j], (unsigned long long)__double_as_longlong(red[0]));
}

// E with max|.| <= 2^E (frexp exponent); 0 for an all-zero tile.
__global__ void k_exponents(const unsigned long long* bits, int count, int* E) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int e = 0;
    const double m = __longlong_as_double((long long)bits[i]);
    if (m > 0.0) frexp(m, &e);
    E[i] = e;
}

// w = 2^(E-(B-1)) sum_l A_l 2^(-B l) + O(2^(E-BS)), A_l integers in [-2^(B-1), 2^(B-1)]
// (|w| <= 2^E; B = 7..9 bits per limb).
template <int S>
__device__ __forceinline__ void split_limbs(double w, int E, int B, uint16_t (&out)[S]) {
    double r = ldexp(w, (B - 1) - E);  // |r| <= 2^(B-1)
    const double base = ldexp(1.0, B);
#pragma unroll
    for (int l = 0; l < S; ++l) {
        const double a = rint(r);
        r = (r - a) * base;  // exact: |r - a| <= 1/2
        // |a| <= 256 has at most 9 significant bits: the top half of its FP32 pattern
        // is its exact BF16 pattern
        out[l] = (uint16_t)(__float_as_uint((float)a) >> 16);
    }
}

// Lower triangle of W (column-major) -> limb rows rt*NT + i*S + l of WL (k contiguous):
// R rows of L^{-1} per tile, row r in tile rt = (r + off) / R at i = (r + off) % R (the
// tiles end at row n, the first one is short), the S limbs of row i side by side, row tiles
// NT rows apart.
template <int S>
__global__ void __launch_bounds__(256)
k_split_w(const double* __restrict__ W, int64_t ldw, int64_t n, int R, int off, int NT, int B,
          const int* __restrict__ E_w, uint16_t* __restrict__ WL, int64_t n_pad) {
    __shared__ double tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
    if (k0 > r0 + 31) return;  // strictly upper tile: stays zero
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    for (int j = ty; j < 32; j += 8) {
        const int64_t r = r0 + tx, k = k0 + j;
        tile[j][tx] = (r < n && k < n && k <= r) ? W[r + k * ldw] : 0.0;
    }
    __syncthreads();
    const int64_t N = NT;
    for (int j = ty; j < 32; j += 8) {
        const int64_t r = r0 + j, k = k0 + tx;
        if (r >= n || k >= n || k > r) continue;
        const int64_t rt = (r + off) / R, i = (r + off) % R;
        uint16_t limbs[S];
        split_limbs<S>(tile[tx][j], E_w[rt], B, limbs);
#pragma unroll
        for (int l = 0; l < S; ++l) WL[(rt * N + i * S + l) * n_pad + k] = limbs[l];
    }
}

// Z (n x R_e, column-major) -> limb rows base + j*sj + l*sl of WL: a separate linear tile
// (limb-major, sj = 1, sl = R_e) or the last rows of the last row tile (the limbs of a
// linear row side by side like those of a row of L^{-1}, sj = S, sl = 1).
template <int S>
__global__ void __launch_bounds__(256)
k_split_z(const double* __restrict__ Z, int64_t n, int B, const int* __restrict__ E_e,
          uint16_t* __restrict__ WL, int64_t n_pad, int64_t base_row, int sj, int sl) {
    const int j = blockIdx.y;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint16_t limbs[S];
        split_limbs<S>(Z[k + (int64_t)j * n], E_e[j], B, limbs);
#pragma unroll
        for (int l = 0; l < S; ++l)
            WL[(base_row + (int64_t)j * sj + (int64_t)l * sl) * n_pad + k] = limbs[l];
    }
}

// Fused linear rows: exponent per (row tile rt, linear row j) over k in the tile's range.
__global__ void __launch_bounds__(256)
k_absmax_zf(const double* __restrict__ Z, int64_t n, int R, int off, unsigned long long* bits) {
    const int rt = blockIdx.x, j = blockIdx.y, R_e = gridDim.y;
    const int64_t k1 = min64(n, (int64_t)(rt + 1) * R - off);
    const int64_t k0 = (int64_t)rt * R - off < 0 ? 0 : (int64_t)rt * R - off;
    double m = 0.0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) m = fmax(m, fabs(Z[k + (int64_t)j * n]));
    __shared__ double red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && red[0] > 0.0)
        atomicMax(&bits[(int64_t)rt * R_e + j], (unsigned long long)__double_as_longlong(red[0]));
}

// Z (n x R_e) -> for every k, limb rows rt*NT + R*S + l*R_e + j of row tile
// rt = (k + off) / R: each tile carries Z only on its own k-range (the k of its own rows),
// so the tiles' partial sums add up to Z^T x.
template <int S>
__global__ void __launch_bounds__(256)
k_split_zf(const double* __restrict__ Z, int64_t n, int R, int off, int NT, int R_e, int B,
           const int* __restrict__ E_e, uint16_t* __restrict__ WL, int64_t n_pad) {
    const int j = blockIdx.y;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rt = (k + off) / R;
        uint16_t limbs[S];
        split_limbs<S>(Z[k + (int64_t)j * n], E_e[rt * R_e + j], B, limbs);
#pragma unroll
        for (int l = 0; l < S; ++l)
            WL[(rt * NT + (int64_t)R * S + (int64_t)l * R_e + j) * n_pad + k] = limbs[l];
    }
}

// ----------------------------------------------------------------------------
// Host launchers.
// ----------------------------------------------------------------------------
cudaError_t launch_limb_split(MixedDev& m, const double* W, int64_t ldw, const double* Z,
                              cudaStream_t s, int64_t* launches) {
    cudaError_t e;
    const int64_t n = m.n;
    if ((e = cudaMemsetAsync(m.WL, 0, (size_t)m.rows_total * m.n_pad * 2, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.bits, 0, (size_t)m.n_exp() * 8, s)) != cudaSuccess) return e;
    const int off = m.row_off();
    k_absmax_w<<<dim3((unsigned)ceil_div(n, 256), (unsigned)m.n_rt), 256, 0, s>>>(W, ldw, n, m.R,
                                                                                 off, m.bits);
    if (m.fused)
        k_absmax_zf<<<dim3((unsigned)m.n_rt, (unsigned)m.R_e), 256, 0, s>>>(Z, n, m.R, off,
                                                                           m.bits + m.n_rt);
    else
        k_absmax_z<<<dim3(64, (unsigned)m.R_e), 256, 0, s>>>(Z, n, m.bits + m.n_rt);
    k_exponents<<<(unsigned)ceil_div(m.n_exp(), 128), 128, 0, s>>>(m.bits, m.n_exp(), m.E);
    const dim3 gw((unsigned)ceil_div(n, 32), (unsigned)ceil_div((int64_t)m.n_rt * m.R, 32));
    const dim3 gz(64, (unsigned)m.R_e);
    // a separate linear tile after the row tiles, or the last R_e rows of the last row tile
    const int64_t zbase = m.ztail ? (int64_t)(m.n_rt - 1) * m.NT + (int64_t)(m.R - m.R_e) * m.S
                                  : (int64_t)m.n_rt * m.NT;
    const int zsj = m.ztail ? m.S : 1, zsl = m.ztail ? 1 : m.R_e;
#define GWAS_SPLIT(SS)                                                                       \
    k_split_w<SS><<<gw, 256, 0, s>>>(W, ldw, n, m.R, off, m.NT, m.radix, m.E, m.WL, m.n_pad); \
    if (m.fused)                                                                             \
        k_split_zf<SS><<<gz, 256, 0, s>>>(Z, n, m.R, off, m.NT, m.R_e, m.radix, m.E + m.n_rt,   \
                                          m.WL, m.n_pad);                                    \
    else                                                                                     \
        k_split_z<SS><<<gz, 256, 0, s>>>(Z, n, m.radix, m.E + m.n_rt, m.WL, m.n_pad, zbase,     \
                                         zsj, zsl);
    switch (m.S) {
        case 2: GWAS_SPLIT(2) break;
        case 3: GWAS_SPLIT(3) break;
        case 4: GWAS_SPLIT(4) break;
        case 5: GWAS_SPLIT(5) break;
        default:
            return cudaErrorInvalidValue;
    }
#undef GWAS_SPLIT
    if (launches) *launches += 6;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_geno_bf16(const MixedDev& m, const int8_t* X, int64_t ldx, int64_t mb,
                             uint8_t* bad, cudaStream_t s, int64_t snp0) {
    const int64_t count = mb - snp0;
    if (count <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(count, GENO_WARPS), 1 << 20);
    k_geno_bf16<<<grid, GENO_WARPS * 32, 0, s>>>(X + snp0 * ldx, ldx, m.n, count,
                                                 m.Xb + snp0 * m.n_pad, m.n_pad, bad + snp0);
    return cudaGetLastError();
}

cudaError_t launch_geno_bf16_batch(const BatchJob* jobs, int n_jobs, int64_t n_snps,
                                   cudaStream_t s) {
    if (n_snps <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n_snps, GENO_WARPS), 1 << 20);
    k_geno_bf16_batch<<<grid, GENO_WARPS * 32, 0, s>>>(jobs, n_jobs, n_snps);
    return cudaGetLastError();
}

}  // namespace gwas
