// Per-cohort setup in FP64: M, its Cholesky factor L, the explicit inverse L^{-1}
// and a generic FP64 GEMM used for the blocked steps (Algorithm 1 before its loop).
//
// FP64 arithmetic stays on the CUDA cores (DFMA): the setup is O(n^3) once per
// cohort, and its stability needs FP64 (Section 2: L L^T := M, triangular solves).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace gwas {

// ----------------------------------------------------------------------------
// a1: M := sigma2 (h Phi + (1-h) I), lower triangle; strict upper triangle := 0.
// ----------------------------------------------------------------------------
__global__ void k_build_M(const double* __restrict__ src, int64_t lds, double* __restrict__ M,
                          int64_t ldm, int64_t n, int is_phi, double h, double sigma2) {
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            double v = 0.0;
            if (i >= j) {
                const double a = src[i + j * lds];
                v = is_phi ? sigma2 * (h * a + (i == j ? 1.0 - h : 0.0)) : a;
            }
            M[i + j * ldm] = v;
        }
    }
}

cudaError_t launch_build_M(const double* src, int64_t lds, double* M, int64_t ldm, int64_t n,
                           int is_phi, double h, double sigma2, cudaStream_t s) {
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(n, 256), 64),
              (unsigned)std::min<int64_t>(n, 65535));
    k_build_M<<<grid, 256, 0, s>>>(src, lds, M, ldm, n, is_phi, h, sigma2);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Generic FP64 GEMM, 64 x 64 output tile per CTA, 256 threads, 4 x 4 per thread.
// Thread (tx, ty) owns rows tx + 16 a and columns ty + 16 b of the tile, so a warp
// stores 16 consecutive rows of a column-major C.
// ----------------------------------------------------------------------------
// acc[a][b] += sum_{k in [kbeg, kend)} op(A)(i0 + tx + 16a, k) op(B)(k, j0 + ty + 16b)
template <bool TA, bool TB>
__device__ __forceinline__ void gemm_tile(const GemmF64& g, int64_t i0, int64_t j0, int64_t kbeg,
                                          int64_t kend, double (&acc)[4][4]) {
    __shared__ double As[KC64][T64 + 1];  // As[k][i] = op(A)(i0 + i, k0 + k)
    __shared__ double Bs[KC64][T64 + 1];  // Bs[k][j] = op(B)(k0 + k, j0 + j)
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    for (int64_t k0 = kbeg; k0 < kend; k0 += KC64) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;
            int ii, kk;
            if (!TA) { ii = e % T64; kk = e / T64; } else { kk = e % KC64; ii = e / KC64; }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < g.M && gk < kend) v = TA ? g.A[gk + gi * g.lda] : g.A[gi + gk * g.lda];
            As[kk][ii] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;
            int jj, kk;
            if (!TB) { kk = e % KC64; jj = e / KC64; } else { jj = e % T64; kk = e / T64; }
            const int64_t gj = j0 + jj, gk = k0 + kk;
            double v = 0.0;
            if (gj < g.N && gk < kend) v = TB ? g.B[gj + gk * g.ldb] : g.B[gk + gj * g.ldb];
            Bs[kk][jj] = v;
        }
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
        __syncthreads();
    }
}

// One 64 x 64 output tile (bi, bj) of C := alpha op(A) op(B) + beta C.
template <bool TA, bool TB>
__device__ __forceinline__ void gemm_tile_job(const GemmF64& g, int64_t bi, int64_t bj) {
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t i0 = bi * T64, j0 = bj * T64;
    if (g.c_lower && j0 > i0) return;
    int64_t kbeg = 0, kend = g.K;
    if (g.a_lower) kend = min64(kend, i0 + T64);
    if (g.a_upper) kbeg = i0;
    if (g.b_lower && j0 > kbeg) kbeg = j0;

    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    gemm_tile<TA, TB>(g, i0, j0, kbeg, kend, acc);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t gi = i0 + tx + 16 * a;
        if (gi >= g.M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t gj = j0 + ty + 16 * b;
            if (gj >= g.N) continue;
            double* c = g.C + gi + gj * g.ldc;
            const double v = g.alpha * acc[a][b];
            *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
        }
    }
}

// Tile (bx, by) of an mt x nt tile grid, renumbered so that with a lower-triangular op(A)
// (a row tile's k-range grows with its row) the heaviest row tiles come first (row tiles
// in descending order, the column fastest) and the long ones do not form the tail.
__device__ __forceinline__ void tile_order(const GemmF64& g, int64_t bx, int64_t by, int64_t mt,
                                           int64_t nt, int64_t& bi, int64_t& bj) {
    bi = bx;
    bj = by;
    if (g.a_lower) {
        const int64_t lin = by * mt + bx;
        bi = mt - 1 - lin / nt;
        bj = lin % nt;
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_f64(GemmF64 g) {
    int64_t bi, bj;
    tile_order(g, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y, bi, bj);
    gemm_tile_job<TA, TB>(g, bi, bj);
}

// Several independent products in one launch (grid z = product); the grid covers the
// largest product's tiles and each CTA outside its own product's tiles returns.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_f64_batched(const GemmF64* __restrict__ gs) {
    const GemmF64 g = gs[blockIdx.z];
    const int64_t mt = (g.M + T64 - 1) / T64, nt = (g.N + T64 - 1) / T64;
    if ((int64_t)blockIdx.x >= mt || (int64_t)blockIdx.y >= nt) return;
    int64_t bi, bj;
    tile_order(g, blockIdx.x, blockIdx.y, mt, nt, bi, bj);
    gemm_tile_job<TA, TB>(g, bi, bj);
}

// Skinny products (one 64 x 64 output tile, long K: the Gram matrices A^T B of n x q
// panels): CTA s accumulates k in [s chunk, (s+1) chunk) into ws[s]; k_splitk_reduce adds
// the slices in ascending s (fixed order) and applies alpha and beta.
__global__ void __launch_bounds__(256) k_gemm_tn_splitk(GemmF64 g, int64_t chunk, double* ws) {
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t kbeg = (int64_t)blockIdx.x * chunk, kend = min64(g.K, kbeg + chunk);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    gemm_tile<true, false>(g, 0, 0, kbeg, kend, acc);
    double* w = ws + (int64_t)blockIdx.x * T64 * T64;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) w[(tx + 16 * a) + (ty + 16 * b) * T64] = acc[a][b];
}

__global__ void k_splitk_reduce(GemmF64 g, int splits, const double* __restrict__ ws) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = e % T64, j = e / T64;
    if (j >= T64 || i >= g.M || j >= g.N) return;
    double sum = 0.0;
    for (int s2 = 0; s2 < splits; ++s2) sum += ws[(int64_t)s2 * T64 * T64 + i + j * T64];
    double* c = g.C + i + (int64_t)j * g.ldc;
    const double v = g.alpha * sum;
    *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
}

// Skinny B (N <= 16 columns, M large: Xbar_L = W X_L, Ybar = W Y, Z = W^T [Xbar_L | Ybar]).
// A 64 x 64 output tile would run these at N/64 of its FP64 work; here a CTA covers all
// NC columns of a few rows, B's k-chunk is staged in shared memory and the partial sums
// over k are added in a fixed order. Grid y = chunks of NC columns.
constexpr int SKB = 64;  // k per staged chunk of B

// op(A) = A: 32 rows x 8 k-slices per CTA (each warp loads 32 consecutive rows of a
// column of A); a lower-triangular A takes its row tiles heaviest first.
template <int NC>
__global__ void __launch_bounds__(256) k_gemm_skinny_n(GemmF64 g) {
    __shared__ double Bs[SKB][NC];
    __shared__ double red[8][32][NC + 1];
    const int tid = threadIdx.x, r = tid % 32, ks = tid / 32;
    const int64_t nbx = gridDim.x;
    const int64_t bx = g.a_lower ? nbx - 1 - blockIdx.x : blockIdx.x;
    const int64_t i0 = bx * 32, i = i0 + r, j0 = (int64_t)blockIdx.y * NC;
    int64_t kbeg = 0, kend = g.K;
    if (g.a_lower) kend = min64(kend, i0 + 32);
    if (g.a_upper) kbeg = i0;
    double acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += SKB) {
        for (int e = tid; e < SKB * NC; e += 256) {
            const int kk = e / NC, jj = e % NC;
            const int64_t k = k0 + kk, j = j0 + jj;
            Bs[kk][jj] = (k < kend && j < g.N) ? g.B[k + j * g.ldb] : 0.0;
        }
        __syncthreads();
        for (int kk = ks; kk < SKB; kk += 8) {
            const int64_t k = k0 + kk;
            const double a = (i < g.M && k < kend) ? g.A[i + k * g.lda] : 0.0;
#pragma unroll
            for (int j = 0; j < NC; ++j) acc[j] = fma(a, Bs[kk][j], acc[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) red[ks][r][j] = acc[j];
    __syncthreads();
    if (ks == 0 && i < g.M) {
        for (int j = 0; j < NC && j0 + j < g.N; ++j) {
            double v = 0.0;
            for (int q = 0; q < 8; ++q) v += red[q][r][j];
            double* c = g.C + i + (j0 + j) * g.ldc;
            *c = (g.beta == 0.0) ? g.alpha * v : fma(g.beta, *c, g.alpha * v);
        }
    }
}

// op(A) = A^T: 8 output rows x 32 k-lanes per CTA (each warp reads 32 consecutive k of one
// column of A); an upper-triangular op(A) starts at the CTA's first row.
template <int NC>
__global__ void __launch_bounds__(256) k_gemm_skinny_t(GemmF64 g) {
    __shared__ double Bs[SKB][NC];
    const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
    const int64_t i0 = (int64_t)blockIdx.x * 8, i = i0 + w, j0 = (int64_t)blockIdx.y * NC;
    int64_t kbeg = 0, kend = g.K;
    if (g.a_upper) kbeg = i0;
    if (g.a_lower) kend = min64(kend, i0 + 8);
    double acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += SKB) {
        for (int e = tid; e < SKB * NC; e += 256) {
            const int kk = e / NC, jj = e % NC;
            const int64_t k = k0 + kk, j = j0 + jj;
            Bs[kk][jj] = (k < kend && j < g.N) ? g.B[k + j * g.ldb] : 0.0;
        }
        __syncthreads();
        for (int kk = lane; kk < SKB; kk += 32) {
            const int64_t k = k0 + kk;
            const double a = (i < g.M && k < kend) ? g.A[k + i * g.lda] : 0.0;
#pragma unroll
            for (int j = 0; j < NC; ++j) acc[j] = fma(a, Bs[kk][j], acc[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        double v = acc[j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        acc[j] = v;
    }
    if (lane == 0 && i < g.M) {
        for (int j = 0; j < NC && j0 + j < g.N; ++j) {
            double* c = g.C + i + (j0 + j) * g.ldc;
            *c = (g.beta == 0.0) ? g.alpha * acc[j] : fma(g.beta, *c, g.alpha * acc[j]);
        }
    }
}

template <int NC>
static cudaError_t launch_skinny(const GemmF64& g, cudaStream_t s) {
    const unsigned gy = (unsigned)ceil_div(g.N, NC);
    if (g.transA) k_gemm_skinny_t<NC><<<dim3((unsigned)ceil_div(g.M, 8), gy), 256, 0, s>>>(g);
    else k_gemm_skinny_n<NC><<<dim3((unsigned)ceil_div(g.M, 32), gy), 256, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t gemm_f64(const GemmF64& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    const bool skinny = g.transA && !g.transB && g.M <= T64 && g.N <= T64 && g.K >= 8192 &&
                        !g.a_lower && !g.a_upper && !g.b_lower && !g.c_lower;
    if (skinny) {
        const int64_t splits = std::min<int64_t>(304, ceil_div(g.K, 256));
        const int64_t chunk = round_up(ceil_div(g.K, splits), KC64);
        const int nsplit = (int)ceil_div(g.K, chunk);
        double* ws = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws),
                                        (size_t)nsplit * T64 * T64 * sizeof(double), s);
        if (e != cudaSuccess) return e;
        k_gemm_tn_splitk<<<(unsigned)nsplit, 256, 0, s>>>(g, chunk, ws);
        k_splitk_reduce<<<T64 * T64 / 256, 256, 0, s>>>(g, nsplit, ws);
        e = cudaGetLastError();
        const cudaError_t f = cudaFreeAsync(ws, s);
        return e != cudaSuccess ? e : f;
    }
    // skinny B: all of its columns per CTA (products of L^{-1} with a few vectors)
    if (!g.transB && g.N <= 16 && g.M >= 256 && g.K >= 256 && !g.b_lower && !g.c_lower) {
        if (g.N <= 4) return launch_skinny<4>(g, s);
        if (g.N <= 8) return launch_skinny<8>(g, s);
        return launch_skinny<16>(g, s);
    }
    dim3 grid((unsigned)ceil_div(g.M, T64), (unsigned)ceil_div(g.N, T64));
    if (!g.transA && !g.transB) k_gemm_f64<false, false><<<grid, 256, 0, s>>>(g);
    else if (!g.transA && g.transB) k_gemm_f64<false, true><<<grid, 256, 0, s>>>(g);
    else if (g.transA && !g.transB) k_gemm_f64<true, false><<<grid, 256, 0, s>>>(g);
    else k_gemm_f64<true, true><<<grid, 256, 0, s>>>(g);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// a2 diagonal block: unblocked Cholesky of one kb x kb block (kb <= 64) in shared
// memory, then D = L_kk^{-1} by recursive halving: the four 16 x 16 diagonal blocks are
// inverted by forward substitution (one thread per column), then merged into 32 x 32 and
// 64 x 64 inverses with [[A, 0], [B, C]]^{-1} = [[A^{-1}, 0], [-C^{-1} B A^{-1}, C^{-1}]].
// ----------------------------------------------------------------------------
constexpr int POTRF_SMEM = (2 * T64 * (T64 + 1) + 32 * 33 + 2 * T64) * (int)sizeof(double);

__global__ void __launch_bounds__(256) k_potrf_diag(double* __restrict__ A, int64_t lda, int kb,
                                                    int64_t base, double* __restrict__ D,
                                                    int* __restrict__ info) {
    // S (64 x 65), Dn (64 x 65), Tm (32 x 33), the pivots and their reciprocals: dynamic
    // shared memory, opted in at launch.
    extern __shared__ double smem_potrf[];
    double (*S)[T64 + 1] = reinterpret_cast<double (*)[T64 + 1]>(smem_potrf);
    double (*Dn)[T64 + 1] = reinterpret_cast<double (*)[T64 + 1]>(smem_potrf + T64 * (T64 + 1));
    double (*Tm)[33] = reinterpret_cast<double (*)[33]>(smem_potrf + 2 * T64 * (T64 + 1));
    double* rinv = smem_potrf + 2 * T64 * (T64 + 1) + 32 * 33;
    double* pv = rinv + T64;
    __shared__ int fail;
    const int tid = threadIdx.x;
    if (tid == 0) fail = -1;
    // rows and columns beyond kb carry the identity, so the 64 x 64 inverse below is that
    // of [[L_kk, 0], [0, I]]; they are written back as zeros
    for (int e = tid; e < T64 * T64; e += blockDim.x) {
        const int i = e % T64, j = e / T64;
        S[i][j] = (i < kb && j < kb && i >= j) ? A[i + j * lda] : (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        // one thread takes the pivot and its reciprocal (FP64 square roots and divisions
        // are slow on this part: 256 redundant ones cost more than the barrier); the
        // pivots go to pv and replace the diagonal at the end
        if (tid == 0) {
            const double d = S[j][j];
            const double piv = d > 0.0 ? sqrt(d) : nan("");
            pv[j] = piv;
            rinv[j] = 1.0 / piv;
            if (!(d > 0.0) && fail < 0) fail = j;
        }
        __syncthreads();
        const double rp = rinv[j];
        for (int i = j + 1 + tid; i < kb; i += blockDim.x) S[i][j] *= rp;
        __syncthreads();
        const int w = kb - j - 1;  // trailing (w x w) lower update
        for (int e = tid; e < w * w; e += blockDim.x) {
            const int i = j + 1 + e % w, k = j + 1 + e / w;
            if (i >= k) S[i][k] -= S[i][j] * S[k][j];
        }
        __syncthreads();
    }
    if (tid >= kb && tid < T64) rinv[tid] = 1.0;  // the identity rows
    if (tid < kb) S[tid][tid] = pv[tid];
    __syncthreads();

    // 16 x 16 diagonal blocks: thread (b, c) solves L_bb d = e_c, its column in registers
    if (tid < T64) {
        const int b = tid / 16, c = tid % 16, o = 16 * b;
        double dc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < i; ++k) acc = fma(S[o + i][o + k], dc[k], acc);
            dc[i] = ((i == c ? 1.0 : 0.0) - acc) * rinv[o + i];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) Dn[o + i][o + c] = dc[i];
    }
    // strictly upper parts stay zero
    for (int e = tid; e < T64 * T64; e += blockDim.x) {
        const int i = e % T64, j = e / T64;
        if (i / 16 <= j / 16 && !(i / 16 == j / 16)) Dn[i][j] = 0.0;
    }
    __syncthreads();
    // merge pairs of h x h inverses into 2h x 2h ones, h = 16 then 32
    for (int h = 16; h < T64; h *= 2) {
        const int nb = T64 / (2 * h);          // merged blocks at this level
        const int outs = nb * h * h;           // entries of B A^{-1} (and of the new block)
        // Tm = B A^{-1}: B = L[o+h .. o+2h, o .. o+h], A^{-1} = Dn[o .. o+h, o .. o+h]
        for (int e = tid; e < outs; e += blockDim.x) {
            const int m = e / (h * h), r = e % (h * h), i = r % h, j = r / h, o = 2 * h * m;
            double acc = 0.0;
            for (int k = j; k < h; ++k) acc = fma(S[o + h + i][o + k], Dn[o + k][o + j], acc);
            Tm[m * h + i][j] = acc;            // nb * h = 32 rows of Tm
        }
        __syncthreads();
        // Dn[o+h .., o ..] = -C^{-1} Tm with C^{-1} = Dn[o+h .., o+h ..] (lower)
        for (int e = tid; e < outs; e += blockDim.x) {
            const int m = e / (h * h), r = e % (h * h), i = r % h, j = r / h, o = 2 * h * m;
            double acc = 0.0;
            for (int k = 0; k <= i; ++k) acc = fma(Dn[o + h + i][o + h + k], Tm[m * h + k][j], acc);
            Dn[o + h + i][o + j] = -acc;
        }
        __syncthreads();
    }
    for (int e = tid; e < T64 * T64; e += blockDim.x) {
        const int i = e % T64, j = e / T64;
        if (i < kb && j < kb) A[i + j * lda] = (i >= j) ? S[i][j] : 0.0;
        D[i + j * T64] = (i < kb && j < kb) ? Dn[i][j] : 0.0;
    }
    if (tid == 0 && fail >= 0) atomicMin(info, (int)(base + fail));
}

// Two-level right-looking blocked Cholesky: panels of NB = 256 columns, each factored in
// 64-column blocks (diagonal block in shared memory, the rows below by D_k^T, then the
// rank-64 update of the panel's remaining columns only); the columns right of the panel
// get one rank-NB update per panel, so the large trailing GEMMs run with K = 256.
namespace {

constexpr int64_t CHOL_NB = 4 * T64;  // panel width

// Panel [p0, pend) of the factor, in 64-column blocks: the diagonal block in shared memory
// (D_k = L_kk^{-1} into Dinv), the rows below it by D_k^T, then the rank-64 update of the
// panel's remaining columns only.
cudaError_t factor_panel(double* A, int64_t lda, int64_t n, int64_t p0, int64_t pend, double* Dinv,
                         int* d_info, cudaStream_t s, int64_t& nl) {
    cudaError_t e;
    for (int64_t k0 = p0; k0 < pend; k0 += T64) {
        const int kb = (int)std::min<int64_t>(T64, n - k0);
        double* Akk = A + k0 + k0 * lda;
        double* Dk = Dinv + (k0 / T64) * T64 * T64;
        k_potrf_diag<<<1, 256, POTRF_SMEM, s>>>(Akk, lda, kb, k0, Dk, d_info);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int64_t below = n - k0 - kb;
        if (below <= 0) break;
        double* P = A + (k0 + kb) + k0 * lda;  // rows below the block
        // L_ik := A_ik L_kk^{-T} = A_ik D_k^T (one column tile: in place is safe)
        GemmF64 g;
        g.M = below; g.N = kb; g.K = kb;
        g.A = P; g.lda = lda; g.B = Dk; g.ldb = T64; g.transB = true;
        g.C = P; g.ldc = lda;
        if ((e = gemm_f64(g, s)) != cudaSuccess) return e;
        ++nl;
        // the panel's remaining columns [k0 + kb, pend) -= L_below L_(those rows)^T
        const int64_t w = pend - (k0 + kb);
        if (w > 0) {
            GemmF64 u;
            u.M = below; u.N = w; u.K = kb;
            u.A = P; u.lda = lda; u.B = P; u.ldb = lda; u.transB = true;
            u.C = A + (k0 + kb) + (k0 + kb) * lda; u.ldc = lda;
            u.alpha = -1.0; u.beta = 1.0; u.c_lower = true;
            if ((e = gemm_f64(u, s)) != cudaSuccess) return e;
            ++nl;
        }
    }
    return cudaSuccess;
}

// Columns [c0, c1) of the trailing matrix, rows c0 .. n-1 (lower tiles only):
// A(c0:, c0:c1) -= L(c0:, p0:pend) L(c0:c1, p0:pend)^T. Every 64 x 64 output tile of a
// column range sits on the same grid from the diagonal and sums over the same k order,
// so splitting [pend, n) into column ranges leaves each element's arithmetic unchanged.
cudaError_t trailing_update(double* A, int64_t lda, int64_t n, int64_t p0, int64_t pend,
                            int64_t c0, int64_t c1, cudaStream_t s, int64_t& nl) {
    if (c1 <= c0) return cudaSuccess;
    const double* Q = A + c0 + p0 * lda;
    GemmF64 u;
    u.M = n - c0; u.N = c1 - c0; u.K = pend - p0;
    u.A = Q; u.lda = lda; u.B = Q; u.ldb = lda; u.transB = true;
    u.C = A + c0 + c0 * lda; u.ldc = lda;
    u.alpha = -1.0; u.beta = 1.0; u.c_lower = true;
    ++nl;
    return gemm_f64(u, s);
}

}  // namespace

cudaError_t cholesky_blocked(double* A, int64_t lda, int64_t n, double* Dinv, int* d_info,
                             cudaStream_t s, int64_t* launches, const CholLookahead* la) {
    int64_t nl = 0;
    cudaError_t e = cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         POTRF_SMEM);
    if (e != cudaSuccess) return e;
    if (!la || !la->panel) {
        for (int64_t p0 = 0; p0 < n; p0 += CHOL_NB) {
            const int64_t pend = std::min<int64_t>(n, p0 + CHOL_NB);
            if ((e = factor_panel(A, lda, n, p0, pend, Dinv, d_info, s, nl)) != cudaSuccess) return e;
            if ((e = trailing_update(A, lda, n, p0, pend, pend, n, s, nl)) != cudaSuccess) return e;
        }
        if (launches) *launches += nl;
        return cudaSuccess;
    }
    // Lookahead by one panel. Panel p's trailing update is split at the end of panel p+1:
    // (a) its columns [pend, pend2) go on the panel stream, right before panel p+1 is
    // factored there; (b) the columns [pend2, n) go on s. Panel p+1 (and (a)) also need
    // panel p-1's (b), which updated the same columns, so the panel stream waits for it
    // first; (b) of panel p then runs on s beside (a) and the factorisation of panel p+1.
    cudaStream_t sp = la->panel;
    cudaEvent_t ev_start = la->ev[0], ev_panel = la->ev[1], ev_rest = la->ev[2];
#define CKL(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
    CKL(cudaEventRecord(ev_start, s));
    CKL(cudaStreamWaitEvent(sp, ev_start, 0));
    bool rest_pending = false;  // a (b) update on s that the panel stream has not waited for
    for (int64_t p0 = 0; p0 < n; p0 += CHOL_NB) {
        const int64_t pend = std::min<int64_t>(n, p0 + CHOL_NB);
        CKL(factor_panel(A, lda, n, p0, pend, Dinv, d_info, sp, nl));
        if (pend >= n) break;
        const int64_t pend2 = std::min<int64_t>(n, pend + CHOL_NB);
        CKL(cudaEventRecord(ev_panel, sp));
        if (rest_pending) CKL(cudaStreamWaitEvent(sp, ev_rest, 0));  // panel p-1's (b)
        CKL(cudaStreamWaitEvent(s, ev_panel, 0));
        rest_pending = false;
        if (pend2 < n) {
            CKL(trailing_update(A, lda, n, p0, pend, pend2, n, s, nl));  // (b)
            CKL(cudaEventRecord(ev_rest, s));
            rest_pending = true;
        }
        CKL(trailing_update(A, lda, n, p0, pend, pend, pend2, sp, nl));  // (a)
    }
    CKL(cudaEventRecord(ev_panel, sp));
    CKL(cudaStreamWaitEvent(s, ev_panel, 0));
#undef CKL
    if (launches) *launches += nl;
    return cudaSuccess;
}

// ----------------------------------------------------------------------------
// a3: W := L^{-1} by recursive halving on 64-aligned splits,
//   [[L11, 0], [L21, L22]]^{-1} = [[W11, 0], [-W22 L21 W11, W22]],
// evaluated level by level from the leaves (the 64 x 64 diagonal inverses D_k) up: the
// nodes of one level are independent, so each level is two batched launches over all
// of its nodes (T := L21 W11, then W21 := -W22 T) instead of two launches per node.
// ----------------------------------------------------------------------------
__global__ void k_copy_diag_inv(const double* __restrict__ Dinv, int64_t n, double* __restrict__ W,
                                int64_t ldw) {
    const int64_t r0 = (int64_t)blockIdx.x * T64;
    const int kb = (int)min64(T64, n - r0);
    const double* D = Dinv + (int64_t)blockIdx.x * T64 * T64;
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
        const int i = e % kb, j = e / kb;
        W[(r0 + i) + (r0 + j) * ldw] = D[i + j * T64];
    }
}

namespace {

struct TrtriNode {
    int64_t r0, s1, s2;
};

void trtri_nodes(int64_t r0, int64_t size, size_t depth, std::vector<std::vector<TrtriNode>>& lv) {
    if (size <= T64) return;
    const int64_t s1 = round_up(ceil_div(size, 2), T64);
    const int64_t s2 = size - s1;
    if (lv.size() <= depth) lv.resize(depth + 1);
    lv[depth].push_back({r0, s1, s2});
    trtri_nodes(r0, s1, depth + 1, lv);
    trtri_nodes(r0 + s1, s2, depth + 1, lv);
}

}  // namespace

cudaError_t trtri_lower(const double* L, int64_t ldl, int64_t n, const double* Dinv, double* W,
                        int64_t ldw, double* tmp, cudaStream_t s, int64_t* launches) {
    int64_t nl = 0;
    const int64_t nt = ceil_div(n, T64);
    k_copy_diag_inv<<<(unsigned)nt, 256, 0, s>>>(Dinv, n, W, ldw);
    ++nl;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::vector<std::vector<TrtriNode>> lv;
    trtri_nodes(0, n, 0, lv);
    // descriptors level by level: the level's T products, then its W21 products; each
    // node's T gets its own part of tmp (a level's T blocks take at most (n/2)^2 doubles,
    // the size of tmp)
    std::vector<GemmF64> gs;
    std::vector<size_t> level_first;
    for (size_t d = 0; d < lv.size(); ++d) {
        level_first.push_back(gs.size());
        std::vector<GemmF64> wprod;
        int64_t off = 0;
        for (const TrtriNode& nd : lv[d]) {
            GemmF64 g;  // T := L21 W11   (s2 x s1; W11 lower triangular)
            g.M = nd.s2; g.N = nd.s1; g.K = nd.s1;
            g.A = L + (nd.r0 + nd.s1) + nd.r0 * ldl; g.lda = ldl;
            g.B = W + nd.r0 + nd.r0 * ldw; g.ldb = ldw; g.b_lower = true;
            g.C = tmp + off; g.ldc = nd.s2;
            GemmF64 h;  // W21 := -W22 T   (W22 lower triangular)
            h.M = nd.s2; h.N = nd.s1; h.K = nd.s2;
            h.A = W + (nd.r0 + nd.s1) + (nd.r0 + nd.s1) * ldw; h.lda = ldw; h.a_lower = true;
            h.B = tmp + off; h.ldb = nd.s2;
            h.C = W + (nd.r0 + nd.s1) + nd.r0 * ldw; h.ldc = ldw; h.alpha = -1.0;
            gs.push_back(g);
            wprod.push_back(h);
            off += nd.s2 * nd.s1;
        }
        gs.insert(gs.end(), wprod.begin(), wprod.end());
    }
    level_first.push_back(gs.size());
    if (gs.empty()) {
        if (launches) *launches += nl;
        return cudaSuccess;
    }
    GemmF64* d_gs = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&d_gs), gs.size() * sizeof(GemmF64), s)) !=
        cudaSuccess)
        return e;
    e = cudaMemcpyAsync(d_gs, gs.data(), gs.size() * sizeof(GemmF64), cudaMemcpyHostToDevice, s);
    for (size_t d = lv.size(); e == cudaSuccess && d-- > 0;) {
        const size_t first = level_first[d], count = (level_first[d + 1] - first) / 2;
        int64_t mt = 0, ntl = 0;  // both products of a node have the same s2 x s1 shape
        for (size_t k = 0; k < count; ++k) {
            mt = std::max(mt, ceil_div(gs[first + k].M, T64));
            ntl = std::max(ntl, ceil_div(gs[first + k].N, T64));
        }
        const dim3 grid((unsigned)mt, (unsigned)ntl, (unsigned)count);
        k_gemm_f64_batched<false, false><<<grid, 256, 0, s>>>(d_gs + first);          // T
        k_gemm_f64_batched<false, false><<<grid, 256, 0, s>>>(d_gs + first + count);  // W21
        nl += 2;
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(d_gs, s);
    if (launches) *launches += nl;
    return e != cudaSuccess ? e : f;
}

}  // namespace gwas
