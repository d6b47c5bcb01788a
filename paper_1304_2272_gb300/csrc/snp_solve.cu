// Per-SNP tail of Algorithm 1's loop (Section 2.1): add the row-tile partial sums,
// set S_i = [[S_TL, *], [S_BLi, S_BRi]] and bbar_i = [bbar_T; bbar_Bi], and solve
// S_i b_i = bbar_i through a p x p Cholesky factorisation (Section 2, sixth step).
// The row-tile partials are first added by k_reduce_partials (many warps per SNP group,
// fixed order), then one thread per SNP forms and solves S_i, everything in FP64.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace gwas {

// Singular S_i: a Cholesky pivot at or below this fraction of max_j S_jj.
constexpr double SINGULAR_RTOL = 1e-12;

// The row-tile partials of one reduction value: value v of SNP i is
// sum_{r < count} base[r * stride + i].
struct PartialSet {
    double* base;
    int64_t stride;
    int count;
};

// Reduction value v of SNP i (v < q: S_BLi[v]; v == q: S_BRi; v > q: bbar_Bi[v-q-1]).
// FP64 path: every value is a sum of per-row-tile partials.
struct RedFp64 {
    const double* part;
    int64_t ldp;
    int n_tiles;
    int nred;
    __device__ PartialSet set(int v) const {
        return {const_cast<double*>(part) + (int64_t)v * ldp, (int64_t)nred * ldp, n_tiles};
    }
    __device__ double operator()(int v, int64_t i) const {
        double s = 0.0;
        for (int r = 0; r < n_tiles; ++r) s += part[((int64_t)r * nred + v) * ldp + i];
        return s;
    }
};

// Mixed path: S_BRi from row-tile partials, the linear terms come whole.
struct RedMixed {
    const double* sq;
    const double* lin;
    int64_t ldp;
    int n_tiles;
    int q;
    int lin_tiles;  // 1: whole linear values; n_tiles: one partial per row tile
    int R_e;
    __device__ PartialSet set(int v) const {
        if (v == q) return {const_cast<double*>(sq), ldp, n_tiles};
        const int j = v < q ? v : v - 1;
        return {const_cast<double*>(lin) + (int64_t)j * ldp, (int64_t)R_e * ldp, lin_tiles};
    }
    __device__ double operator()(int v, int64_t i) const {
        if (v == q) {
            double s = 0.0;
            for (int r = 0; r < n_tiles; ++r) s += sq[(int64_t)r * ldp + i];
            return s;
        }
        const int j = v < q ? v : v - 1;
        double s = 0.0;
        for (int r = 0; r < lin_tiles; ++r) s += lin[((int64_t)r * R_e + j) * ldp + i];
        return s;
    }
};

// P > 0: p known at compile time (every loop unrolls, the p x p factor lives in
// registers); P = 0: any p <= MAX_P (arrays in local memory).
template <int P, class Red>
__device__ __forceinline__ void solve_snp(const CohortDev& c, const Red& red,
                                          const uint8_t* __restrict__ bad, int64_t i,
                                          double* __restrict__ b, double* __restrict__ wald,
                                          uint8_t* __restrict__ status,
                                          double* __restrict__ cov = nullptr) {
    constexpr int PM = P > 0 ? P : MAX_P;
    const int p = P > 0 ? P : c.q + 1;
    const int q = p - 1, t = c.t;

    double sbl[PM];  // S_BLi (q values) then S_BRi
#pragma unroll
    for (int v = 0; v < p; ++v) sbl[v] = red(v, i);
    // C C^T = S_i (C lower triangular, column by column).
    double C[PM][PM];
    double rc[PM];   // 1 / C_jj: one FP64 division per pivot (division is costly here)
    double smax = sbl[q];
#pragma unroll
    for (int a = 0; a < q; ++a) smax = fmax(smax, c.S_TL[a + a * q]);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < p; ++j) {
        double d = (j < q) ? c.S_TL[j + j * q] : sbl[q];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= C[j][k] * C[j][k];
        if (!(d > SINGULAR_RTOL * smax)) { ok = false; d = 1.0; }
        C[j][j] = sqrt(d);
        rc[j] = 1.0 / C[j][j];
#pragma unroll
        for (int r = j + 1; r < p; ++r) {
            double s = (r < q) ? c.S_TL[r + j * q] : sbl[j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= C[r][k] * C[j][k];
            C[r][j] = s * rc[j];
        }
    }
    const uint8_t fl = bad[i];
    const bool collinear = (fl & FLAG_CONSTANT) && c.ones_singular;
    const uint8_t st = (fl & FLAG_BAD_DOSAGE) ? 2 : ((ok && !collinear) ? 0 : 1);
    const double nanv = nan("");
    const double cpp2 = C[p - 1][p - 1] * C[p - 1][p - 1];  // 1 / (S_i^{-1})_pp
    for (int j = 0; j < t; ++j) {
        double z[PM];
#pragma unroll
        for (int r = 0; r < p; ++r) {
            double s = (r < q) ? c.bbar_T[r + (int64_t)j * q] : red(q + 1 + j, i);
#pragma unroll
            for (int k = 0; k < r; ++k) s -= C[r][k] * z[k];
            z[r] = s * rc[r];
        }
#pragma unroll
        for (int r = p - 1; r >= 0; --r) {
            double s = z[r];
#pragma unroll
            for (int k = r + 1; k < p; ++k) s -= C[k][r] * z[k];
            z[r] = s * rc[r];
        }
        double* bo = b + (i * t + j) * p;
#pragma unroll
        for (int r = 0; r < p; ++r) bo[r] = st ? nanv : z[r];
        if (wald) wald[i * t + j] = st ? nanv : z[p - 1] * z[p - 1] * cpp2;
    }
    status[i] = st;
    if (cov) {
        // S_i^{-1} = C^{-T} C^{-1} (the covariance of b_i; M carries sigma^2): G = C^{-1}
        // column by column, then the symmetric product, written in full (column-major)
        double G[PM][PM];
#pragma unroll
        for (int cc = 0; cc < p; ++cc) {
#pragma unroll
            for (int r = 0; r < p; ++r) G[r][cc] = 0.0;
            G[cc][cc] = rc[cc];
#pragma unroll
            for (int r = cc + 1; r < p; ++r) {
                double acc = 0.0;
#pragma unroll
                for (int k = cc; k < r; ++k) acc = fma(C[r][k], G[k][cc], acc);
                G[r][cc] = -acc * rc[r];
            }
        }
        double* co = cov + i * p * p;
#pragma unroll
        for (int a2 = 0; a2 < p; ++a2)
#pragma unroll
            for (int b2 = 0; b2 < p; ++b2) {
                double acc = 0.0;
#pragma unroll
                for (int k = 0; k < p; ++k) acc = fma(G[k][a2], G[k][b2], acc);
                co[a2 + b2 * p] = st ? nanv : acc;
            }
    }
}

// Adds the row-tile partials of every reduction value and writes the total over the first
// partial (r = 0), so that the solve reads one value. A block covers 32 consecutive SNPs of
// one value: warp w adds rows r = w, w + 8, ... in ascending order, then warp 0 adds the
// eight warp sums in warp order. The order depends only on the row-tile count, never on
// the block size or the SNP's position, so results stay reproducible bit for bit.
constexpr int RED_WARPS = 8;

__device__ __forceinline__ void reduce_set(const PartialSet& ps, int64_t i, bool valid,
                                           double (*sh)[32]) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    double s = 0.0;
    if (valid)
        for (int r = warp; r < ps.count; r += RED_WARPS) s += ps.base[(int64_t)r * ps.stride + i];
    sh[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && valid) {
        double tot = sh[0][lane];
#pragma unroll
        for (int w = 1; w < RED_WARPS; ++w) tot += sh[w][lane];
        ps.base[i] = tot;
    }
}

template <class Red>
__global__ void __launch_bounds__(RED_WARPS * 32)
k_reduce_partials(Red red, int64_t mb) {
    __shared__ double sh[RED_WARPS][32];
    const int64_t i = blockIdx.x * 32LL + threadIdx.x % 32;
    reduce_set(red.set((int)blockIdx.y), i, i < mb, sh);
}

__device__ __forceinline__ int find_job(const BatchJob* __restrict__ jobs, int n_jobs, int64_t g) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (jobs[mid].snp_base <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <bool MIXED>
__global__ void __launch_bounds__(RED_WARPS * 32)
k_reduce_partials_batch(const BatchJob* __restrict__ jobs, int n_jobs, int64_t n_snps) {
    __shared__ double sh[RED_WARPS][32];
    const int64_t g = blockIdx.x * 32LL + threadIdx.x % 32;
    const int v = (int)blockIdx.y;
    const BatchJob& j = jobs[find_job(jobs, n_jobs, g < n_snps ? g : n_snps - 1)];
    const int64_t i = g - j.snp_base;
    const bool valid = g < n_snps && i < j.mb && v < n_red(j.c);
    PartialSet ps{nullptr, 0, 0};
    if (MIXED) {
        RedMixed red{j.sq_part, j.lin, j.ldp, j.n_tiles_mx, j.c.q, j.lin_tiles, j.c.q + j.c.t};
        if (valid) ps = red.set(v);
    } else {
        RedFp64 red{j.part, j.ldp, j.n_rt64, n_red(j.c)};
        if (valid) ps = red.set(v);
    }
    reduce_set(ps, i, valid, sh);
}

template <int P, class Red>
__global__ void __launch_bounds__(128)
k_snp_solve(CohortDev c, Red red, const uint8_t* __restrict__ bad, int64_t mb,
            double* __restrict__ b, double* __restrict__ wald, uint8_t* __restrict__ status,
            double* __restrict__ cov) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= mb) return;
    solve_snp<P>(c, red, bad, i, b, wald, status, cov);
}

// One thread per SNP; p = 2, 3, 4 get their own unrolled kernels.
template <class Red>
cudaError_t launch_solve(const CohortDev& c, const Red& red, const uint8_t* bad, int64_t mb,
                         double* b, double* wald, uint8_t* status, double* cov, cudaStream_t s) {
    const unsigned grid = (unsigned)ceil_div(mb, 128);
    switch (c.q + 1) {
        case 2: k_snp_solve<2><<<grid, 128, 0, s>>>(c, red, bad, mb, b, wald, status, cov); break;
        case 3: k_snp_solve<3><<<grid, 128, 0, s>>>(c, red, bad, mb, b, wald, status, cov); break;
        case 4: k_snp_solve<4><<<grid, 128, 0, s>>>(c, red, bad, mb, b, wald, status, cov); break;
        default: k_snp_solve<0><<<grid, 128, 0, s>>>(c, red, bad, mb, b, wald, status, cov); break;
    }
    return cudaGetLastError();
}

// Batched cohorts: one thread per SNP of every cohort (partials already reduced).
template <int P, bool MIXED>
__global__ void __launch_bounds__(128)
k_snp_solve_batch(const BatchJob* __restrict__ jobs, int n_jobs, int64_t n_snps) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_snps) return;
    const BatchJob& j = jobs[find_job(jobs, n_jobs, g)];
    const int64_t i = g - j.snp_base;
    if (i >= j.mb) return;
    if (MIXED) {
        RedMixed red{j.sq_part, j.lin, j.ldp, 1, j.c.q, 1, j.c.q + j.c.t};
        solve_snp<P>(j.c, red, j.bad, i, j.b, j.wald, j.status);
    } else {
        RedFp64 red{j.part, j.ldp, 1, n_red(j.c)};
        solve_snp<P>(j.c, red, j.bad, i, j.b, j.wald, j.status);
    }
}

template <class Red>
cudaError_t reduce_partials(const Red& red, int nred, int64_t mb, cudaStream_t s) {
    k_reduce_partials<<<dim3((unsigned)ceil_div(mb, 32), (unsigned)nred), RED_WARPS * 32, 0, s>>>(
        red, mb);
    return cudaGetLastError();
}

cudaError_t launch_reduce_fp64(const CohortDev& c, double* part, int64_t ldp, int n_tiles,
                               int64_t mb, cudaStream_t s) {
    if (mb <= 0) return cudaSuccess;
    return reduce_partials(RedFp64{part, ldp, n_tiles, n_red(c)}, n_red(c), mb, s);
}

cudaError_t launch_snp_solve(const CohortDev& c, double* part, int64_t ldp, int n_tiles,
                             const uint8_t* bad, int64_t mb, double* b, double* wald,
                             uint8_t* status, cudaStream_t s, double* cov) {
    if (mb <= 0) return cudaSuccess;
    cudaError_t e = launch_reduce_fp64(c, part, ldp, n_tiles, mb, s);
    if (e != cudaSuccess) return e;
    return launch_solve(c, RedFp64{part, ldp, 1, n_red(c)}, bad, mb, b, wald, status, cov, s);
}

cudaError_t launch_snp_solve_batch(const BatchJob* jobs, int n_jobs, int64_t n_snps, int p,
                                   int max_nred, bool mixed, cudaStream_t s) {
    if (n_snps <= 0) return cudaSuccess;
    const dim3 gr((unsigned)ceil_div(n_snps, 32), (unsigned)max_nred);
    if (mixed) k_reduce_partials_batch<true><<<gr, RED_WARPS * 32, 0, s>>>(jobs, n_jobs, n_snps);
    else k_reduce_partials_batch<false><<<gr, RED_WARPS * 32, 0, s>>>(jobs, n_jobs, n_snps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)ceil_div(n_snps, 128);
    // every cohort of a batch has the same p
#define GWAS_BATCH_SOLVE(PP)                                                          \
    if (mixed) k_snp_solve_batch<PP, true><<<grid, 128, 0, s>>>(jobs, n_jobs, n_snps); \
    else k_snp_solve_batch<PP, false><<<grid, 128, 0, s>>>(jobs, n_jobs, n_snps);
    switch (p) {
        case 2: GWAS_BATCH_SOLVE(2) break;
        case 3: GWAS_BATCH_SOLVE(3) break;
        case 4: GWAS_BATCH_SOLVE(4) break;
        default: GWAS_BATCH_SOLVE(0) break;
    }
#undef GWAS_BATCH_SOLVE
    return cudaGetLastError();
}

cudaError_t launch_snp_solve_mixed(const CohortDev& c, const MixedDev& m, const uint8_t* bad,
                                   int64_t mb, double* b, double* wald, uint8_t* status,
                                   cudaStream_t s, double* cov, int64_t snp0) {
    const int64_t count = mb - snp0;
    if (count <= 0) return cudaSuccess;
    const int q = c.q, p = q + 1;
    // SNPs snp0 .. mb-1: their partials are columns snp0 .. of every partial row
    double* sq = m.sq_part + snp0;
    double* lin = m.lin + snp0;
    cudaError_t e = reduce_partials(RedMixed{sq, lin, m.ldp, m.n_rt, q, m.lin_tiles(), m.R_e},
                                    n_red(c), count, s);
    if (e != cudaSuccess) return e;
    return launch_solve(c, RedMixed{sq, lin, m.ldp, 1, q, 1, m.R_e}, bad + snp0, count,
                        b + snp0 * c.t * p, wald ? wald + snp0 * c.t : nullptr, status + snp0,
                        cov ? cov + snp0 * p * p : nullptr, s);
}

}  // namespace gwas
