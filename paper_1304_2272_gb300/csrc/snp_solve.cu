// Per-SNP tail of Algorithm 1's loop (Section 2.1): add the row-tile partial sums,
// set S_i = [[S_TL, *], [S_BLi, S_BRi]] and bbar_i = [bbar_T; bbar_Bi], and solve
// S_i b_i = bbar_i through a p x p Cholesky factorisation (Section 2, sixth step).
// One thread per SNP, everything in FP64.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace gwas {

// Singular S_i: a Cholesky pivot at or below this fraction of max_j S_jj.
constexpr double SINGULAR_RTOL = 1e-12;

// Reduction value v of SNP i (v < q: S_BLi[v]; v == q: S_BRi; v > q: bbar_Bi[v-q-1]).
// FP64 path: every value is a sum of per-row-tile partials, added in ascending order.
struct RedFp64 {
    const double* part;
    int64_t ldp;
    int n_tiles;
    int nred;
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

template <class Red>
__device__ __forceinline__ void solve_snp(const CohortDev& c, const Red& red,
                                          const uint8_t* __restrict__ bad, int64_t i,
                                          double* __restrict__ b, double* __restrict__ wald,
                                          uint8_t* __restrict__ status) {
    const int q = c.q, t = c.t, p = q + 1;

    double sbl[MAX_P];  // S_BLi (q values) then S_BRi
    for (int v = 0; v < p; ++v) sbl[v] = red(v, i);
    // C C^T = S_i (C lower triangular, column by column).
    double C[MAX_P][MAX_P];
    double smax = sbl[q];
    for (int a = 0; a < q; ++a) smax = fmax(smax, c.S_TL[a + a * q]);
    bool ok = true;
    for (int j = 0; j < p; ++j) {
        double d = (j < q) ? c.S_TL[j + j * q] : sbl[q];
        for (int k = 0; k < j; ++k) d -= C[j][k] * C[j][k];
        if (!(d > SINGULAR_RTOL * smax)) { ok = false; d = 1.0; }
        C[j][j] = sqrt(d);
        for (int r = j + 1; r < p; ++r) {
            double s = (r < q) ? c.S_TL[r + j * q] : sbl[j];
            for (int k = 0; k < j; ++k) s -= C[r][k] * C[j][k];
            C[r][j] = s / C[j][j];
        }
    }
    const uint8_t st = bad[i] ? 2 : (ok ? 0 : 1);
    const double nanv = nan("");
    const double cpp2 = C[p - 1][p - 1] * C[p - 1][p - 1];  // 1 / (S_i^{-1})_pp
    for (int j = 0; j < t; ++j) {
        double z[MAX_P];
        for (int r = 0; r < p; ++r) {
            double s = (r < q) ? c.bbar_T[r + (int64_t)j * q] : red(q + 1 + j, i);
            for (int k = 0; k < r; ++k) s -= C[r][k] * z[k];
            z[r] = s / C[r][r];
        }
        for (int r = p - 1; r >= 0; --r) {
            double s = z[r];
            for (int k = r + 1; k < p; ++k) s -= C[k][r] * z[k];
            z[r] = s / C[r][r];
        }
        double* bo = b + (i * t + j) * p;
        for (int r = 0; r < p; ++r) bo[r] = st ? nanv : z[r];
        if (wald) wald[i * t + j] = st ? nanv : z[p - 1] * z[p - 1] * cpp2;
    }
    status[i] = st;
}

template <class Red>
__global__ void __launch_bounds__(128)
k_snp_solve(CohortDev c, Red red, const uint8_t* __restrict__ bad, int64_t mb,
            double* __restrict__ b, double* __restrict__ wald, uint8_t* __restrict__ status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= mb) return;
    solve_snp(c, red, bad, i, b, wald, status);
}

// Batched cohorts: one thread per SNP of every cohort.
template <bool MIXED>
__global__ void __launch_bounds__(128)
k_snp_solve_batch(const BatchJob* __restrict__ jobs, int n_jobs, int64_t n_snps) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_snps) return;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (jobs[mid].snp_base <= g) lo = mid;
        else hi = mid - 1;
    }
    const BatchJob& j = jobs[lo];
    const int64_t i = g - j.snp_base;
    if (i >= j.mb) return;
    if (MIXED) {
        RedMixed red{j.sq_part, j.lin, j.ldp, j.n_tiles_mx, j.c.q, j.lin_tiles, j.c.q + j.c.t};
        solve_snp(j.c, red, j.bad, i, j.b, j.wald, j.status);
    } else {
        RedFp64 red{j.part, j.ldp, j.n_rt64, n_red(j.c)};
        solve_snp(j.c, red, j.bad, i, j.b, j.wald, j.status);
    }
}

cudaError_t launch_snp_solve(const CohortDev& c, const double* part, int64_t ldp, int n_tiles,
                             const uint8_t* bad, int64_t mb, double* b, double* wald,
                             uint8_t* status, cudaStream_t s) {
    if (mb <= 0) return cudaSuccess;
    RedFp64 red{part, ldp, n_tiles, n_red(c)};
    k_snp_solve<<<(unsigned)ceil_div(mb, 128), 128, 0, s>>>(c, red, bad, mb, b, wald, status);
    return cudaGetLastError();
}

cudaError_t launch_snp_solve_batch(const BatchJob* jobs, int n_jobs, int64_t n_snps, bool mixed,
                                   cudaStream_t s) {
    if (n_snps <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)ceil_div(n_snps, 128);
    if (mixed) k_snp_solve_batch<true><<<grid, 128, 0, s>>>(jobs, n_jobs, n_snps);
    else k_snp_solve_batch<false><<<grid, 128, 0, s>>>(jobs, n_jobs, n_snps);
    return cudaGetLastError();
}

cudaError_t launch_snp_solve_mixed(const CohortDev& c, const MixedDev& m, const uint8_t* bad,
                                   int64_t mb, double* b, double* wald, uint8_t* status,
                                   cudaStream_t s) {
    if (mb <= 0) return cudaSuccess;
    RedMixed red{m.sq_part, m.lin, m.ldp, m.n_rt, c.q, m.lin_tiles(), m.R_e};
    k_snp_solve<<<(unsigned)ceil_div(mb, 128), 128, 0, s>>>(c, red, bad, mb, b, wald, status);
    return cudaGetLastError();
}

}  // namespace gwas
