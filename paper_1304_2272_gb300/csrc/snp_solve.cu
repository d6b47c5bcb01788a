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

__global__ void __launch_bounds__(128)
k_snp_solve(CohortDev c, const double* __restrict__ part, int64_t ldp, int n_tiles,
            const uint8_t* __restrict__ bad, int64_t mb, double* __restrict__ b,
            double* __restrict__ wald, uint8_t* __restrict__ status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= mb) return;
    const int q = c.q, t = c.t, p = q + 1, nred = q + 1 + t;

    // S_BLi (q values) and S_BRi, summed over row tiles in ascending order.
    double red[MAX_P];
    for (int v = 0; v < p; ++v) {
        double s = 0.0;
        for (int r = 0; r < n_tiles; ++r) s += part[((int64_t)r * nred + v) * ldp + i];
        red[v] = s;
    }
    // C C^T = S_i (C lower triangular, column by column).
    double C[MAX_P][MAX_P];
    double smax = red[q];
    for (int a = 0; a < q; ++a) smax = fmax(smax, c.S_TL[a + a * q]);
    bool ok = true;
    for (int j = 0; j < p; ++j) {
        double d = (j < q) ? c.S_TL[j + j * q] : red[q];
        for (int k = 0; k < j; ++k) d -= C[j][k] * C[j][k];
        if (!(d > SINGULAR_RTOL * smax)) { ok = false; d = 1.0; }
        C[j][j] = sqrt(d);
        for (int r = j + 1; r < p; ++r) {
            double s = (r < q) ? c.S_TL[r + j * q] : red[j];
            for (int k = 0; k < j; ++k) s -= C[r][k] * C[j][k];
            C[r][j] = s / C[j][j];
        }
    }
    uint8_t st = bad[i] ? 2 : (ok ? 0 : 1);
    const double nanv = nan("");
    const double cpp2 = C[p - 1][p - 1] * C[p - 1][p - 1];  // 1 / (S_i^{-1})_pp
    for (int j = 0; j < t; ++j) {
        double z[MAX_P];
        for (int r = 0; r < p; ++r) {
            double s;
            if (r < q) {
                s = c.bbar_T[r + (int64_t)j * q];
            } else {
                s = 0.0;
                for (int tt = 0; tt < n_tiles; ++tt)
                    s += part[((int64_t)tt * nred + (q + 1 + j)) * ldp + i];
            }
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

cudaError_t launch_snp_solve(const CohortDev& c, const double* part, int64_t ldp, int n_tiles,
                             const uint8_t* bad, int64_t mb, double* b, double* wald,
                             uint8_t* status, cudaStream_t s) {
    if (mb <= 0) return cudaSuccess;
    k_snp_solve<<<(unsigned)ceil_div(mb, 128), 128, 0, s>>>(c, part, ldp, n_tiles, bad, mb, b,
                                                          wald, status);
    return cudaGetLastError();
}

}  // namespace gwas
