// REML log-likelihood and its gradient for M(h, sigma^2) = sigma^2 (h Phi + (1-h) I),
// and the per-SNP derivative db_i/dh, on the GPU in FP64.
//
// Null model y = X_L beta + e, e ~ N(0, M) (the model behind the paper's M, Section 1):
//   l = -1/2 [ (n-q) log 2 pi + log|M| + log|X_L^T M^-1 X_L| + y^T P y ],
//   P = M^-1 - M^-1 X_L (X_L^T M^-1 X_L)^-1 X_L^T M^-1.
// Its adjoint with respect to M is  lbar_M = -1/2 (P - P y y^T P), so for any parameter
// dl/dtheta = <lbar_M, dM/dtheta>, which with dM/dh = sigma^2 (Phi - I) and
// dM/dsigma^2 = M / sigma^2 becomes
//   dl/dh      = -1/2 sigma^2 [ tr(P Phi) - tr P - (Py)^T Phi (Py) + |Py|^2 ],
//   dl/dsigma2 = -1/2 [ (n - q) - y^T P y ] / sigma^2.
// With Z = M^-1 [X_L | Y] = L^-T [Xbar_L | Ybar] and A = X_L^T M^-1 X_L = S_TL:
//   tr(P Phi) - tr P = <M^-1, Phi> - tr M^-1 - tr(A^-1 (Z_L^T Phi Z_L - Z_L^T Z_L)),
//   Py = z_y - Z_L A^-1 bbar_T,  y^T P y = |ybar|^2 - bbar_T^T A^-1 bbar_T,
// so the n x n work is one product M^-1 = L^-T L^-1, one Frobenius product with Phi, and
// the small Gram matrices Z^T Z and Z^T Phi Z.
//
// db_i/dh: differentiating the normal equations X_i^T M^-1 (y - X_i b_i) = 0 and using
// dM/dh = (M - sigma^2 I)/h (h > 0) gives db_i/dh = (sigma^2/h) S_i^-1 X_i^T M^-2 r_i,
// r_i = y - X_i b_i. Its per-SNP pieces X_L^T M^-2 x_i, |M^-1 x_i|^2 and Y^T M^-2 x_i are
// the reductions of the FP64 block kernel run with M^-1 in place of L^-1 and Z in place
// of [Xbar_L | Ybar]: the block of M^-1 x_i is recomputed from the dosages, not stored.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace gwas {

__global__ void __launch_bounds__(256) k_logdiag(const double* __restrict__ L, int64_t ldl,
                                                 int64_t n, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += log(L[i + i * ldl]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_logdiag(const double* L, int64_t ldl, int64_t n, double* out, cudaStream_t s) {
    k_logdiag<<<1, 256, 0, s>>>(L, ldl, n, out);
    return cudaGetLastError();
}

// Block b: columns [256 b, 256 b + 256), rows strided by the thread index.
__global__ void __launch_bounds__(256)
k_frob_part(const double* __restrict__ A, const double* __restrict__ B, int64_t ld, int64_t n,
            double* __restrict__ part) {
    __shared__ double r1[256], r2[256];
    const int64_t j0 = (int64_t)blockIdx.x * 256, j1 = min64(n, j0 + 256);
    double f = 0.0, tr = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const double* a = A + j * ld;
        const double* bcol = B + j * ld;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            f = fma(a[i], bcol[i], f);
            if (i == j) tr += a[i];
        }
    }
    r1[threadIdx.x] = f;
    r2[threadIdx.x] = tr;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            r1[threadIdx.x] += r1[threadIdx.x + w];
            r2[threadIdx.x] += r2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = r1[0];
        part[2 * blockIdx.x + 1] = r2[0];
    }
}

__global__ void k_frob_sum(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double f = 0.0, tr = 0.0;
    for (int b = 0; b < nb; ++b) {
        f += part[2 * b];
        tr += part[2 * b + 1];
    }
    out[0] = f;
    out[1] = tr;
}

cudaError_t launch_frob_trace(const double* A, const double* B, int64_t ld, int64_t n,
                              double* part, double* out, cudaStream_t s) {
    const int nb = (int)ceil_div(n, 256);
    k_frob_part<<<nb, 256, 0, s>>>(A, B, ld, n, part);
    k_frob_sum<<<1, 32, 0, s>>>(part, nb, out);
    return cudaGetLastError();
}

// q x q Cholesky of a column-major SPD matrix into C (row-major local array).
__device__ static bool small_chol(const double* A, int q, double (&C)[MAX_P][MAX_P]) {
    for (int j = 0; j < q; ++j) {
        double d = A[j + j * q];
        for (int k = 0; k < j; ++k) d -= C[j][k] * C[j][k];
        if (!(d > 0.0)) return false;
        C[j][j] = sqrt(d);
        for (int r = j + 1; r < q; ++r) {
            double s = A[r + j * q];
            for (int k = 0; k < j; ++k) s -= C[r][k] * C[j][k];
            C[r][j] = s / C[j][j];
        }
    }
    return true;
}

// x := A^-1 x through the factor C of A.
__device__ static void small_solve(const double (&C)[MAX_P][MAX_P], int q, double* x) {
    for (int r = 0; r < q; ++r) {
        double s = x[r];
        for (int k = 0; k < r; ++k) s -= C[r][k] * x[k];
        x[r] = s / C[r][r];
    }
    for (int r = q - 1; r >= 0; --r) {
        double s = x[r];
        for (int k = r + 1; k < q; ++k) s -= C[k][r] * x[k];
        x[r] = s / C[r][r];
    }
}

__global__ void k_reml_assemble(RemlDev r) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int q = r.q, t = r.t, nz = q + t, jy = q + r.j;
    double C[MAX_P][MAX_P];
    double* out = r.out;
    // Zc^T Phi Zc, entry (a, b)
    auto g2 = [&](int a, int b) {
        const double v = r.G2[a + b * nz];
        return r.identity ? (v / r.sigma2 - (1.0 - r.h) * r.G1[a + b * nz]) / r.h : v;
    };
    if (!small_chol(r.S_TL, q, C)) {
        for (int k = 0; k < 8; ++k) out[k] = nan("");
        return;
    }
    double logdet_A = 0.0;
    for (int a = 0; a < q; ++a) logdet_A += 2.0 * log(C[a][a]);
    double beta[MAX_P];
    for (int a = 0; a < q; ++a) beta[a] = r.bbar_T[a + r.j * q];
    small_solve(C, q, beta);
    double yPy = *r.yy;
    for (int a = 0; a < q; ++a) yPy -= r.bbar_T[a + r.j * q] * beta[a];
    // tr(A^-1 D), D = Z_L^T Phi Z_L - Z_L^T Z_L: column by column of A^-1
    double trAD = 0.0;
    for (int b = 0; b < q; ++b) {
        double col[MAX_P];
        for (int a = 0; a < q; ++a) col[a] = (a == b) ? 1.0 : 0.0;
        small_solve(C, q, col);  // column b of A^-1
        for (int a = 0; a < q; ++a)
            trAD += col[a] * (g2(b, a) - r.G1[b + a * nz]);
    }
    // Py = Zc v with v = [-beta; e_j]: quadratic forms in G1 and G2
    double pp = 0.0, pPhip = 0.0;
    for (int a = 0; a < nz; ++a) {
        const double va = a < q ? -beta[a] : (a == jy ? 1.0 : 0.0);
        if (va == 0.0) continue;
        for (int b = 0; b < nz; ++b) {
            const double vb = b < q ? -beta[b] : (b == jy ? 1.0 : 0.0);
            if (vb == 0.0) continue;
            pp += va * vb * r.G1[a + b * nz];
            pPhip += va * vb * g2(a, b);
        }
    }
    const double n = (double)r.n;
    double s2 = r.sigma2;
    double logdet_M = 2.0 * (*r.logdet_M);
    const double tr_minv = r.identity ? r.frob[0] : r.frob[1];
    const double minv_phi = r.identity ? (n / s2 - (1.0 - r.h) * tr_minv) / r.h : r.frob[0];
    double tr_dMh = s2 * ((minv_phi - tr_minv) - trAD);       // tr(P dM/dh)
    double q_dMh = s2 * (pPhip - pp);                        // (Py)^T dM/dh (Py)
    const double s2_hat = s2 * yPy / (n - q);
    if (r.profile) {
        // M = rho M_in with rho = s2_hat / s2: P -> P/rho, Py -> Py/rho, dM/dh -> rho dM/dh
        const double rho = s2_hat / s2;
        logdet_M += n * log(rho);
        logdet_A -= q * log(rho);
        yPy /= rho;
        q_dMh /= rho;
        s2 = s2_hat;
    }
    const double LOG2PI = 1.8378770664093454836;
    out[0] = -0.5 * ((n - q) * LOG2PI + logdet_M + logdet_A + yPy);
    out[1] = -0.5 * (tr_dMh - q_dMh);
    out[2] = -0.5 * ((n - q) - yPy) / s2;
    out[3] = s2_hat;
    out[4] = yPy;
    out[5] = logdet_M;
    out[6] = logdet_A;
    out[7] = s2;
}

cudaError_t launch_reml_assemble(const RemlDev& r, cudaStream_t s) {
    if (r.q < 1 || r.q + r.t > MAX_P + MAX_T) return cudaErrorInvalidValue;
    k_reml_assemble<<<1, 32, 0, s>>>(r);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// db_i/dh, one thread per SNP (partials already reduced: n_tiles = 1).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_dbdh(CohortDev c, const double* __restrict__ pf, const double* __restrict__ pa, int64_t ldp,
       int n_tiles, const double* __restrict__ G1, double scale, const uint8_t* __restrict__ bad,
       int64_t mb, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= mb) return;
    const int q = c.q, t = c.t, p = q + 1, nred = q + 1 + t, nz = q + t;
    auto sum = [&](const double* part, int v) {
        double s = 0.0;
        for (int r = 0; r < n_tiles; ++r) s += part[((int64_t)r * nred + v) * ldp + i];
        return s;
    };
    double sbl[MAX_P], gl[MAX_P];
    for (int v = 0; v < p; ++v) {
        sbl[v] = sum(pf, v);  // S_BLi then S_BRi
        gl[v] = sum(pa, v);   // X_L^T M^-2 x_i then |M^-1 x_i|^2
    }
    double C[MAX_P][MAX_P];
    double smax = sbl[q];
    for (int a = 0; a < q; ++a) smax = fmax(smax, c.S_TL[a + a * q]);
    bool ok = true;
    for (int j = 0; j < p; ++j) {
        double d = (j < q) ? c.S_TL[j + j * q] : sbl[q];
        for (int k = 0; k < j; ++k) d -= C[j][k] * C[j][k];
        if (!(d > 1e-12 * smax)) { ok = false; d = 1.0; }
        C[j][j] = sqrt(d);
        for (int r = j + 1; r < p; ++r) {
            double s = (r < q) ? c.S_TL[r + j * q] : sbl[j];
            for (int k = 0; k < j; ++k) s -= C[r][k] * C[j][k];
            C[r][j] = s / C[j][j];
        }
    }
    const bool valid = ok && !bad[i];
    for (int j = 0; j < t; ++j) {
        double bvec[MAX_P];
        for (int a = 0; a < q; ++a) bvec[a] = c.bbar_T[a + (int64_t)j * q];
        bvec[q] = sum(pf, q + 1 + j);
        small_solve(C, p, bvec);  // b_i for phenotype j
        const double bp = bvec[q];
        // u = X_i^T M^-2 r_i
        double u[MAX_P];
        for (int a = 0; a < q; ++a) {
            double s = G1[a + (q + j) * nz];
            for (int k = 0; k < q; ++k) s -= G1[a + k * nz] * bvec[k];
            u[a] = s - gl[a] * bp;
        }
        double s = sum(pa, q + 1 + j);
        for (int k = 0; k < q; ++k) s -= gl[k] * bvec[k];
        u[q] = s - gl[q] * bp;
        small_solve(C, p, u);
        double* o = out + (i * t + j) * p;
        for (int a = 0; a < p; ++a) o[a] = valid ? scale * u[a] : nan("");
    }
}

cudaError_t launch_dbdh(const CohortDev& c, const double* part_fwd, double* part_adj,
                        int64_t ldp, int n_tiles, const double* G1, double scale,
                        const uint8_t* bad, int64_t mb, double* dbdh, cudaStream_t s) {
    if (mb <= 0) return cudaSuccess;
    cudaError_t e = launch_reduce_fp64(c, part_adj, ldp, n_tiles, mb, s);
    if (e != cudaSuccess) return e;
    k_dbdh<<<(unsigned)ceil_div(mb, 128), 128, 0, s>>>(c, part_fwd, part_adj, ldp, 1, G1,
                                                       scale, bad, mb, dbdh);
    return cudaGetLastError();
}

}  // namespace gwas
