// C ABI of the REML log-likelihood, its adjoint gradient and db_i/dh (include/gwas.h):
// gwas_reml and gwas_solve_block_grad_device on a context of gwas_api.cu.
#include "api_internal.h"

using namespace gwas_api;

// ============================================================================
// REML log-likelihood, its gradient, and db_i/dh.
// ============================================================================
namespace {

// M^-1 = W^T W (W = L^-1 lower triangular) into c->Minv.
cudaError_t form_minv(gwas_ctx* c, cudaStream_t s) {
    const int64_t n = c->n, ld = c->ld;
    cudaError_t e;
    if (!c->Minv && (e = dmalloc(&c->Minv, (size_t)ld * ld)) != cudaSuccess) return e;
    GemmF64 mi;
    mi.M = n; mi.N = n; mi.K = n; mi.A = c->W; mi.lda = ld; mi.transA = true; mi.a_upper = true;
    mi.B = c->W; mi.ldb = ld; mi.b_lower = true; mi.C = c->Minv; mi.ldc = ld;
    if ((e = gemm_f64(mi, s)) != cudaSuccess) return e;
    c->minv_ready = true;
    return cudaSuccess;
}

// Layout of c->small: G1 and G2 ((q+t)^2 each), PhiZ (n x (q+t)), then scalars.
struct SmallLayout {
    int64_t nz, g1, g2, phiz, yy, logdet, frob, fpart, out, total;
    explicit SmallLayout(const gwas_ctx* c) {
        nz = c->q + c->t;
        g1 = 0;
        g2 = g1 + nz * nz;
        phiz = g2 + nz * nz;
        yy = phiz + c->n * nz;
        logdet = yy + 1;
        frob = logdet + 1;
        fpart = frob + 2;
        out = fpart + 2 * ceil_div(c->n, 256);
        total = out + 8;
    }
};

}  // namespace

extern "C" gwas_status gwas_reml(gwas_ctx* c, const double* Phi, double h, double sigma2,
                                 const double* XL, const double* Y, int pheno, int profile,
                                 gwas_reml_result* out) {
    Range range_("gwas_reml");
    if (!c || !out) return GWAS_ERR_ARG;
    if (!Phi || !XL || !Y) return fail(c, GWAS_ERR_ARG, "gwas_reml: NULL input");
    if (pheno < 0 || pheno >= c->t) return fail(c, GWAS_ERR_ARG, "gwas_reml: phenotype out of range");
    gwas_status st = gwas_factor(c, Phi, 1, h, sigma2, XL, Y);
    if (st != GWAS_OK) return st;
    DeviceGuard g(c->device);
    const int64_t n = c->n, ld = c->ld, nz = c->q + c->t;
    cudaStream_t s = c->s_comp;
    const SmallLayout sl(c);
    // For h >= 1e-2 Phi enters only through M: Phi Z and <M^-1, Phi> follow from M, Z and
    // tr M^-1 = |L^-1|_F^2, so neither Phi nor M^-1 (n^3/3 flops) is formed; below it the
    // identities would divide a cancellation by h, and Phi and M^-1 are used directly.
    const bool identity = h >= 1e-2;
    if (!c->Z) CK(dmalloc(&c->Z, (size_t)n * nz));
    if (!c->small) CK(dmalloc(&c->small, (size_t)sl.total));
    double* sm = c->small;
    if (!identity) {
        if (!c->Phi) CK(dmalloc(&c->Phi, (size_t)ld * ld));
        if (!c->Minv) CK(dmalloc(&c->Minv, (size_t)ld * ld));
        // the full Phi (the Frobenius product reads both triangles)
        CK(cudaMemcpy2DAsync(c->Phi, ld * sizeof(double), Phi, n * sizeof(double),
                             n * sizeof(double), n, cudaMemcpyDefault, s));
        // M^-1 = W^T W (W = L^-1 lower triangular)
        CK(form_minv(c, s));
    }
    if (!c->mixed) {  // the mixed factor already formed Z
        GemmF64 z;
        z.M = n; z.N = c->q; z.K = n; z.A = c->W; z.lda = ld; z.transA = true; z.a_upper = true;
        z.B = c->XLbar; z.ldb = n; z.C = c->Z; z.ldc = n;
        CK(gemm_f64(z, s));
        GemmF64 zy = z;
        zy.N = c->t; zy.B = c->Ybar; zy.C = c->Z + (size_t)n * c->q;
        CK(gemm_f64(zy, s));
    }
    // G1 = Z^T Z; G2 = Z^T Phi Z (identity: Z^T [X_L | Y]); |ybar_j|^2
    GemmF64 g1;
    g1.M = nz; g1.N = nz; g1.K = n; g1.A = c->Z; g1.lda = n; g1.transA = true; g1.B = c->Z;
    g1.ldb = n; g1.C = sm + sl.g1; g1.ldc = nz;
    CK(gemm_f64(g1, s));
    GemmF64 g2 = g1;
    g2.C = sm + sl.g2;
    if (identity) {
        g2.B = c->XLY;
    } else {
        GemmF64 pz;
        pz.M = n; pz.N = nz; pz.K = n; pz.A = c->Phi; pz.lda = ld; pz.B = c->Z; pz.ldb = n;
        pz.C = sm + sl.phiz; pz.ldc = n;
        CK(gemm_f64(pz, s));
        g2.B = sm + sl.phiz;
    }
    CK(gemm_f64(g2, s));
    GemmF64 yy;
    yy.M = 1; yy.N = 1; yy.K = n; yy.A = c->Ybar + (size_t)n * pheno; yy.lda = n; yy.transA = true;
    yy.B = c->Ybar + (size_t)n * pheno; yy.ldb = n; yy.C = sm + sl.yy; yy.ldc = 1;
    CK(gemm_f64(yy, s));
    CK(launch_logdiag(c->L, ld, n, sm + sl.logdet, s));
    if (identity)
        CK(launch_frob_trace(c->W, c->W, ld, n, sm + sl.fpart, sm + sl.frob, s));
    else
        CK(launch_frob_trace(c->Minv, c->Phi, ld, n, sm + sl.fpart, sm + sl.frob, s));
    RemlDev r;
    r.n = n; r.q = c->q; r.t = c->t; r.j = pheno; r.h = h; r.sigma2 = sigma2;
    r.profile = profile ? 1 : 0;
    r.S_TL = c->S_TL; r.bbar_T = c->bbar_T; r.G1 = sm + sl.g1; r.G2 = sm + sl.g2;
    r.yy = sm + sl.yy; r.logdet_M = sm + sl.logdet; r.frob = sm + sl.frob; r.out = sm + sl.out;
    r.identity = identity ? 1 : 0;
    CK(launch_reml_assemble(r, s));
    double host[8];
    CK(cudaMemcpyAsync(host, sm + sl.out, sizeof host, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out->loglik = host[0];
    out->dl_dh = host[1];
    out->dl_dsigma2 = host[2];
    out->sigma2_hat = host[3];
    out->yPy = host[4];
    out->logdet_M = host[5];
    out->logdet_A = host[6];
    out->sigma2 = host[7];
    c->grad_ready = true;
    c->grad_h = h;
    c->grad_s2 = sigma2;
    if (!std::isfinite(host[0])) return fail(c, GWAS_ERR_NOT_SPD, "gwas_reml: X_L^T M^-1 X_L is not SPD");
    return GWAS_OK;
}

extern "C" gwas_status gwas_solve_block_grad_device(gwas_ctx* c, const int8_t* X, int64_t mb,
                                                    double* b, double* wald, uint8_t* status,
                                                    double* dbdh) {
    gwas_status st = check_block_args(c, X, mb, b, status);
    if (st != GWAS_OK) return st;
    if (!dbdh) return fail(c, GWAS_ERR_ARG, "gwas_solve_block_grad_device: NULL dbdh");
    if (c->mixed) return fail(c, GWAS_ERR_UNSUPPORTED, "db/dh is built for GWAS_PREC_FP64 contexts");
    if (!c->grad_ready) return fail(c, GWAS_ERR_STATE, "db/dh needs a gwas_reml at the current h");
    if (!(c->grad_h > 0.0)) return fail(c, GWAS_ERR_ARG, "db/dh needs h > 0");
    DeviceGuard g(c->device);
    const int64_t n = c->n;
    const int n_tiles = (int)ceil_div(n, T64);
    if (!c->part2) CK(dmalloc(&c->part2, (size_t)n_tiles * (c->q + 1 + c->t) * c->ldp));
    if (!c->minv_ready) {  // gwas_reml did not need M^-1 (h >= 1e-2): form it once
        CK(form_minv(c, c->s_comp));
        c->stats.kernel_launches += 1;
    }
    // forward: b_i, Wald, status, and the partials of S_i and bbar_i
    if ((st = run_block(c, X, mb, b, wald, status)) != GWAS_OK) return st;
    // adjoint: the same kernel with M^-1 (dense) and Z = M^-1 [X_L | Y]
    CohortDev adj = cohort_view(c);
    adj.W = c->Minv;
    adj.ldw = c->ld;
    adj.dense = true;
    adj.XLbar = c->Z;
    adj.Ybar = c->Z + (size_t)n * c->q;
    CK(launch_block_fp64(adj, X, n, mb, c->part2, c->ldp, c->bad, c->s_comp));
    const SmallLayout sl(c);
    CK(launch_dbdh(cohort_view(c), c->part, c->part2, c->ldp, n_tiles, c->small + sl.g1,
                   c->grad_s2 / c->grad_h, c->bad, mb, dbdh, c->s_comp));
    c->stats.kernel_launches += 3;
    return GWAS_OK;
}
