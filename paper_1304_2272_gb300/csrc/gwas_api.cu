// C ABI of the engine (include/gwas.h): context, device memory, streams and the
// double-buffered block pipeline of Algorithm 2 (Section 3).
//
// Streams: one H2D copy stream, one compute stream, one D2H copy stream. Two device
// slots alternate between blocks; CUDA events order "copy block k+1 in" against
// "compute block k" and "copy b of block k-1 out", which is the paper's
// load_start/load_wait/store_start/store_wait pattern with the disk replaced by
// pinned host memory and the second memory region by the second device slot.
#include "api_internal.h"

namespace gwas_api {
gwas_status fail(gwas_ctx* c, gwas_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

gwas_status cuda_fail(gwas_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();  // clear a sticky launch error where possible
    return fail(c, e == cudaErrorMemoryAllocation ? GWAS_ERR_OOM : GWAS_ERR_CUDA, m);
}

CohortDev cohort_view(const gwas_ctx* c) {
    CohortDev v;
    v.n = c->n; v.q = c->q; v.t = c->t;
    v.W = c->W; v.ldw = c->ld;
    v.XLbar = c->XLbar; v.Ybar = c->Ybar; v.S_TL = c->S_TL; v.bbar_T = c->bbar_T;
    v.ones_singular = c->ones_singular;
    return v;
}

cudaEvent_t pooled_event(gwas_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Adds the event times of completed timed launches to stats.trsm_ms and recycles their
// events; with wait = false it stops at the first launch still in flight, so a long
// timed run keeps a bounded number of pending events.
void fold_timings(gwas_ctx* c, bool wait) {
    size_t k = 0;
    for (; k < c->timed.size(); ++k) {
        auto& pr = c->timed[k];
        if (!wait && cudaEventQuery(pr.second) != cudaSuccess) break;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) c->stats.trsm_ms += ms;
        c->ev_pool.push_back(pr.first);
        c->ev_pool.push_back(pr.second);
    }
    c->timed.erase(c->timed.begin(), c->timed.begin() + (std::ptrdiff_t)k);
}

// The block compute on the compute stream: trsm + fused reductions, then the
// per-SNP solve. X, b, wald, status are device pointers.
gwas_status run_block(gwas_ctx* c, const int8_t* X, int64_t mb, double* b, double* wald,
                      uint8_t* status, double* cov) {
    Range range_("gwas block");
    CohortDev cv = cohort_view(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->opts.timing) {
        if (c->timed.size() >= 64) fold_timings(c, false);
        e0 = pooled_event(c);
        e1 = pooled_event(c);
        CK(cudaEventRecord(e0, c->s_comp));
    }
    // mixed blocks of 1024 SNPs or more go in two halves [0, h) and [h, mb) (h a multiple
    // of 256): s_comp runs conversion(0) -> block(0) -> block(1) -> solves(1), s_aux runs
    // conversion(1) beside block(0) and solves(0) beside block(1); s_comp waits for s_aux
    // before the call returns, so the block stays ordered on the context's stream
    const int64_t h = (c->mixed && c->s_aux && mb >= 1024) ? round_up(ceil_div(mb, 2), 256) : mb;
    const bool split = h < mb;
    if (c->mixed) {
        // the dosage conversion runs before the timed region of the dominant kernel
        if (c->opts.timing) CK(cudaEventRecord(e1, c->s_comp));
        CK(launch_geno_bf16(c->mx, X, c->n, h, c->bad, c->s_comp));
        if (split) {
            CK(cudaEventRecord(c->ev_conv0, c->s_comp));
            CK(cudaStreamWaitEvent(c->s_aux, c->ev_conv0, 0));
            CK(launch_geno_bf16(c->mx, X, c->n, mb, c->bad, c->s_aux, h));
            CK(cudaEventRecord(c->ev_conv1, c->s_aux));
        }
        if (c->opts.timing) CK(cudaEventRecord(e0, c->s_comp));
        CK(launch_block_mixed(c->mx, h, c->num_sms, c->s_comp));
        if (split) {
            CK(cudaEventRecord(c->ev_blk0, c->s_comp));
            CK(cudaStreamWaitEvent(c->s_comp, c->ev_conv1, 0));
            CK(launch_block_mixed(c->mx, mb, c->num_sms, c->s_comp, h));
        }
    } else {
        CK(launch_block_fp64(cv, X, c->n, mb, c->part, c->ldp, c->bad, c->s_comp));
    }
    if (c->opts.timing) {
        CK(cudaEventRecord(e1, c->s_comp));
        c->timed.emplace_back(e0, e1);
    }
    if (c->mixed) {
        if (split) {
            CK(cudaStreamWaitEvent(c->s_aux, c->ev_blk0, 0));
            CK(launch_snp_solve_mixed(cv, c->mx, c->bad, h, b, wald, status, c->s_aux, cov));
            CK(cudaEventRecord(c->ev_solve0, c->s_aux));
            CK(launch_snp_solve_mixed(cv, c->mx, c->bad, mb, b, wald, status, c->s_comp, cov, h));
            CK(cudaStreamWaitEvent(c->s_comp, c->ev_solve0, 0));
            c->stats.kernel_launches += 6;  // a second conversion, block kernel and solve
        } else {
            CK(launch_snp_solve_mixed(cv, c->mx, c->bad, mb, b, wald, status, c->s_comp, cov));
            c->stats.kernel_launches += 2;
        }
    } else {
        CK(launch_snp_solve(cv, c->part, c->ldp, (int)ceil_div(c->n, T64), c->bad, mb, b, wald,
                            status, c->s_comp, cov));
        c->stats.kernel_launches += 1;
    }
    c->stats.kernel_launches += 2;
    c->stats.trsm_launches += 1;
    c->stats.blocks += 1;
    c->stats.snps += mb;
    return GWAS_OK;
}

void apply_tile_cfg(MixedDev& m, int tile_cfg) {
    m.cfg_stages = 0;
    m.cfg_group_mb = 40;
    m.cfg_single_cta = false;
    m.cfg_pair = false;
    m.cfg_fuse = false;
    m.cfg_ztail = false;
    m.cfg_radix = 0;
    if (tile_cfg >= 0) {
        m.cfg_stages = tile_cfg & 0xF;
        const int g = (tile_cfg >> 4) & 0xFF;
        if (g > 0) m.cfg_group_mb = g;
        m.cfg_single_cta = ((tile_cfg >> 12) & 1) != 0;
        m.cfg_pair = ((tile_cfg >> 13) & 1) != 0;
        // bit 17 fuses the linear rows into the limb tiles; bit 14 (a separate linear
        // tile, the default) takes precedence
        m.cfg_fuse = ((tile_cfg >> 17) & 1) != 0 && ((tile_cfg >> 14) & 1) == 0;
        // bit 21: the linear rows at the end of the last row tile (unless fused)
        m.cfg_ztail = ((tile_cfg >> 21) & 1) != 0 && !m.cfg_fuse;
        m.cfg_radix = (tile_cfg >> 15) & 3;
    }
}

// (Re)allocate the mixed path's buffers whose size depends on the tile height R.
cudaError_t mixed_alloc_layout(MixedDev& m) {
    cudaFree(m.WL); cudaFree(m.bits); cudaFree(m.E); cudaFree(m.sq_part); cudaFree(m.lin);
    m.WL = nullptr; m.bits = nullptr; m.E = nullptr; m.sq_part = nullptr; m.lin = nullptr;
    cudaError_t e;
    if ((e = dmalloc(&m.WL, (size_t)m.rows_total * m.n_pad)) != cudaSuccess) return e;
    if ((e = dmalloc(&m.bits, (size_t)m.n_exp())) != cudaSuccess) return e;
    if ((e = dmalloc(&m.E, (size_t)m.n_exp())) != cudaSuccess) return e;
    if ((e = dmalloc(&m.sq_part, (size_t)m.n_rt * m.ldp)) != cudaSuccess) return e;
    return dmalloc(&m.lin, (size_t)m.lin_tiles() * m.R_e * m.ldp);
}

void free_all(gwas_ctx* c) {
    cudaFree(c->L); cudaFree(c->W); cudaFree(c->Dinv); cudaFree(c->XLbar); cudaFree(c->Ybar);
    cudaFree(c->S_TL); cudaFree(c->bbar_T); cudaFree(c->d_info); cudaFree(c->part);
    cudaFree(c->bad); cudaFree(c->Xunpack);
    cudaFree(c->Phi); cudaFree(c->Minv); cudaFree(c->part2); cudaFree(c->small);
    cudaFree(c->XLY);
    cudaFree(c->Z); cudaFree(c->mx.WL); cudaFree(c->mx.bits); cudaFree(c->mx.E);
    cudaFree(c->mx.Xb); cudaFree(c->mx.sq_part); cudaFree(c->mx.lin); cudaFree(c->mx.err);
    for (int s = 0; s < 2; ++s) {
        cudaFree(c->Xslot[s]); cudaFree(c->bslot[s]); cudaFree(c->wslot[s]); cudaFree(c->sslot[s]);
        cudaFree(c->Pslot[s]);
        if (c->ev_h2d[s]) cudaEventDestroy(c->ev_h2d[s]);
        if (c->ev_comp[s]) cudaEventDestroy(c->ev_comp[s]);
        if (c->ev_d2h[s]) cudaEventDestroy(c->ev_d2h[s]);
    }
    for (auto& pr : c->timed) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (auto e : c->done_ev) cudaEventDestroy(e);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t ev : {c->ev_conv0, c->ev_conv1, c->ev_blk0, c->ev_solve0})
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->chol.ev)
        if (ev) cudaEventDestroy(ev);
    if (c->chol.panel) cudaStreamDestroy(c->chol.panel);
    if (c->s_aux) cudaStreamDestroy(c->s_aux);
    if (c->s_comp) cudaStreamDestroy(c->s_comp);
    if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
    if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
}

gwas_status check_block_args(gwas_ctx* c, const int8_t* X, int64_t mb, double* b,
                                    uint8_t* status) {
    if (!c) return GWAS_ERR_ARG;
    if (!c->factored) return fail(c, GWAS_ERR_STATE, "solve before a successful gwas_factor");
    if (!X || !b || !status) return fail(c, GWAS_ERR_ARG, "solve: NULL pointer");
    if (mb < 1 || mb > c->opts.m_blk) return fail(c, GWAS_ERR_ARG, "solve: need 1 <= mb <= m_blk");
    return GWAS_OK;
}

}  // namespace gwas_api

using namespace gwas_api;
extern "C" {

void gwas_default_opts(gwas_opts* o) {
    if (!o) return;
    o->precision = GWAS_PREC_FP64;
    o->m_blk = 16384;
    o->n_limbs = 3;
    o->tile_cfg = -1;
    o->device = 0;
    o->timing = 0;
    o->use_graph = 1;
}

gwas_status gwas_init(int64_t n, int p, int t, const gwas_opts* opts, gwas_ctx** out) {
    if (!out) return GWAS_ERR_ARG;
    *out = nullptr;
    gwas_opts o;
    gwas_default_opts(&o);
    if (opts) o = *opts;
    if (n < 1 || p < 2 || p > MAX_P || t < 1 || t > MAX_T || o.m_blk < 1) return GWAS_ERR_ARG;
    if (o.precision != GWAS_PREC_FP64 && o.precision != GWAS_PREC_MIXED) return GWAS_ERR_ARG;
    if (n > (int64_t)1 << 31) return GWAS_ERR_ARG;
    if (o.precision == GWAS_PREC_MIXED) {
        // exact FP32 accumulation of integer limb products needs n 2^B < 2^24 with B >= 7
        // bits per limb (n < 2^17); the linear tile must fit one UMMA (N <= 256); with 5
        // limbs of 9 bits the recombined value stays below 2^61 and a tile's sum of
        // R <= 51 squares below 2^126 (int64, unsigned int128)
        if (o.n_limbs < 2 || o.n_limbs > 5 || mixed_radix(n) == 0 ||
            o.n_limbs * ((p - 1) + t) > 256)
            return GWAS_ERR_UNSUPPORTED;
    }
    gwas_ctx* c = new gwas_ctx();
    c->opts = o;
    c->device = o.device;
    c->n = n; c->p = p; c->q = p - 1; c->t = t;
    c->ld = round_up(n, T64);
    DeviceGuard g(c->device);
    auto bail = [&](cudaError_t e, const char* w) {
        cuda_fail(c, e, w);
        gwas_status st = e == cudaErrorMemoryAllocation ? GWAS_ERR_OOM : GWAS_ERR_CUDA;
        free_all(c);
        delete c;
        return st;
    };
#define CKI(call)                                  \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return bail(e_, #call); \
    } while (0)
    const int64_t nt = ceil_div(n, T64);
    const size_t nn = (size_t)c->ld * (size_t)c->ld;
    CKI(cudaSetDevice(c->device));
    CKI(dmalloc(&c->L, nn));
    CKI(dmalloc(&c->W, nn));
    CKI(dmalloc(&c->Dinv, (size_t)nt * T64 * T64));
    CKI(dmalloc(&c->XLbar, (size_t)n * c->q));
    CKI(dmalloc(&c->Ybar, (size_t)n * t));
    CKI(dmalloc(&c->S_TL, (size_t)c->q * c->q));
    CKI(dmalloc(&c->bbar_T, (size_t)c->q * t));
    CKI(dmalloc(&c->d_info, 1));
    c->ldp = round_up(o.m_blk, 32);
    const int nred = c->q + 1 + t;
    c->mixed = (o.precision == GWAS_PREC_MIXED);
    CKI(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    if (!c->mixed) {
        CKI(dmalloc(&c->part, (size_t)nt * nred * c->ldp));
    } else {
        MixedDev& m = c->mx;
        apply_tile_cfg(m, o.tile_cfg);
        mixed_layout(m, n, o.n_limbs, c->q + t, o.m_blk);
        if (!mixed_shape_built(m)) {
            free_all(c);
            delete c;
            return GWAS_ERR_UNSUPPORTED;
        }
        CKI(dmalloc(&c->Z, (size_t)n * (c->q + t)));
        CKI(mixed_alloc_layout(m));
        CKI(dmalloc(&m.Xb, (size_t)m.mb_pad_max * m.n_pad));
        CKI(cudaMemset(m.Xb, 0, (size_t)m.mb_pad_max * m.n_pad * sizeof(uint16_t)));
        CKI(dmalloc(&m.err, 1));
        CKI(cudaMemset(m.err, 0, sizeof(int)));
    }
    CKI(dmalloc(&c->bad, (size_t)o.m_blk));
    for (int s = 0; s < 2; ++s) {
        CKI(cudaEventCreateWithFlags(&c->ev_h2d[s], cudaEventDisableTiming));
        CKI(cudaEventCreateWithFlags(&c->ev_comp[s], cudaEventDisableTiming));
        CKI(cudaEventCreateWithFlags(&c->ev_d2h[s], cudaEventDisableTiming));
    }
    CKI(cudaStreamCreateWithFlags(&c->s_comp, cudaStreamNonBlocking));
    {
        int least = 0, greatest = 0;
        CKI(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CKI(cudaStreamCreateWithPriority(&c->chol.panel, cudaStreamNonBlocking, greatest));
        for (cudaEvent_t& ev : c->chol.ev) CKI(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    if (c->mixed) {
        CKI(cudaStreamCreateWithFlags(&c->s_aux, cudaStreamNonBlocking));
        for (cudaEvent_t* ev : {&c->ev_conv0, &c->ev_conv1, &c->ev_blk0, &c->ev_solve0})
            CKI(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    }
    CKI(cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking));
    CKI(cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking));
#undef CKI
    *out = c;
    return GWAS_OK;
}

gwas_status gwas_factor(gwas_ctx* c, const double* M_or_Phi, int is_phi, double h,
                        double sigma2, const double* XL, const double* Y) {
    Range range_("gwas_factor");
    if (!c) return GWAS_ERR_ARG;
    if (!M_or_Phi || !XL || !Y) return fail(c, GWAS_ERR_ARG, "gwas_factor: NULL input");
    if (is_phi && !(h >= 0.0 && h <= 1.0 && sigma2 > 0.0))
        return fail(c, GWAS_ERR_ARG, "gwas_factor: need 0 <= h <= 1 and sigma2 > 0");
    DeviceGuard g(c->device);
    c->factored = false;
    c->grad_ready = false;
    c->minv_ready = false;
    c->err_index = -1;
    const int64_t n = c->n, ld = c->ld;
    cudaStream_t s = c->s_comp;
    CK(cudaStreamSynchronize(c->s_h2d));
    CK(cudaStreamSynchronize(c->s_d2h));
    cudaEvent_t f0 = pooled_event(c), f1 = pooled_event(c);
    CK(cudaEventRecord(f0, s));
    int64_t nl = 0;
    // Phi (or M) is staged in the W buffer, then M is built into L's buffer.
    CK(cudaMemcpy2DAsync(c->W, ld * sizeof(double), M_or_Phi, n * sizeof(double),
                         n * sizeof(double), n, cudaMemcpyDefault, s));
    // [X_L | Y] (kept for the REML identities); the inputs are all on the device from here
    if (!c->XLY) CK(dmalloc(&c->XLY, (size_t)n * (c->q + c->t)));
    double* XLin = c->XLY;
    double* Yin = XLin + (size_t)n * c->q;
    CK(cudaMemcpyAsync(XLin, XL, (size_t)n * c->q * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(Yin, Y, (size_t)n * c->t * sizeof(double), cudaMemcpyDefault, s));
    const int init = 0x7fffffff;
    CK(cudaMemcpyAsync(c->d_info, &init, sizeof(int), cudaMemcpyHostToDevice, s));
    cudaEvent_t fu = pooled_event(c);
    CK(cudaEventRecord(fu, s));
    CK(launch_build_M(c->W, ld, c->L, ld, n, is_phi, h, sigma2, s));
    ++nl;
    CK(cholesky_blocked(c->L, ld, n, c->Dinv, c->d_info, s, &nl, &c->chol));
    // W := L^{-1}
    CK(cudaMemsetAsync(c->W, 0, (size_t)ld * ld * sizeof(double), s));
    const int64_t half = round_up(ceil_div(n, 2), T64);
    TmpDev tmp_buf;
    CK(cudaMalloc(&tmp_buf.p, (size_t)half * half * sizeof(double)));
    double* tmp = (double*)tmp_buf.p;
    CK(trtri_lower(c->L, ld, n, c->Dinv, c->W, ld, tmp, s, &nl));
    // Xbar_L := W X_L, Ybar := W Y
    {
        GemmF64 a;
        a.M = n; a.N = c->q; a.K = n; a.A = c->W; a.lda = ld; a.a_lower = true;
        a.B = XLin; a.ldb = n; a.C = c->XLbar; a.ldc = n;
        CK(gemm_f64(a, s));
        GemmF64 b = a;
        b.N = c->t; b.B = Yin; b.C = c->Ybar;
        CK(gemm_f64(b, s));
        // S_TL := Xbar_L^T Xbar_L, bbar_T := Xbar_L^T Ybar
        GemmF64 st;
        st.M = c->q; st.N = c->q; st.K = n; st.A = c->XLbar; st.lda = n; st.transA = true;
        st.B = c->XLbar; st.ldb = n; st.C = c->S_TL; st.ldc = c->q;
        CK(gemm_f64(st, s));
        GemmF64 bt = st;
        bt.N = c->t; bt.B = c->Ybar; bt.C = c->bbar_T;
        CK(gemm_f64(bt, s));
        nl += 4;
        if (c->mixed) {
            // Z := W^T [Xbar_L | Ybar] (so S_BLi = Z_L^T x_i and bbar_Bi = Z_y^T x_i)
            GemmF64 z;
            z.M = n; z.N = c->q; z.K = n; z.A = c->W; z.lda = ld; z.transA = true;
            z.a_upper = true; z.B = c->XLbar; z.ldb = n; z.C = c->Z; z.ldc = n;
            CK(gemm_f64(z, s));
            GemmF64 zy = z;
            zy.N = c->t; zy.B = c->Ybar; zy.C = c->Z + (size_t)n * c->q;
            CK(gemm_f64(zy, s));
            nl += 2;
            CK(mixed_prepare(c->mx, c->W, ld, c->Z, s, &nl));
        }
    }
    // Mixed path: a SNP whose dosages are all equal is exactly collinear with X_L when the
    // all-ones column is, a pivot the limb arithmetic cannot resolve against the
    // 1e-12 threshold. Decide it once the way the FP64 path decides any SNP: one FP64
    // block solve of a column of ones.
    TmpDev probe_buf;
    uint8_t* probe_st = nullptr;
    if (c->mixed) {
        const int64_t nt = ceil_div(n, T64), nred = c->q + 1 + c->t, ldp = 32;
        const size_t part_b = (size_t)nt * nred * ldp * sizeof(double);
        const size_t b_b = round_up((int64_t)c->t * c->p * sizeof(double), 256);
        const size_t ones_b = round_up(n, 256);
        CK(cudaMalloc(&probe_buf.p, part_b + b_b + ones_b + 512));
        double* part = (double*)probe_buf.p;
        double* bo = (double*)((char*)probe_buf.p + part_b);
        int8_t* ones = (int8_t*)((char*)probe_buf.p + part_b + b_b);
        uint8_t* flags = (uint8_t*)ones + ones_b;
        probe_st = flags + 256;
        CK(cudaMemsetAsync(ones, 1, (size_t)n, s));
        CohortDev cv = cohort_view(c);
        cv.ones_singular = false;
        CK(launch_block_fp64(cv, ones, n, 1, part, ldp, flags, s));
        CK(launch_snp_solve(cv, part, ldp, (int)nt, flags, 1, bo, nullptr, probe_st, s));
        nl += 3;
    }
    CK(cudaEventRecord(f1, s));
    int info = 0;
    uint8_t ones_status = 0;
    CK(cudaMemcpyAsync(&info, c->d_info, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (probe_st)
        CK(cudaMemcpyAsync(&ones_status, probe_st, 1, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f, ms_up = 0.f;
    cudaEventElapsedTime(&ms, f0, f1);
    cudaEventElapsedTime(&ms_up, f0, fu);
    c->ev_pool.push_back(f0);
    c->ev_pool.push_back(f1);
    c->ev_pool.push_back(fu);
    c->stats.factor_ms = ms;
    c->stats.factor_upload_ms = ms_up;
    c->stats.factor_launches = nl;
    c->ones_singular = (ones_status == 1);
    if (info != init) {
        c->err_index = info;
        char buf[128];
        snprintf(buf, sizeof buf, "gwas_factor: M is not SPD (pivot %d)", info);
        return fail(c, GWAS_ERR_NOT_SPD, buf);
    }
    c->factored = true;
    return GWAS_OK;
}

// The host-memory path's device slots are allocated on its first use, so contexts that
// only ever take device pointers (gwas_solve_block_device, batches) never hold them.
static gwas_status ensure_host_slots(gwas_ctx* c) {
    const int64_t mblk = c->opts.m_blk;
    for (int s = 0; s < 2; ++s) {  // each buffer on its own, so a failed call can be retried
        if (!c->Xslot[s]) CK(dmalloc(&c->Xslot[s], (size_t)c->n * mblk));
        if (!c->bslot[s]) CK(dmalloc(&c->bslot[s], (size_t)mblk * c->t * c->p));
        if (!c->wslot[s]) CK(dmalloc(&c->wslot[s], (size_t)mblk * c->t));
        if (!c->sslot[s]) CK(dmalloc(&c->sslot[s], (size_t)mblk));
    }
    return GWAS_OK;
}

// One block from HOST memory through the double-buffered slots: the upload (int8
// dosages, or 2-bit calls unpacked on the compute stream) overlaps the previous
// block's compute, whose outputs leave on the D2H stream.
static gwas_status host_block(gwas_ctx* c, const void* X, bool packed, const int8_t* code,
                              int64_t mb, double* b, double* wald, uint8_t* status) {
    DeviceGuard g(c->device);
    gwas_status st;
    if ((st = ensure_host_slots(c)) != GWAS_OK) return st;
    const int64_t pbytes = ceil_div(c->n, 4);
    if (packed)
        for (int k = 0; k < 2; ++k)
            if (!c->Pslot[k]) CK(dmalloc(&c->Pslot[k], (size_t)pbytes * c->opts.m_blk));
    const int s = c->slot;
    c->slot ^= 1;
    const int64_t t = c->t, p = c->p;
    const size_t in_bytes = packed ? (size_t)(pbytes * mb) : (size_t)(c->n * mb);
    // load_start: the slot's previous block must be consumed by the compute stream
    CK(cudaStreamWaitEvent(c->s_h2d, c->ev_comp[s], 0));
    CK(cudaMemcpyAsync(packed ? (void*)c->Pslot[s] : (void*)c->Xslot[s], X, in_bytes,
                       cudaMemcpyHostToDevice, c->s_h2d));
    CK(cudaEventRecord(c->ev_h2d[s], c->s_h2d));
    // load_wait, and the slot's previous outputs must have left for the host
    CK(cudaStreamWaitEvent(c->s_comp, c->ev_h2d[s], 0));
    CK(cudaStreamWaitEvent(c->s_comp, c->ev_d2h[s], 0));
    if (packed) {
        CK(launch_unpack_2bit(c->Pslot[s], c->n, mb, code, c->Xslot[s], c->s_comp));
        c->stats.kernel_launches += 1;
    }
    st = run_block(c, c->Xslot[s], mb, c->bslot[s], wald ? c->wslot[s] : nullptr, c->sslot[s]);
    if (st != GWAS_OK) return st;
    CK(cudaEventRecord(c->ev_comp[s], c->s_comp));
    // store_start
    CK(cudaStreamWaitEvent(c->s_d2h, c->ev_comp[s], 0));
    CK(cudaMemcpyAsync(b, c->bslot[s], (size_t)mb * t * p * sizeof(double), cudaMemcpyDeviceToHost,
                       c->s_d2h));
    if (wald)
        CK(cudaMemcpyAsync(wald, c->wslot[s], (size_t)mb * t * sizeof(double),
                           cudaMemcpyDeviceToHost, c->s_d2h));
    CK(cudaMemcpyAsync(status, c->sslot[s], (size_t)mb, cudaMemcpyDeviceToHost, c->s_d2h));
    CK(cudaEventRecord(c->ev_d2h[s], c->s_d2h));
    // completion of this block for gwas_wait_block (drop the leading ones already done)
    while (!c->done_ev.empty() && cudaEventQuery(c->done_ev.front()) == cudaSuccess) {
        c->ev_pool.push_back(c->done_ev.front());
        c->done_ev.erase(c->done_ev.begin());
        ++c->done_base;
    }
    cudaEvent_t done = pooled_event(c);
    CK(cudaEventRecord(done, c->s_d2h));
    c->done_ev.push_back(done);
    ++c->host_blocks;
    c->stats.h2d_bytes += (int64_t)in_bytes;
    c->stats.d2h_bytes += mb * t * p * 8 + (wald ? mb * t * 8 : 0) + mb;
    return GWAS_OK;
}

gwas_status gwas_solve_block(gwas_ctx* c, const int8_t* X, int64_t mb, double* b, double* wald,
                             uint8_t* status) {
    gwas_status st = check_block_args(c, X, mb, b, status);
    if (st != GWAS_OK) return st;
    return host_block(c, X, false, nullptr, mb, b, wald, status);
}

gwas_status gwas_solve_block_packed(gwas_ctx* c, const uint8_t* Xp, int64_t mb,
                                    const int8_t* code, double* b, double* wald,
                                    uint8_t* status) {
    gwas_status st = check_block_args(c, (const int8_t*)Xp, mb, b, status);
    if (st != GWAS_OK) return st;
    if (!code) return fail(c, GWAS_ERR_ARG, "solve_block_packed: NULL code table");
    return host_block(c, Xp, true, code, mb, b, wald, status);
}

gwas_status gwas_solve_block_packed_device(gwas_ctx* c, const uint8_t* Xp, int64_t mb,
                                           const int8_t* code, double* b, double* wald,
                                           uint8_t* status) {
    gwas_status st = check_block_args(c, (const int8_t*)Xp, mb, b, status);
    if (st != GWAS_OK) return st;
    if (!code) return fail(c, GWAS_ERR_ARG, "solve_block_packed_device: NULL code table");
    DeviceGuard g(c->device);
    if (!c->Xunpack) CK(dmalloc(&c->Xunpack, (size_t)c->n * c->opts.m_blk));
    CK(launch_unpack_2bit(Xp, c->n, mb, code, c->Xunpack, c->s_comp));
    c->stats.kernel_launches += 1;
    return run_block(c, c->Xunpack, mb, b, wald, status);
}

gwas_status gwas_solve_block_device(gwas_ctx* c, const int8_t* X, int64_t mb, double* b,
                                    double* wald, uint8_t* status) {
    gwas_status st = check_block_args(c, X, mb, b, status);
    if (st != GWAS_OK) return st;
    DeviceGuard g(c->device);
    return run_block(c, X, mb, b, wald, status);
}

gwas_status gwas_solve_block_cov_device(gwas_ctx* c, const int8_t* X, int64_t mb, double* b,
                                        double* wald, uint8_t* status, double* cov) {
    gwas_status st = check_block_args(c, X, mb, b, status);
    if (st != GWAS_OK) return st;
    if (!cov) return fail(c, GWAS_ERR_ARG, "gwas_solve_block_cov_device: NULL cov");
    DeviceGuard g(c->device);
    return run_block(c, X, mb, b, wald, status, cov);
}

gwas_status gwas_solve_all(gwas_ctx* c, const int8_t* X, int64_t m, double* b, double* wald,
                           uint8_t* status) {
    if (!c) return GWAS_ERR_ARG;
    if (m < 0) return fail(c, GWAS_ERR_ARG, "solve_all: m < 0");
    const int64_t mblk = c->opts.m_blk, t = c->t, p = c->p;
    for (int64_t i0 = 0; i0 < m; i0 += mblk) {
        const int64_t mb = std::min<int64_t>(mblk, m - i0);
        gwas_status st = gwas_solve_block(c, X + i0 * c->n, mb, b + i0 * t * p,
                                          wald ? wald + i0 * t : nullptr, status + i0);
        if (st != GWAS_OK) return st;
    }
    return gwas_sync(c, -1);
}

gwas_status gwas_sync(gwas_ctx* c, int timeout_ms) {
    if (!c) return GWAS_ERR_ARG;
    DeviceGuard g(c->device);
    cudaStream_t ss[3] = {c->s_h2d, c->s_comp, c->s_d2h};
    auto check_kernel_flag = [&]() -> gwas_status {
        if (!c->mixed || !c->mx.err) return GWAS_OK;
        int code = 0;
        CK(cudaMemcpy(&code, c->mx.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (code == 0) return GWAS_OK;
        CK(cudaMemset(c->mx.err, 0, sizeof(int)));
        char buf[128];
        snprintf(buf, sizeof buf, "mixed block kernel: a pipeline wait timed out (site %d)", code);
        return fail(c, GWAS_ERR_CUDA, buf);
    };
    if (timeout_ms < 0) {
        for (auto s : ss) CK(cudaStreamSynchronize(s));
        return check_kernel_flag();
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        bool done = true;
        for (auto s : ss) {
            cudaError_t e = cudaStreamQuery(s);
            if (e == cudaErrorNotReady) { done = false; continue; }
            if (e != cudaSuccess) return cuda_fail(c, e, "gwas_sync");
        }
        if (done) return check_kernel_flag();
        const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(
                            std::chrono::steady_clock::now() - t0).count();
        if (el >= timeout_ms) return fail(c, GWAS_ERR_TIMEOUT, "gwas_sync: timed out");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

gwas_status gwas_wait_block(gwas_ctx* c, int64_t block, int timeout_ms) {
    if (!c) return GWAS_ERR_ARG;
    if (block < 0 || block >= c->host_blocks)
        return fail(c, GWAS_ERR_ARG, "gwas_wait_block: no such host-path block");
    if (block < c->done_base) return GWAS_OK;
    DeviceGuard g(c->device);
    cudaEvent_t e = c->done_ev[(size_t)(block - c->done_base)];
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(e);
        if (q == cudaSuccess) return GWAS_OK;
        if (q != cudaErrorNotReady) return cuda_fail(c, q, "gwas_wait_block");
        if (timeout_ms >= 0) {
            const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (el >= timeout_ms) return fail(c, GWAS_ERR_TIMEOUT, "gwas_wait_block: timed out");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

gwas_status gwas_host_alloc(size_t bytes, void** out) {
    if (!out) return GWAS_ERR_ARG;
    *out = nullptr;
    if (bytes == 0) return GWAS_OK;
    return cudaHostAlloc(out, bytes, cudaHostAllocPortable) == cudaSuccess ? GWAS_OK : GWAS_ERR_OOM;
}

gwas_status gwas_host_free(void* p) {
    if (!p) return GWAS_OK;
    return cudaFreeHost(p) == cudaSuccess ? GWAS_OK : GWAS_ERR_CUDA;
}

gwas_status gwas_finalize(gwas_ctx* c) {
    if (!c) return GWAS_OK;
    {
        DeviceGuard g(c->device);
        cudaStreamSynchronize(c->s_h2d);
        cudaStreamSynchronize(c->s_comp);
        if (c->s_aux) cudaStreamSynchronize(c->s_aux);
        cudaStreamSynchronize(c->s_d2h);
        free_all(c);
    }
    delete c;
    return GWAS_OK;
}

const char* gwas_last_error(const gwas_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t gwas_error_index(const gwas_ctx* c) { return c ? c->err_index : -1; }

gwas_status gwas_get_stats(gwas_ctx* c, gwas_stats* out) {
    if (!c || !out) return GWAS_ERR_ARG;
    DeviceGuard g(c->device);
    gwas_status st = gwas_sync(c, -1);
    if (st != GWAS_OK) return st;
    fold_timings(c, true);
    *out = c->stats;
    return GWAS_OK;
}

gwas_status gwas_reset_stats(gwas_ctx* c) {
    if (!c) return GWAS_ERR_ARG;
    gwas_stats tmp;
    gwas_status st = gwas_get_stats(c, &tmp);
    const double fms = c->stats.factor_ms, fup = c->stats.factor_upload_ms;
    const int64_t fl = c->stats.factor_launches;
    c->stats = gwas_stats{};
    c->stats.factor_ms = fms;
    c->stats.factor_upload_ms = fup;
    c->stats.factor_launches = fl;
    return st;
}

void* gwas_stream(const gwas_ctx* c) { return c ? (void*)c->s_comp : nullptr; }

}  // extern "C"

// ============================================================================
// Tile configuration and the autotuner.
// ============================================================================
extern "C" {

gwas_status gwas_set_tile_cfg(gwas_ctx* c, int tile_cfg) {
    if (!c) return GWAS_ERR_ARG;
    if (!c->mixed) {
        c->opts.tile_cfg = tile_cfg;
        return GWAS_OK;
    }
    DeviceGuard g(c->device);
    CK(cudaStreamSynchronize(c->s_comp));
    MixedDev& m = c->mx;
    const int old_R = m.R, old_NT = m.NT, old_radix = m.radix;
    const bool old_pair = m.pair, old_fused = m.fused, old_ztail = m.ztail;
    const int old_nrt = m.n_rt;
    apply_tile_cfg(m, tile_cfg);
    mixed_layout(m, c->n, m.S, m.R_e, c->opts.m_blk);
    if (!mixed_shape_built(m)) {
        apply_tile_cfg(m, c->opts.tile_cfg);
        mixed_layout(m, c->n, m.S, m.R_e, c->opts.m_blk);
        return fail(c, GWAS_ERR_UNSUPPORTED, "gwas_set_tile_cfg: no kernel for that layout");
    }
    c->opts.tile_cfg = tile_cfg;
    const bool relayout = m.R != old_R || m.NT != old_NT || m.fused != old_fused ||
                          m.ztail != old_ztail || m.n_rt != old_nrt;
    const bool was_factored = c->factored;
    if (relayout || (was_factored && (m.pair != old_pair || m.radix != old_radix))) {
        // the limbs are rebuilt: until that succeeds the context holds no usable factor
        // (a failed re-allocation must not leave a solve launching on freed buffers)
        c->factored = false;
        if (relayout) CK(mixed_alloc_layout(m));
        if (was_factored) {
            int64_t nl = 0;
            CK(mixed_prepare(m, c->W, c->ld, c->Z, c->s_comp, &nl));
            CK(cudaStreamSynchronize(c->s_comp));
            c->factored = true;
        }
    }
    return GWAS_OK;
}

gwas_status gwas_autotune(gwas_ctx* c, const int8_t* X, int64_t mb_max, int reps, gwas_tune* out) {
    Range range_("gwas_autotune");
    if (!c || !out) return GWAS_ERR_ARG;
    if (!c->factored) return fail(c, GWAS_ERR_STATE, "gwas_autotune before gwas_factor");
    if (mb_max < 1 || mb_max > c->opts.m_blk) mb_max = c->opts.m_blk;
    if (reps < 1) reps = 3;
    DeviceGuard g(c->device);
    // dosages: the caller's, or synthetic ones (the timing does not depend on the values)
    TmpDev xbuf, outbuf;
    const int8_t* Xd = X;
    if (!Xd) {
        CK(cudaMalloc(&xbuf.p, (size_t)c->n * mb_max));
        CK(launch_fill_dosages((int8_t*)xbuf.p, (int64_t)c->n * mb_max, 0x9E3779B97F4A7C15ull,
                               c->s_comp));
        Xd = (const int8_t*)xbuf.p;
    }
    const size_t bbytes = (size_t)mb_max * c->t * c->p * sizeof(double);
    CK(cudaMalloc(&outbuf.p, bbytes + (size_t)mb_max * c->t * sizeof(double) + mb_max + 256));
    double* bo = (double*)outbuf.p;
    double* wo = bo + (size_t)mb_max * c->t * c->p;
    uint8_t* so = (uint8_t*)(wo + (size_t)mb_max * c->t);

    std::vector<int> cfgs;
    if (c->mixed) {
        // a radix cap set by the caller (tile_cfg bits 15-16) is kept
        const int keep = c->opts.tile_cfg >= 0 ? (c->opts.tile_cfg & (3 << 15)) : 0;
        for (int variant : {1 << 12, 1 << 13, (1 << 17) | (1 << 12), (1 << 17) | (1 << 13),
                            (1 << 21) | (1 << 12), (1 << 21) | (1 << 13)})
            for (int group : {40, 80, 160})
                for (int stages : {0, 4}) cfgs.push_back(keep | variant | (group << 4) | stages);
    } else {
        cfgs.push_back(-1);
    }
    std::vector<int64_t> mbs;
    for (int64_t mb : {(int64_t)4096, (int64_t)8192, (int64_t)16384, mb_max})
        if (mb <= mb_max && (mbs.empty() || mbs.back() != mb)) mbs.push_back(mb);
    std::sort(mbs.begin(), mbs.end());
    mbs.erase(std::unique(mbs.begin(), mbs.end()), mbs.end());

    const int saved_cfg = c->opts.tile_cfg;
    const int saved_timing = c->opts.timing;
    const gwas_stats saved_stats = c->stats;
    c->opts.timing = 0;
    cudaEvent_t e0 = pooled_event(c), e1 = pooled_event(c);
    // time `runs` back-to-back block solves of mb SNPs after one untimed one: ms per SNP
    auto time_cfg = [&](int64_t mb, int runs, double* per_snp) -> gwas_status {
        gwas_status s2 = run_block(c, Xd, mb, bo, wo, so);
        if (s2 != GWAS_OK) return s2;
        CK(cudaEventRecord(e0, c->s_comp));
        for (int r = 0; r < runs; ++r)
            if ((s2 = run_block(c, Xd, mb, bo, wo, so)) != GWAS_OK) return s2;
        CK(cudaEventRecord(e1, c->s_comp));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        *per_snp = ms / (runs * (double)mb);
        return GWAS_OK;
    };
    // coarse sweep over every (configuration, block size), then the four fastest are
    // timed again, interleaved over three rounds with twice the launches; the choice is
    // the fastest of those (best round each), which keeps one lucky short timing from
    // deciding between near-equal candidates
    struct Cand { double per_snp; int cfg; int64_t mb; };
    std::vector<Cand> coarse;
    int tried = 0;
    gwas_status st = GWAS_OK;
    for (int cfg : cfgs) {
        if ((st = gwas_set_tile_cfg(c, cfg)) == GWAS_ERR_UNSUPPORTED) {
            st = GWAS_OK;
            continue;
        }
        if (st != GWAS_OK) break;
        for (int64_t mb : mbs) {
            double v = 0.0;
            if ((st = time_cfg(mb, reps, &v)) != GWAS_OK) break;
            ++tried;
            coarse.push_back({v, cfg, mb});
        }
        if (st != GWAS_OK) break;
    }
    std::stable_sort(coarse.begin(), coarse.end(),
                     [](const Cand& a, const Cand& b) { return a.per_snp < b.per_snp; });
    if (coarse.size() > 4) coarse.resize(4);
    std::vector<double> fine(coarse.size(), 1e300);
    for (int round = 0; round < 3 && st == GWAS_OK && coarse.size() > 1; ++round) {
        for (size_t k = 0; k < coarse.size() && st == GWAS_OK; ++k) {
            double v = 0.0;
            if ((st = gwas_set_tile_cfg(c, coarse[k].cfg)) != GWAS_OK) break;
            if ((st = time_cfg(coarse[k].mb, 2 * reps, &v)) != GWAS_OK) break;
            fine[k] = std::min(fine[k], v);
        }
    }
    double best = 1e300;
    int best_cfg = saved_cfg;
    int64_t best_mb = mbs.back();
    for (size_t k = 0; k < coarse.size(); ++k) {
        const double v = coarse.size() > 1 ? fine[k] : coarse[k].per_snp;
        if (v < best) {
            best = v;
            best_cfg = coarse[k].cfg;
            best_mb = coarse[k].mb;
        }
    }
    // Short timings run below the power cap and do not see the power that DRAM traffic
    // costs in a long run; larger L2 groups of SNP tiles re-read more dosages (n = 10k:
    // 3.9 GB per block with 40 MB groups, 7.9 GB with 160 MB at equal short-run time). So
    // among the candidates within 1 % of the fastest, the one with the smallest group wins.
    if (c->mixed && coarse.size() > 1) {
        const double best_time = best;
        auto group_of = [](int cfg) { return ((cfg >> 4) & 0xFF) ? ((cfg >> 4) & 0xFF) : 40; };
        for (size_t k = 0; k < coarse.size(); ++k) {
            if (fine[k] <= 1.01 * best_time && group_of(coarse[k].cfg) < group_of(best_cfg)) {
                best = fine[k];
                best_cfg = coarse[k].cfg;
                best_mb = coarse[k].mb;
            }
        }
    }
    c->ev_pool.push_back(e0);
    c->ev_pool.push_back(e1);
    c->opts.timing = saved_timing;
    c->stats = saved_stats;  // runs made by the tuner are not the caller's work
    const gwas_status st2 = gwas_set_tile_cfg(c, st == GWAS_OK ? best_cfg : saved_cfg);
    if (st != GWAS_OK) return st;
    if (st2 != GWAS_OK) return st2;
    gwas_status sk = gwas_sync(c, -1);
    if (sk != GWAS_OK) return sk;
    out->tile_cfg = best_cfg;
    out->m_blk = best_mb;
    out->ms_per_snp = best;
    out->snps_per_s = 1e3 / best;
    out->candidates = tried;
    return GWAS_OK;
}

}  // extern "C"
