// C ABI of batches of cohorts (include/gwas.h, gwas_batch_*): one grouped launch of the
// block kernel over every cohort of the batch, optionally replayed from a CUDA graph.
#include "api_internal.h"

using namespace gwas_api;

// ============================================================================
// Batches of cohorts: each cohort keeps its own context (factor, L^{-1}, limbs,
// buffers); a batched solve is ONE grouped launch of the block kernel over every
// cohort's (row tile, SNP tile) units, optionally captured in a CUDA graph.
// ============================================================================
struct gwas_batch {
    gwas_opts opts{};
    int device = 0;
    int n_cohorts = 0;
    int p = 0, q = 0, t = 0;
    bool mixed = false;
    std::vector<gwas_ctx*> ctx;
    cudaStream_t s = nullptr;
    // Mixed batches run in parts (contiguous cohort ranges of about equal tensor work) on
    // two streams: part k's dosage conversion overlaps part k-1's block kernel, part k-1's
    // p x p solves overlap part k's block kernel, and part k's CTAs fill the tail of part
    // k-1's persistent grid.
    cudaStream_t s2 = nullptr;
    static constexpr int kMaxParts = 7;
    int n_parts = 1;
    int part_c0[kMaxParts + 1] = {};          // cohorts of part k: [part_c0[k], part_c0[k+1])
    int64_t part_snps[kMaxParts] = {}, part_units[kMaxParts] = {};
    bool part_small[kMaxParts] = {};          // every cohort of part k has small limb sums
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_conv[kMaxParts] = {};      // part k's conversion done
    BatchJob* d_jobs = nullptr;
    CohortMx* d_tab = nullptr;
    CUtensorMap* d_maps = nullptr;
    int* d_err = nullptr;
    // configuration the device tables (and the graph) were built for
    std::vector<uintptr_t> key;
    int64_t total_snps = 0, units_fp64 = 0, units_mx = 0;
    int stages = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string err;
    gwas_stats stats{};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timed;
};

namespace {

gwas_status bfail(gwas_batch* b, gwas_status st, const std::string& msg) {
    if (b) b->err = msg;
    return st;
}

#define CKB(call)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            cudaGetLastError();                                                         \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? GWAS_ERR_OOM : GWAS_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));           \
        }                                                                               \
    } while (0)

void batch_free(gwas_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto& pr : b->timed) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    cudaFree(b->d_jobs); cudaFree(b->d_tab); cudaFree(b->d_maps); cudaFree(b->d_err);
    for (cudaEvent_t ev : b->ev_conv) if (ev) cudaEventDestroy(ev);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->s2) cudaStreamDestroy(b->s2);
    if (b->s) cudaStreamDestroy(b->s);
    for (auto* c : b->ctx) gwas_finalize(c);
}

// As fold_timings, for a batch (its events are created per solve and destroyed here).
void batch_fold_timings(gwas_batch* b, bool wait) {
    size_t k = 0;
    for (; k < b->timed.size(); ++k) {
        auto& pr = b->timed[k];
        if (!wait && cudaEventQuery(pr.second) != cudaSuccess) break;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) b->stats.trsm_ms += ms;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    b->timed.erase(b->timed.begin(), b->timed.begin() + (std::ptrdiff_t)k);
}

// Enqueue the batched solve on the batch stream (device tables already current). A mixed
// batch in several parts forks onto the second stream and joins back before returning, so
// the whole solve stays ordered on b->s (and is captured as one graph).
gwas_status batch_enqueue(gwas_batch* b) {
    const int nc = b->n_cohorts;
    if (b->mixed) {
        const int P = b->n_parts;
        if (P > 1) {
            CKB(cudaEventRecord(b->ev_fork, b->s));
            CKB(cudaStreamWaitEvent(b->s2, b->ev_fork, 0));
        }
        for (int k = 0; k < P; ++k) {
            cudaStream_t st = (k % 2 == 0) ? b->s : b->s2;
            const int c0 = b->part_c0[k], nck = b->part_c0[k + 1] - c0;
            // the conversions run one after another, each beside the previous part's
            // block kernel
            if (k > 0) CKB(cudaStreamWaitEvent(st, b->ev_conv[k - 1], 0));
            CKB(launch_geno_bf16_batch(b->d_jobs + c0, nck, b->part_snps[k], st));
            if (P > 1) CKB(cudaEventRecord(b->ev_conv[k], st));
            CKB(launch_block_mixed_batch(b->d_tab + c0, b->d_maps + 3 * c0, nck, b->part_units[k],
                                         b->ctx[0]->mx, b->stages, b->d_err, b->part_small[k],
                                         b->ctx[0]->num_sms, st));
            CKB(launch_snp_solve_batch(b->d_jobs + c0, nck, b->part_snps[k], b->p,
                                       b->q + 1 + b->t, true, st));
        }
        if (P > 1) {
            CKB(cudaEventRecord(b->ev_join, b->s2));
            CKB(cudaStreamWaitEvent(b->s, b->ev_join, 0));
        }
    } else {
        CKB(launch_block_fp64_batch(b->d_jobs, nc, b->units_fp64, b->s));
        CKB(launch_snp_solve_batch(b->d_jobs, nc, b->total_snps, b->p, b->q + 1 + b->t, false, b->s));
    }
    return GWAS_OK;
}

}  // namespace

extern "C" {

gwas_status gwas_batch_init(int n_cohorts, const int64_t* n, int p, int t, const gwas_opts* opts,
                            gwas_batch** out) {
    if (!out) return GWAS_ERR_ARG;
    *out = nullptr;
    if (n_cohorts < 1 || !n) return GWAS_ERR_ARG;
    gwas_opts o;
    gwas_default_opts(&o);
    if (opts) o = *opts;
    gwas_batch* b = new gwas_batch();
    b->opts = o;
    b->device = o.device;
    b->n_cohorts = n_cohorts;
    b->p = p; b->q = p - 1; b->t = t;
    b->mixed = (o.precision == GWAS_PREC_MIXED);
    // every cohort takes the same tile configuration, hence the same kernel variant (the
    // tile height depends on the limb count only, the fusion of the linear rows on p, t)
    gwas_opts oc = o;
    for (int c = 0; c < n_cohorts; ++c) {
        gwas_ctx* cx = nullptr;
        const gwas_status st = gwas_init(n[c], p, t, &oc, &cx);
        if (st != GWAS_OK) {
            DeviceGuard g(b->device);
            batch_free(b);
            delete b;
            return st;
        }
        b->ctx.push_back(cx);
    }
    DeviceGuard g(b->device);
    auto bail = [&](cudaError_t e) {
        cudaGetLastError();
        batch_free(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? GWAS_ERR_OOM : GWAS_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    if (b->mixed && n_cohorts > 1) {
        if ((e = cudaStreamCreateWithFlags(&b->s2, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e);
        if ((e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming)) != cudaSuccess)
            return bail(e);
        for (cudaEvent_t& ev : b->ev_conv)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return bail(e);
    }
    if ((e = cudaMalloc(&b->d_jobs, sizeof(BatchJob) * n_cohorts)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&b->d_tab, sizeof(CohortMx) * n_cohorts)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * 3 * n_cohorts)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&b->d_err, sizeof(int))) != cudaSuccess) return bail(e);
    if ((e = cudaMemset(b->d_err, 0, sizeof(int))) != cudaSuccess) return bail(e);
    if (b->mixed) {
        const MixedDev& m = b->ctx[0]->mx;
        b->stages = mixed_stage_count(m);
        if ((e = mixed_batch_prepare(m, b->stages)) != cudaSuccess) return bail(e);
    }
    *out = b;
    return GWAS_OK;
}

gwas_status gwas_batch_factor(gwas_batch* b, int cohort, const double* M_or_Phi, int is_phi,
                              double h, double sigma2, const double* XL, const double* Y) {
    if (!b) return GWAS_ERR_ARG;
    if (cohort < 0 || cohort >= b->n_cohorts) return bfail(b, GWAS_ERR_ARG, "cohort out of range");
    const gwas_status st = gwas_factor(b->ctx[cohort], M_or_Phi, is_phi, h, sigma2, XL, Y);
    if (st != GWAS_OK) b->err = std::string("cohort ") + std::to_string(cohort) + ": " +
                                gwas_last_error(b->ctx[cohort]);
    b->key.clear();  // cohort constants changed: rebuild tables and graph
    return st;
}

gwas_status gwas_batch_solve_device(gwas_batch* b, const int8_t* const* X, const int64_t* mb,
                                    double* const* bo, double* const* wald,
                                    uint8_t* const* status) {
    Range range_("gwas batch solve");
    if (!b) return GWAS_ERR_ARG;
    if (!X || !mb || !bo || !status) return bfail(b, GWAS_ERR_ARG, "batch solve: NULL array");
    const int nc = b->n_cohorts;
    std::vector<uintptr_t> key;
    key.reserve(5 * nc);
    for (int c = 0; c < nc; ++c) {
        gwas_ctx* cx = b->ctx[c];
        if (!cx->factored) return bfail(b, GWAS_ERR_STATE, "batch solve before every cohort's factor");
        if (!X[c] || !bo[c] || !status[c]) return bfail(b, GWAS_ERR_ARG, "batch solve: NULL pointer");
        if (mb[c] < 1 || mb[c] > cx->opts.m_blk)
            return bfail(b, GWAS_ERR_ARG, "batch solve: need 1 <= mb[c] <= m_blk");
        key.push_back((uintptr_t)X[c]);
        key.push_back((uintptr_t)mb[c]);
        key.push_back((uintptr_t)bo[c]);
        key.push_back((uintptr_t)(wald ? wald[c] : nullptr));
        key.push_back((uintptr_t)status[c]);
    }
    DeviceGuard g(b->device);
    if (key != b->key) {
        // rebuild the device tables for this set of pointers and sizes
        CKB(cudaStreamSynchronize(b->s));
        std::vector<BatchJob> jobs(nc);
        std::vector<CohortMx> tab(nc);
        std::vector<CUtensorMap> maps(3 * nc);
        // parts of about equal tensor work (mixed, two or more cohorts): contiguous cohort
        // ranges, each with its own SNP and unit numbering
        int P = 1;
        b->part_c0[0] = 0;
        if (b->mixed && nc > 1 && b->s2) {
            std::vector<int64_t> w(nc);
            int64_t total = 0;
            for (int c = 0; c < nc; ++c) total += (w[c] = mixed_cohort_work(b->ctx[c]->mx, mb[c]));
            // tile_cfg bits 18-20: the number of parts (0 = six: measured on 48 cohorts of
            // n ~ U[1000, 8000] at power-capped clocks, BF16 TFLOP/s per MHz 0.72 with 2
            // parts, 0.70-0.76 with 3-4 (earlier epilogue), 0.80-0.85 with 4, 0.87 with 6,
            // 0.84 with 7)
            const int want = b->opts.tile_cfg >= 0 ? (b->opts.tile_cfg >> 18) & 7 : 0;
            P = std::min(nc, std::min(gwas_batch::kMaxParts, want > 0 ? want : 6));
            int64_t acc = 0;
            int k = 1;
            for (int c = 0; c < nc && k < P; ++c) {
                acc += w[c];
                // close part k-1 after cohort c once it holds its share of the work, leaving
                // at least one cohort for every later part
                if (acc * P >= total * k || nc - (c + 1) == P - k) b->part_c0[k++] = c + 1;
            }
        }
        b->part_c0[P] = nc;
        b->n_parts = P;
        int64_t snp = 0, u64 = 0, umx = 0, tot_snps = 0, tot_mx = 0;
        int part = 0;
        for (int c = 0; c < nc; ++c) {
            if (c == b->part_c0[part + 1]) {  // a new part: numbering restarts
                b->part_snps[part] = snp;
                b->part_units[part] = umx;
                ++part;
                snp = 0;
                umx = 0;
            }
            gwas_ctx* cx = b->ctx[c];
            BatchJob& j = jobs[c];
            j.c = cohort_view(cx);
            j.X = X[c];
            j.mb = mb[c];
            j.snp_base = snp;
            j.unit_base = u64;
            j.n_rt64 = (int)ceil_div(cx->n, T64);
            j.n_ct64 = (int)ceil_div(mb[c], T64);
            j.part = cx->part;
            j.ldp = cx->mixed ? cx->mx.ldp : cx->ldp;
            j.bad = cx->bad;
            j.b = bo[c];
            j.wald = wald ? wald[c] : nullptr;
            j.status = status[c];
            snp += mb[c];
            tot_snps += mb[c];
            if (b->mixed) {
                j.Xb = cx->mx.Xb;
                j.n_pad = cx->mx.n_pad;
                // cohorts of one part given the same dosages (several traits of one cohort,
                // each with its own M) convert them once and share the BF16 rows and flags
                int src = c;
                for (int e = b->part_c0[part]; e < c; ++e) {
                    if (X[e] == X[c] && mb[e] == mb[c] && b->ctx[e]->n == cx->n &&
                        jobs[e].convert) {
                        j.Xb = jobs[e].Xb;
                        j.bad = jobs[e].bad;
                        j.convert = 0;
                        src = e;
                        break;
                    }
                }
                j.sq_part = cx->mx.sq_part;
                j.lin = cx->mx.lin;
                j.n_tiles_mx = cx->mx.n_rt;
                j.lin_tiles = cx->mx.lin_tiles();
                tab[c] = mixed_cohort_entry(cx->mx, mb[c], umx);
                const int64_t uc = mixed_cohort_units(cx->mx, mb[c]);
                umx += uc;
                tot_mx += uc;
                maps[3 * c + 0] = b->ctx[src]->mx.tmX;
                // CTA pairs: each CTA loads half of a limb tile
                maps[3 * c + 1] = cx->mx.pair ? cx->mx.tmWh : cx->mx.tmW;
                maps[3 * c + 2] = cx->mx.pair ? cx->mx.tmEh : cx->mx.tmE;
            } else {
                u64 += (int64_t)j.n_rt64 * j.n_ct64;
            }
        }
        CKB(cudaMemcpy(b->d_jobs, jobs.data(), sizeof(BatchJob) * nc, cudaMemcpyHostToDevice));
        if (b->mixed) {
            CKB(cudaMemcpy(b->d_tab, tab.data(), sizeof(CohortMx) * nc, cudaMemcpyHostToDevice));
            CKB(cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * 3 * nc,
                           cudaMemcpyHostToDevice));
        }
        b->part_snps[part] = snp;
        b->part_units[part] = umx;
        for (int k = 0; k < P; ++k) {
            b->part_small[k] = true;
            for (int c = b->part_c0[k]; c < b->part_c0[k + 1]; ++c)
                if (!b->mixed || !tab[c].small_sums) b->part_small[k] = false;
        }
        b->total_snps = tot_snps;
        b->units_fp64 = u64;
        b->units_mx = tot_mx;
        if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        b->key = key;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->opts.timing) {
        if (b->timed.size() >= 64) batch_fold_timings(b, false);
        CKB(cudaEventCreate(&e0));
        CKB(cudaEventCreate(&e1));
        CKB(cudaEventRecord(e0, b->s));
    }
    if (b->opts.use_graph) {
        if (!b->gexec) {
            CKB(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
            const gwas_status st = batch_enqueue(b);
            cudaGraph_t gr = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->s, &gr);
            if (st != GWAS_OK) { if (gr) cudaGraphDestroy(gr); return st; }
            CKB(ec);
            b->graph = gr;
            CKB(cudaGraphInstantiate(&b->gexec, b->graph, 0));
        }
        CKB(cudaGraphLaunch(b->gexec, b->s));
    } else {
        const gwas_status st = batch_enqueue(b);
        if (st != GWAS_OK) return st;
    }
    if (b->opts.timing) {
        CKB(cudaEventRecord(e1, b->s));
        b->timed.emplace_back(e0, e1);
    }
    b->stats.blocks += 1;
    b->stats.snps += b->total_snps;
    b->stats.kernel_launches += b->mixed ? 4 * b->n_parts : 3;
    b->stats.trsm_launches += 1;
    return GWAS_OK;
}

gwas_status gwas_batch_sync(gwas_batch* b, int timeout_ms) {
    if (!b) return GWAS_ERR_ARG;
    DeviceGuard g(b->device);
    if (timeout_ms < 0) {
        CKB(cudaStreamSynchronize(b->s));
    } else {
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            const cudaError_t e = cudaStreamQuery(b->s);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) CKB(e);
            const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (el >= timeout_ms) return bfail(b, GWAS_ERR_TIMEOUT, "gwas_batch_sync: timed out");
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
    }
    int code = 0;
    CKB(cudaMemcpy(&code, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (code != 0) {
        CKB(cudaMemset(b->d_err, 0, sizeof(int)));
        return bfail(b, GWAS_ERR_CUDA, "batched mixed kernel: a pipeline wait timed out (site " +
                                           std::to_string(code) + ")");
    }
    return GWAS_OK;
}

gwas_status gwas_batch_get_stats(gwas_batch* b, gwas_stats* out) {
    if (!b || !out) return GWAS_ERR_ARG;
    const gwas_status st = gwas_batch_sync(b, -1);
    if (st != GWAS_OK) return st;
    batch_fold_timings(b, true);
    gwas_stats agg = b->stats;
    agg.factor_ms = 0;
    agg.factor_upload_ms = 0;
    agg.factor_launches = 0;
    for (auto* c : b->ctx) {
        agg.factor_ms += c->stats.factor_ms;
        agg.factor_upload_ms += c->stats.factor_upload_ms;
        agg.factor_launches += c->stats.factor_launches;
    }
    *out = agg;
    return GWAS_OK;
}

gwas_status gwas_batch_reset_stats(gwas_batch* b) {
    gwas_stats tmp;
    const gwas_status st = gwas_batch_get_stats(b, &tmp);
    if (b) b->stats = gwas_stats{};
    return st;
}

gwas_status gwas_batch_finalize(gwas_batch* b) {
    if (!b) return GWAS_OK;
    {
        DeviceGuard g(b->device);
        if (b->s) cudaStreamSynchronize(b->s);
        batch_free(b);
    }
    delete b;
    return GWAS_OK;
}

const char* gwas_batch_last_error(const gwas_batch* b) { return b ? b->err.c_str() : "null batch"; }

void* gwas_batch_stream(const gwas_batch* b) { return b ? (void*)b->s : nullptr; }

}  // extern "C"
