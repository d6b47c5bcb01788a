// Internal declarations shared by the C-ABI translation units (gwas_api.cu: contexts
// and the block pipeline; reml_api.cu: REML and db/dh; batch_api.cu: batches of cohorts).
// Not part of the ABI.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gwas.h"
#include "common.cuh"
#include "kernels.h"

using namespace gwas;

struct gwas_ctx {
    gwas_opts opts{};
    int device = 0;
    int64_t n = 0;
    int p = 0, q = 0, t = 0;
    int64_t ld = 0;               // leading dimension of L and W
    double* L = nullptr;          // n x n: M, then its Cholesky factor
    double* W = nullptr;          // n x n: L^{-1}
    double* Dinv = nullptr;       // diagonal 64 x 64 inverses
    double* XLbar = nullptr;      // n x q
    double* Ybar = nullptr;       // n x t
    double* S_TL = nullptr;       // q x q
    double* bbar_T = nullptr;     // q x t
    int* d_info = nullptr;
    // block pipeline
    int8_t* Xslot[2] = {nullptr, nullptr};
    double* bslot[2] = {nullptr, nullptr};
    double* wslot[2] = {nullptr, nullptr};
    uint8_t* sslot[2] = {nullptr, nullptr};
    uint8_t* Pslot[2] = {nullptr, nullptr};  // 2-bit packed host blocks (first use)
    int8_t* Xunpack = nullptr;    // unpacked dosages of gwas_solve_block_packed_device
    double* part = nullptr;       // row-tile partial sums
    int64_t ldp = 0;
    uint8_t* bad = nullptr;
    // mixed-precision path
    bool mixed = false;
    MixedDev mx;
    double* Z = nullptr;          // n x (q + t): L^{-T} [Xbar_L | Ybar] = M^{-1} [X_L | Y]
    // REML and db/dh (allocated on first use)
    double* Phi = nullptr;        // full Phi, ld
    double* Minv = nullptr;       // M^{-1} = L^{-T} L^{-1}, ld (formed when db/dh needs it)
    bool minv_ready = false;      // Minv holds M^{-1} of the current factor
    double* XLY = nullptr;        // [X_L | Y] (n x (q+t)) as given to the last gwas_factor
    double* part2 = nullptr;      // adjoint partials, FP64 partial layout
    double* small = nullptr;      // G1, G2, PhiZ and scalars
    bool grad_ready = false;
    double grad_h = 0.0, grad_s2 = 0.0;
    bool ones_singular = false;   // the all-ones SNP is collinear with X_L (mixed path)
    int num_sms = 0;
    cudaStream_t s_comp = nullptr, s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_h2d[2] = {}, ev_comp[2] = {}, ev_d2h[2] = {};
    // mixed path: a block is solved in two halves; the second half's dosage conversion
    // and the first half's p x p solves run on s_aux beside the other half's block kernel
    cudaStream_t s_aux = nullptr;
    cudaEvent_t ev_conv0 = nullptr, ev_conv1 = nullptr, ev_blk0 = nullptr, ev_solve0 = nullptr;
    // the blocked Cholesky's panel chain (highest stream priority) beside its trailing
    // updates on s_comp
    CholLookahead chol;
    int slot = 0;
    bool factored = false;
    std::string err;
    int64_t err_index = -1;
    gwas_stats stats{};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timed;  // pending trsm timings
    std::vector<cudaEvent_t> ev_pool;
    // host-path blocks: number submitted, and the completion events (D2H done) of those
    // from index done_base on that are not yet known to be complete
    int64_t host_blocks = 0, done_base = 0;
    std::vector<cudaEvent_t> done_ev;
};

namespace gwas_api {

// NVTX range over one API call (named in profiler timelines; free without a tool).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

gwas_status fail(gwas_ctx* c, gwas_status st, const std::string& msg);
gwas_status cuda_fail(gwas_ctx* c, cudaError_t e, const char* where);

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
    const cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 256);
    if (e != cudaSuccess) *p = nullptr;  // a failed allocation leaves nothing to free or use
    return e;
}

CohortDev cohort_view(const gwas_ctx* c);

// Owns a temporary device allocation for the duration of one call.
struct TmpDev {
    void* p = nullptr;
    ~TmpDev() {
        if (p) cudaFree(p);
    }
};

cudaEvent_t pooled_event(gwas_ctx* c);
void fold_timings(gwas_ctx* c, bool wait);
// The block compute on the compute stream (see gwas_api.cu).
gwas_status run_block(gwas_ctx* c, const int8_t* X, int64_t mb, double* b, double* wald,
                      uint8_t* status, double* cov = nullptr);
void apply_tile_cfg(MixedDev& m, int tile_cfg);
cudaError_t mixed_alloc_layout(MixedDev& m);
void free_all(gwas_ctx* c);
gwas_status check_block_args(gwas_ctx* c, const int8_t* X, int64_t mb, double* b,
                             uint8_t* status);

}  // namespace gwas_api

// Return the CUDA error of `call` as a gwas_status of context `c` (in scope).
#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return gwas_api::cuda_fail(c, e_, #call);  \
    } while (0)
