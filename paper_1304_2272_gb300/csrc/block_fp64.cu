// FP64 hot path of one SNP block (Algorithm 2, Section 3, loop body):
//   Xbar_blk := L^{-1} X_blk, fused with the per-SNP reductions of Algorithm 1
//   S_BLi = Xbar_Ri^T Xbar_L, S_BRi = Xbar_Ri^T Xbar_Ri, bbar_Bi = Xbar_Ri^T ybar.
//
// L^{-1} (= W) is formed once per cohort, so the block's triangular solve becomes a
// lower-triangular matrix product W X_blk with no dependency between row tiles:
// every (row tile, SNP tile) pair is an independent unit, Xbar never reaches global
// memory, and the reductions are taken from the tile while it sits in registers.
// Each unit writes its row-tile partial sums; k_reduce_partials adds them in a fixed
// order (no float atomics, so results are reproducible run to run).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gwas {

// One CTA = one 64-row x 64-SNP unit; 256 threads, 4 rows x 4 SNPs per thread.
// Thread (tx, ty): rows r0 + tx + 16 a, SNPs ty + 16 b. Within an L2 group of SNP tiles the
// units are ordered heaviest row tile first (a row tile needs k below its last row) so the
// tail of the grid is short.
__device__ __forceinline__ void block_fp64_unit(const CohortDev& c, const int8_t* __restrict__ X,
                                                int64_t ldx, int64_t mb, int n_rt, int rt, int ct,
                                                double* __restrict__ part, int64_t ldp,
                                                uint8_t* __restrict__ bad) {
    __shared__ double As[KC64][T64 + 1];  // W(r0 + i, k0 + k)
    __shared__ double Bs[KC64][T64 + 1];  // x(k0 + k, c0 + j) as double
    __shared__ int sbad[T64];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t n = c.n;
    // the row tiles end at row n (tile rt holds rows rt*64 - off ..), so the one short tile
    // is the first, whose k-range is the shortest
    const int64_t off = (int64_t)n_rt * T64 - n;
    const int64_t r0 = (int64_t)rt * T64 - off, c0 = (int64_t)ct * T64;
    const int64_t kend = c.dense ? n : min64(n, r0 + T64);
    const bool check = (rt == n_rt - 1);  // this unit reads every dosage of its SNPs
    if (tid < T64) sbad[tid] = 0;
    __syncthreads();

    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    for (int64_t k0 = 0; k0 < kend; k0 += KC64) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;
            const int ii = e % T64, kk = e / T64;
            const int64_t gi = r0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi >= 0 && gi < n && gk < kend) ? c.W[gi + gk * c.ldw] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;
            const int kk = e % KC64, jj = e / KC64;
            const int64_t gk = k0 + kk, gj = c0 + jj;
            double v = 0.0;
            if (gk < kend && gj < mb) {
                const int d = X[gk + gj * ldx];
                if (check && (unsigned)d > 2u) sbad[jj] = 1;
                v = dosage_to_f64(d);
            }
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

    // Epilogue: partial sums over this tile's rows of xbar * z for
    // z in [Xbar_L(:, 0..q-1) | xbar | Ybar(:, 0..t-1)].
    const int q = c.q, nred = q + 1 + c.t;
    for (int v = 0; v < nred; ++v) {
        double zr[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t gi = r0 + tx + 16 * a;
            double z = 0.0;
            if (gi >= 0 && gi < n) {
                if (v < q) z = c.XLbar[gi + (int64_t)v * n];
                else if (v > q) z = c.Ybar[gi + (int64_t)(v - q - 1) * n];
            }
            zr[a] = z;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) s = fma(acc[a][b], (v == q) ? acc[a][b] : zr[a], s);
            // reduce over the 16 row groups (tx = lanes 0..15 of each half warp)
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            const int64_t gj = c0 + ty + 16 * b;
            if (tx == 0 && gj < mb) part[((int64_t)rt * nred + v) * ldp + gj] = s;
        }
    }
    if (check) {
        __syncthreads();
        if (tid < T64 && c0 + tid < mb) bad[c0 + tid] = (uint8_t)sbad[tid];
    }
}

// Units are taken group by group of `group` SNP tiles (a group's dosages stay in L2 while
// every row tile of L^{-1} passes over them, so each dosage byte comes from DRAM about once
// and each row tile of L^{-1} once per group), and within a group row tile by row tile,
// the heaviest (longest k-range) first.
__global__ void __launch_bounds__(256)
k_block_fp64(CohortDev c, const int8_t* __restrict__ X, int64_t ldx, int64_t mb, int n_rt,
             int n_ct, int group, double* __restrict__ part, int64_t ldp,
             uint8_t* __restrict__ bad) {
    const int64_t u = blockIdx.x;
    const int64_t per_group = (int64_t)n_rt * group;
    const int g = (int)(u / per_group);
    const int gsz = min(group, n_ct - g * group);
    const int local = (int)(u - g * per_group);
    block_fp64_unit(c, X, ldx, mb, n_rt, n_rt - 1 - local / gsz, g * group + local % gsz, part,
                    ldp, bad);
}

// Batched cohorts: one grid over every cohort's units (cohort found by binary search).
__global__ void __launch_bounds__(256)
k_block_fp64_batch(const BatchJob* __restrict__ jobs, int n_jobs) {
    const int64_t u = blockIdx.x;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (jobs[mid].unit_base <= u) lo = mid;
        else hi = mid - 1;
    }
    const BatchJob& j = jobs[lo];
    const int unit = (int)(u - j.unit_base);
    block_fp64_unit(j.c, j.X, j.c.n, j.mb, j.n_rt64, j.n_rt64 - 1 - unit / j.n_ct64,
                    unit % j.n_ct64, j.part, j.ldp, j.bad);
}

cudaError_t launch_block_fp64_batch(const BatchJob* jobs, int n_jobs, int64_t n_units,
                                    cudaStream_t s) {
    if (n_units <= 0) return cudaSuccess;
    if (n_units > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_block_fp64_batch<<<(unsigned)n_units, 256, 0, s>>>(jobs, n_jobs);
    return cudaGetLastError();
}

cudaError_t launch_block_fp64(const CohortDev& c, const int8_t* X, int64_t ldx, int64_t mb,
                              double* part, int64_t ldp, uint8_t* bad, cudaStream_t s) {
    const int n_rt = (int)ceil_div(c.n, T64);
    const int n_ct = (int)ceil_div(mb, T64);
    const int64_t units = (int64_t)n_rt * n_ct;
    if (units <= 0) return cudaSuccess;
    if (units > 0x7fffffffLL) return cudaErrorInvalidValue;
    // SNP tiles per group: 40 MB of int8 dosages
    const int group = (int)std::max<int64_t>(1, std::min<int64_t>(n_ct, (40ll << 20) / (T64 * ldx)));
    k_block_fp64<<<(unsigned)units, 256, 0, s>>>(c, X, ldx, mb, n_rt, n_ct, group, part, ldp, bad);
    return cudaGetLastError();
}

}  // namespace gwas
