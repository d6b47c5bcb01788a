// Mixed-precision hot path of one SNP block on the BF16 tensor cores (tcgen05).
//
// Xbar_blk := L^{-1} X_blk (Algorithm 2, Section 3) is the dominant dense contraction.
// Dosages {0,1,2} are exact in BF16, so only W = L^{-1} needs splitting: per tile of R
// rows with exponent E (max |W| <= 2^E) and B bits per limb,
//     W = 2^(E-(B-1)) * sum_{l<S} A_l * 2^(-B l) + O(2^(E-BS)),   |A_l| <= 2^(B-1) integers,
// and every A_l is exact in BF16. A_l x_i then has integer products <= 2^B whose sums
// stay below 2^24 while n < 2^(24-B), so the FP32 tensor-core accumulation of each limb
// is exact: B = 9 for n < 32768, 8 for n < 65536, 7 for n < 131072. The epilogue
// needs, with the limb sums C_l of a row,
//     T = sum_l C_l * 2^(B (S-1-l)),   xbar = 2^(E-(B-1)-B(S-1)) * T,
// the sum of T^2 over a row tile for S_BRi = Xbar_Ri^T Xbar_Ri: it sums the 32 x 32-bit
// products C_l C_m per power of 2^B in 64-bit integers and combines them once in 128 bits,
// exactly. The only rounding left is the limb truncation of W (relative 2^(-BS) of the
// tile maximum) and one conversion to FP64 per (row tile, SNP).
//
// The linear reductions of Algorithm 1, S_BLi = Xbar_Ri^T Xbar_L and bbar_Bi =
// Xbar_Ri^T ybar, are the same numbers as Z^T x_i with Z = L^{-T} [Xbar_L | Ybar]
// (= M^{-1} [X_L | Y]); Z is split into limbs the same way and rides on the tensor cores
// too: in a separate linear tile per SNP tile, fused into every row tile on its own
// k-range, or as the last rows of the last row tile.
//
// Kernel structure (one persistent CTA per SM, 8 warps):
//   warp 0 lane 0: TMA producer (dosage tile 128 SNPs x 64 k, limb tile N x 64 k),
//   warp 1 lane 0: tcgen05.mma issuer, FP32 accumulators in TMEM (2 x 256 columns),
//   warps 4-7   : epilogue, one SNP per thread (TMEM lane), no cross-thread reduction.
// Every wait is bounded (2 s); on expiry the CTA records an error and winds down.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace gwas {
namespace mx {
constexpr int BM = 128;          // SNPs per tile: UMMA M, TMEM lanes
constexpr int BK = 64;           // k per pipeline stage: one 128-byte swizzle row of BF16
constexpr int BUF = 256;         // TMEM columns per accumulator buffer
constexpr uint32_t EXTRA = 0xFFFFu;
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr int SMEM_BUDGET = 200 * 1024;

// Every row tile is one UMMA of N = 256: one UMMA with M = 128 (or 256 across a CTA pair)
// takes about the same time for any N <= 256, so a tile holds as many rows of L^{-1} as
// S limbs allow, R = floor(256 / S) (85 for 3 limbs), the S limbs of each row side by
// side (column i S + l), zero rows up to 256. With the linear rows fused into the tile,
// R = floor((256 - S R_e) / S); with them as the last rows of the last tile, the tiles
// end at row n + R_e.
constexpr int NT = 256;
__host__ __device__ constexpr int rows_max(int S) { return NT / S; }
}  // namespace mx

// Launch-wide values (shared by every cohort of a batch).
struct MixedArgs {
    CohortMx c;   // the cohort of a single-cohort launch
    int R_e;      // linear rows (q + t)
    int N_e;      // UMMA N of the linear tile
    int stages;
    int n_units;
    int* err;
    int small_sums;  // every cohort of the launch has n 2^B < 2^22 (CohortMx::small_sums)
};

// Unit u -> (rt, ct) inside one cohort. Groups of `group` SNP tiles; inside a group the
// linear tile of every SNP tile comes first (when there is one), then row tiles from the
// heaviest down.
__device__ __forceinline__ void decode_unit(const CohortMx& c, int u, int& rt, int& ct) {
    const int levels = c.n_rt + c.extra;
    const int per_group = c.group * levels;
    const int g = u / per_group;
    const int w = u - g * per_group;
    const int ngroups = (c.n_ct + c.group - 1) / c.group;
    const int gsize = (g == ngroups - 1) ? c.n_ct - g * c.group : c.group;
    const int level = w / gsize;
    ct = g * c.group + (w - level * gsize);
    if (c.extra) rt = (level == 0) ? (int)mx::EXTRA : c.n_rt - level;
    else rt = c.n_rt - 1 - level;
}

__device__ __forceinline__ void record_error(int* err, volatile int* abort_flag, int code) {
    *abort_flag = 1;
    atomicCAS(err, 0, code);
}

// Where a unit's cohort and tensor maps come from: one cohort (maps as kernel
// parameters) or a table of cohorts in global memory (maps in global memory, three per
// cohort: dosages, limb row tiles, linear tile).
struct SrcOne {
    CUtensorMap tmX, tmW, tmE;
    MixedArgs a;
    __device__ __forceinline__ const CohortMx* locate(int u, int& ci, int& local, int&) const {
        ci = 0;
        local = u;
        return &a.c;
    }
    __device__ __forceinline__ const CUtensorMap* mapX(int) const { return &tmX; }
    __device__ __forceinline__ const CUtensorMap* mapB(int, bool ex) const { return ex ? &tmE : &tmW; }
};

struct SrcBatch {
    const CohortMx* tab;
    const CUtensorMap* maps;
    int n_cohorts;
    MixedArgs a;  // launch-wide fields; a.c unused
    // cur: the cohort of the caller's previous unit. A CTA role takes its units in
    // increasing order and the table's unit_base increases, so the cohort only moves
    // forward: one table read per unit instead of a binary search of dependent reads.
    __device__ __forceinline__ const CohortMx* locate(int u, int& ci, int& local, int& cur) const {
        int c = cur;
        while (c + 1 < n_cohorts && tab[c + 1].unit_base <= (int64_t)u) ++c;
        cur = c;
        ci = c;
        local = (int)(u - tab[c].unit_base);
        return &tab[c];
    }
    __device__ __forceinline__ const CUtensorMap* mapX(int ci) const { return maps + 3 * ci; }
    __device__ __forceinline__ const CUtensorMap* mapB(int ci, bool ex) const {
        return maps + 3 * ci + (ex ? 2 : 1);
    }
};

// An exact integer held in an FP32 accumulator as an int. With |v| < 2^22, v + 1.5 2^23
// lies in [2^23, 2^24), where the float spacing is 1, so the sum is exact and its low
// mantissa bits are v + 2^22: one add and one integer subtract instead of a conversion.
template <bool SMALL>
__device__ __forceinline__ int limb_int(uint32_t bits) {
    if (SMALL) return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
    return __float2int_rn(__uint_as_float(bits));
}

// Per-power sums of one 16-row group. With T_i = sum_l C_il 2^(B (S-1-l)),
// T_i^2 = sum_p P_ip 2^(B (2S-2-p)), P_ip = sum_{l+m=p} C_il C_im: the diagonal products
// C_il^2 go to dg[l] (power 2l), the cross products C_il C_im (l < m) to cr[l+m-1], each a
// 32 x 32 -> 64-bit multiply-add (|C_il| < 2^24, so every sum over a tile stays below
// R 2^49 < 2^57).
template <int S, bool SMALL>
__device__ __forceinline__ void sumsq_group(const uint32_t (&v)[S][16], int rows, long long (&dg)[S],
                                            long long (&cr)[2 * S - 3]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (i < rows) {
            int C[S];
#pragma unroll
            for (int l = 0; l < S; ++l) {
                const int col = i * S + l;
                C[l] = limb_int<SMALL>(v[col / 16][col % 16]);
            }
#pragma unroll
            for (int l = 0; l < S; ++l) {
                dg[l] += (long long)C[l] * C[l];
#pragma unroll
                for (int m2 = l + 1; m2 < S; ++m2) cr[l + m2 - 1] += (long long)C[l] * C[m2];
            }
        }
    }
}

// Rows 16 g .. 16 g + 15 of a row tile are the 16 S columns from 16 g S (a multiple of 16);
// a last, shorter group loads ceil(rows S / 16) x 16 columns, which end at or before column
// 256 because R S <= 256.
template <int S>
__device__ __forceinline__ void sumsq_load(uint32_t tb, int R, int g, uint32_t (&v)[S][16]) {
    const int rows = min(16, R - 16 * g);
    const int nld = (rows * S + 15) / 16;  // the same for every thread of the warp
#pragma unroll
    for (int q = 0; q < S; ++q)
        if (q < nld) tc::tmem_ld16(tb + (uint32_t)(16 * g * S + 16 * q), v[q]);
}

// Sum over the R rows of a row tile of T_i^2, the C_il being the S limb sums of row i in
// TMEM columns i S + l: the per-power sums of all rows, combined once in 128 bits
// (mod 2^128; the total is below 2^126, so it is exact). Up to 3 limbs the next 16-row
// group's TMEM loads are in flight while a group is summed.
template <int S, bool SMALL>
__device__ __forceinline__ unsigned __int128 tile_sumsq(uint32_t tb, int R, int B) {
    constexpr int G = (256 / S + 15) / 16;  // 16-row groups of the tallest tile
    long long dg[S], cr[2 * S - 3];
#pragma unroll
    for (int l = 0; l < S; ++l) dg[l] = 0;
#pragma unroll
    for (int p = 0; p < 2 * S - 3; ++p) cr[p] = 0;
    if constexpr (S <= 3) {
        uint32_t v[2][S][16];
        sumsq_load<S>(tb, R, 0, v[0]);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (16 * g < R) {
                tc::tmem_wait_ld();
                if (16 * (g + 1) < R) sumsq_load<S>(tb, R, g + 1, v[(g + 1) & 1]);
                sumsq_group<S, SMALL>(v[g & 1], min(16, R - 16 * g), dg, cr);
            }
        }
    } else {
#pragma unroll 1
        for (int g = 0; 16 * g < R; ++g) {
            uint32_t v[S][16];
            sumsq_load<S>(tb, R, g, v);
            tc::tmem_wait_ld();
            sumsq_group<S, SMALL>(v, min(16, R - 16 * g), dg, cr);
        }
    }
    unsigned __int128 acc = 0;
#pragma unroll
    for (int l = 0; l < S; ++l)
        acc += (unsigned __int128)(__int128)dg[l] << (B * (2 * S - 2 - 2 * l));
#pragma unroll
    for (int p = 1; p <= 2 * S - 3; ++p)
        acc += (unsigned __int128)(__int128)cr[p - 1] << (B * (2 * S - 2 - p) + 1);
    return acc;
}

// The linear reductions of one unit: R_e values T_j = sum_l C_lj 2^(B (S-1-l)) whose limb
// sums sit in TMEM columns col0 + j cj + l cl (limb-major: cj = 1, cl = R_e; rows side by
// side: cj = S, cl = 1), written as T_j 2^(E_j - shift0) to lin[(e0 + j) ldp + snp]. The
// loads of JB linear rows (JB S columns) are issued together and waited for once.
template <int S>
__device__ __forceinline__ void linear_rows(const CohortMx& a, int R_e, uint32_t col0, int cj,
                                            int cl, int64_t e0, int64_t snp) {
    using namespace tc;
    constexpr int JB = 8;
    const int B = a.radix;
    const long long base = 1ll << B;
    const int shift0 = (B - 1) + B * (S - 1);
#pragma unroll 1
    for (int j0 = 0; j0 < R_e; j0 += JB) {
        const int nj = min(JB, R_e - j0);  // the same for every thread of the warp
        uint32_t x[S][JB];
#pragma unroll
        for (int l = 0; l < S; ++l)
#pragma unroll
            for (int j = 0; j < JB; ++j)
                if (j < nj) tmem_ld1(col0 + (uint32_t)((j0 + j) * cj + l * cl), x[l][j]);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < JB; ++j) {
            if (j < nj) {
                long long T = 0;
#pragma unroll
                for (int l = 0; l < S; ++l)
                    T = T * base + (long long)__float2int_rn(__uint_as_float(x[l][j]));
                const int64_t e = e0 + j0 + j;
                if (snp < a.mb) a.lin[e * a.ldp + snp] = ldexp((double)T, a.E_e[e] - shift0);
            }
        }
    }
}

// Epilogue of one unit for the SNP held in TMEM lane `tb` (one thread = one SNP):
// row tiles -> sum over the tile's R rows of xbar^2, exact in 128-bit integers, plus (when
// the linear rows are fused) the tile's partial linear reductions from the fused columns;
// the linear tile -> the q + t linear reductions.
template <int S, bool SMALL>
__device__ __forceinline__ void epilogue_unit(const CohortMx& a, int R_e, uint32_t tb, int rt,
                                              int64_t snp) {
    using namespace tc;
    // x = 2^(E - shift0) T with T = sum_l C_l 2^(B (S-1-l)), B = a.radix bits per limb
    const int B = a.radix;
    const int shift0 = (B - 1) + B * (S - 1);
    const int R = a.R;
    if (rt != (int)mx::EXTRA) {
        // with the linear rows at the end of the last row tile, its last R_e rows are Z's
        const bool zrows = a.ztail && rt == a.n_rt - 1;
        const int R_w = zrows ? R - R_e : R;
        const unsigned __int128 acc = tile_sumsq<S, SMALL>(tb, R_w, B);
        const double hi = (double)(unsigned long long)(acc >> 64);
        const double lo = (double)(unsigned long long)acc;
        const double val = ldexp(fma(hi, 18446744073709551616.0, lo), 2 * (a.E_w[rt] - shift0));
        if (snp < a.mb) a.sq_part[(int64_t)rt * a.ldp + snp] = val;
        if (zrows) linear_rows<S>(a, R_e, tb + (uint32_t)(R_w * S), S, 1, 0, snp);
        // fused linear rows: Z limbs of this tile's k-range, one partial per (rt, j)
        else if (!a.extra && !a.ztail)
            linear_rows<S>(a, R_e, tb + (uint32_t)(R * S), 1, R_e, (int64_t)rt * R_e, snp);
    } else {
        linear_rows<S>(a, R_e, tb, 1, R_e, 0, snp);
    }
}

template <int S, class Src>
__global__ void __launch_bounds__(256, 1) k_block_mixed(const __grid_constant__ Src src) {
    using namespace tc;
    const MixedArgs& a = src.a;
    constexpr int N = mx::NT;  // UMMA N of a row tile (limb rows + fused linear rows)
    constexpr uint32_t A_BYTES = mx::BM * mx::BK * 2;
    const int NB = N > a.N_e ? N : a.N_e;
    const uint32_t B_BYTES = (uint32_t)NB * mx::BK * 2;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + a.stages * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + a.stages * B_BYTES);
    uint64_t* empty = full + a.stages;
    uint64_t* tfull = empty + a.stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* done = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], 4);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, 2 * mx::BUF);
        tmem_relinquish();
    }
    if (warp == 1 && lane == 0) {
        prefetch_tmap(src.mapX(0));
        prefetch_tmap(src.mapB(0, false));
        prefetch_tmap(src.mapB(0, true));
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    const int P = gridDim.x, me = blockIdx.x;
    const int rounds = (a.n_units + P - 1) / P;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int stage = 0;
        uint32_t phase = 0;
        uint32_t issued_parity[16];
        bool issued[16];
        for (int s = 0; s < 16; ++s) issued[s] = false;
        int cur = 0;  // cohort cursor (see SrcBatch::locate)
        for (int r = 0; r < rounds && !*abort_flag; ++r) {
            const int u = r * P + ((r & 1) ? (P - 1 - me) : me);
            if (u >= a.n_units) continue;
            int ci, lu, rt, ct;
            const CohortMx& cm = *src.locate(u, ci, lu, cur);
            decode_unit(cm, lu, rt, ct);
            const bool ex = (rt == (int)mx::EXTRA);
            const int nk = ex ? cm.n_kc_full : min(((rt + 1) * cm.R - cm.off + mx::BK - 1) / mx::BK, cm.n_kc_full);
            const int ybase = ex ? cm.n_rt * N : rt * N;
            const uint32_t bytes = A_BYTES + (uint32_t)(ex ? a.N_e : N) * mx::BK * 2;
            for (int kc = 0; kc < nk; ++kc) {
                if (!mbar_wait(&empty[stage], phase ^ 1, mx::WAIT_NS)) {
                    record_error(a.err, abort_flag, 1);
                    break;
                }
                mbar_arrive_expect_tx(&full[stage], bytes);
                tma_load_2d(sA + stage * A_BYTES, src.mapX(ci), kc * mx::BK,
                            (cm.ct_base + ct) * mx::BM,
                            &full[stage]);
                tma_load_2d(sB + stage * B_BYTES, src.mapB(ci, ex), kc * mx::BK, ybase,
                            &full[stage]);
                issued[stage] = true;
                issued_parity[stage] = phase;
                if (++stage == a.stages) {
                    stage = 0;
                    phase ^= 1;
                }
            }
        }
        if (*abort_flag) {
            // let copies already in flight land before the CTA's shared memory goes away
            for (int s = 0; s < a.stages && s < 16; ++s)
                if (issued[s]) mbar_wait(&full[s], issued_parity[s], 10000000ull);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        int stage = 0;
        uint32_t phase = 0;
        int abuf = 0;
        uint32_t aphase = 0;
        int cur = 0;  // cohort cursor (see SrcBatch::locate)
        for (int r = 0; r < rounds && !*abort_flag; ++r) {
            const int u = r * P + ((r & 1) ? (P - 1 - me) : me);
            if (u >= a.n_units) continue;
            int ci, lu, rt, ct;
            const CohortMx& cm = *src.locate(u, ci, lu, cur);
            decode_unit(cm, lu, rt, ct);
            const bool ex = (rt == (int)mx::EXTRA);
            const int nk = ex ? cm.n_kc_full : min(((rt + 1) * cm.R - cm.off + mx::BK - 1) / mx::BK, cm.n_kc_full);
            if (!mbar_wait(&tempty[abuf], aphase ^ 1, mx::WAIT_NS)) {
                record_error(a.err, abort_flag, 2);
                break;
            }
            fence_after_sync();
            const uint32_t d = tmem_base + (uint32_t)(abuf * mx::BUF);
            const uint32_t idesc = idesc_bf16_f32(mx::BM, ex ? a.N_e : N);
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc) {
                if (!mbar_wait(&full[stage], phase, mx::WAIT_NS)) {
                    record_error(a.err, abort_flag, 3);
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint64_t ad = smem_desc_sw128(smem_u32(sA + stage * A_BYTES));
                const uint64_t bd = smem_desc_sw128(smem_u32(sB + stage * B_BYTES));
#pragma unroll
                for (int kk = 0; kk < mx::BK / 16; ++kk)
                    umma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, (kc | kk) != 0);
                umma_commit(&empty[stage]);
                if (++stage == a.stages) {
                    stage = 0;
                    phase ^= 1;
                }
            }
            if (!ok) break;
            umma_commit(&tfull[abuf]);
            abuf ^= 1;
            if (abuf == 0) aphase ^= 1;
        }
        // every MMA issued by this thread has completed once `done` flips
        umma_commit(done);
        mbar_wait(done, 0, mx::WAIT_NS);
    } else if (warp >= 4) {
        // ---------------- epilogue: one SNP per thread ----------------
        // (one copy of the loop per conversion: a branch inside it would keep both live)
        auto role = [&](auto small) {
            constexpr bool SMALL = decltype(small)::value;
            const int qd = warp & 3;
            int abuf = 0;
            uint32_t aphase = 0;
            int cur = 0;  // cohort cursor (see SrcBatch::locate)
            for (int r = 0; r < rounds && !*abort_flag; ++r) {
                const int u = r * P + ((r & 1) ? (P - 1 - me) : me);
                if (u >= a.n_units) continue;
                int ci, lu, rt, ct;
                const CohortMx& cm = *src.locate(u, ci, lu, cur);
                decode_unit(cm, lu, rt, ct);
                if (!mbar_wait(&tfull[abuf], aphase, mx::WAIT_NS)) {
                    record_error(a.err, abort_flag, 4);
                    break;
                }
                fence_after_sync();
                const uint32_t tb =
                    tmem_base + (uint32_t)(abuf * mx::BUF) + ((uint32_t)(qd * 32) << 16);
                epilogue_unit<S, SMALL>(cm, a.R_e, tb, rt,
                                        (int64_t)(cm.ct_base + ct) * mx::BM + qd * 32 + lane);
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[abuf]);
                abuf ^= 1;
                if (abuf == 0) aphase ^= 1;
            }
        };
        if (a.small_sums) role(std::true_type{});
        else role(std::false_type{});
    }
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        fence_after_sync();
        tmem_dealloc(tmem_base, 2 * mx::BUF);
    }
}


// ----------------------------------------------------------------------------
// CTA-pair variant (cta_group::2): a cluster of 2 CTAs on one TPC computes a
// 256-SNP x N tile with M = 256 UMMAs. Each CTA loads its own 128 SNPs (A) and half of
// the limb tile (N/2 rows of B); the UMMA issued by the even CTA reads both halves, so
// every SM moves 28 KB instead of 40 KB per 64-k stage (3 limbs) and fits 7 stages.
// The even CTA's full barriers collect both CTAs' TMA bytes; its MMA commits arrive
// on the empty / accumulator barriers of both CTAs; both CTAs' epilogues release an
// accumulator buffer on the even CTA's barrier (8 warp arrivals).
// In this kernel a.n_ct counts pairs of 128-SNP tiles.
// ----------------------------------------------------------------------------
template <int S, class Src>
__global__ void __launch_bounds__(256, 1) k_block_mixed2(const __grid_constant__ Src src) {
    using namespace tc;
    const MixedArgs& a = src.a;
    constexpr int N = mx::NT;
    constexpr int NH = N / 2;
    constexpr uint32_t A_BYTES = mx::BM * mx::BK * 2;
    const int NeH = a.N_e / 2;
    const int NBH = NH > NeH ? NH : NeH;
    const uint32_t B_BYTES = (uint32_t)NBH * mx::BK * 2;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + a.stages * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + a.stages * B_BYTES);
    uint64_t* empty = full + a.stages;
    uint64_t* tfull = empty + a.stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* done = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t rank = cluster_ctarank();
    const bool leader = (rank == 0);
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], 8);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc2(tmem_slot, 2 * mx::BUF);
        tmem_relinquish2();
    }
    if (warp == 1 && lane == 0) {
        prefetch_tmap(src.mapX(0));
        prefetch_tmap(src.mapB(0, false));
        prefetch_tmap(src.mapB(0, true));
    }
    fence_before_sync();
    __syncthreads();
    cluster_sync();  // both CTAs' barriers initialised before any cross-CTA signal
    fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    const int P = gridDim.x / 2, me = blockIdx.x / 2;
    const int rounds = (a.n_units + P - 1) / P;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        int stage = 0;
        uint32_t phase = 0;
        uint32_t issued_parity[16];
        bool issued[16];
        for (int s = 0; s < 16; ++s) issued[s] = false;
        int cur = 0;  // cohort cursor (see SrcBatch::locate)
        for (int r = 0; r < rounds && !*abort_flag; ++r) {
            const int u = r * P + ((r & 1) ? (P - 1 - me) : me);
            if (u >= a.n_units) continue;
            int ci, lu, rt, ctp;
            const CohortMx& cm = *src.locate(u, ci, lu, cur);
            decode_unit(cm, lu, rt, ctp);
            const bool ex = (rt == (int)mx::EXTRA);
            const int nk = ex ? cm.n_kc_full : min(((rt + 1) * cm.R - cm.off + mx::BK - 1) / mx::BK, cm.n_kc_full);
            const int half = ex ? NeH : NH;
            const int ybase = (ex ? cm.n_rt * N : rt * N) + (int)rank * half;
            const int ct = cm.ct_base + 2 * ctp + (int)rank;
            const uint32_t pair_bytes = 2u * (A_BYTES + (uint32_t)half * mx::BK * 2);
            for (int kc = 0; kc < nk; ++kc) {
                if (!mbar_wait(&empty[stage], phase ^ 1, mx::WAIT_NS)) {
                    record_error(a.err, abort_flag, 11);
                    break;
                }
                if (leader) mbar_arrive_expect_tx(&full[stage], pair_bytes);
                const uint32_t fbar = mapa_shared(smem_u32(&full[stage]), 0);
                tma_load_2d_pair(sA + stage * A_BYTES, src.mapX(ci), kc * mx::BK, ct * mx::BM,
                                 fbar);
                tma_load_2d_pair(sB + stage * B_BYTES, src.mapB(ci, ex), kc * mx::BK, ybase, fbar);
                issued[stage] = true;
                issued_parity[stage] = phase;
                if (++stage == a.stages) {
                    stage = 0;
                    phase ^= 1;
                }
            }
        }
        if (*abort_flag && leader) {
            for (int s = 0; s < a.stages && s < 16; ++s)
                if (issued[s]) mbar_wait(&full[s], issued_parity[s], 10000000ull);
        }
    } else if (warp == 1 && lane == 0 && leader) {
        // ---------------- MMA issuer (even CTA) ----------------
        int stage = 0;
        uint32_t phase = 0;
        int abuf = 0;
        uint32_t aphase = 0;
        int cur = 0;  // cohort cursor (see SrcBatch::locate)
        for (int r = 0; r < rounds && !*abort_flag; ++r) {
            const int u = r * P + ((r & 1) ? (P - 1 - me) : me);
            if (u >= a.n_units) continue;
            int ci, lu, rt, ctp;
            const CohortMx& cm = *src.locate(u, ci, lu, cur);
            decode_unit(cm, lu, rt, ctp);
            const bool ex = (rt == (int)mx::EXTRA);
            const int nk = ex ? cm.n_kc_full : min(((rt + 1) * cm.R - cm.off + mx::BK - 1) / mx::BK, cm.n_kc_full);
            if (!mbar_wait(&tempty[abuf], aphase ^ 1, mx::WAIT_NS)) {
                record_error(a.err, abort_flag, 12);
                break;
            }
            fence_after_sync();
            const uint32_t d = tmem_base + (uint32_t)(abuf * mx::BUF);
            const uint32_t idesc = idesc_bf16_f32(2 * mx::BM, ex ? a.N_e : N);
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc) {
                if (!mbar_wait(&full[stage], phase, mx::WAIT_NS)) {
                    record_error(a.err, abort_flag, 13);
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint64_t ad = smem_desc_sw128(smem_u32(sA + stage * A_BYTES));
                const uint64_t bd = smem_desc_sw128(smem_u32(sB + stage * B_BYTES));
#pragma unroll
                for (int kk = 0; kk < mx::BK / 16; ++kk)
                    umma_bf16_pair(d, ad + 2 * kk, bd + 2 * kk, idesc, (kc | kk) != 0);
                umma_commit_pair(&empty[stage]);
                if (++stage == a.stages) {
                    stage = 0;
                    phase ^= 1;
                }
            }
            if (!ok) break;
            umma_commit_pair(&tfull[abuf]);
            abuf ^= 1;
            if (abuf == 0) aphase ^= 1;
        }
        umma_commit_pair(done);
        mbar_wait(done, 0, mx::WAIT_NS);
    } else if (warp >= 4) {
        // ---------------- epilogue (both CTAs): one SNP per thread ----------------
        // (one copy of the loop per conversion: a branch inside it would keep both live)
        auto role = [&](auto small) {
            constexpr bool SMALL = decltype(small)::value;
            const int qd = warp & 3;
            int abuf = 0;
            uint32_t aphase = 0;
            int cur = 0;  // cohort cursor (see SrcBatch::locate)
            for (int r = 0; r < rounds && !*abort_flag; ++r) {
                const int u = r * P + ((r & 1) ? (P - 1 - me) : me);
                if (u >= a.n_units) continue;
                int ci, lu, rt, ctp;
                const CohortMx& cm = *src.locate(u, ci, lu, cur);
                decode_unit(cm, lu, rt, ctp);
                if (!mbar_wait(&tfull[abuf], aphase, mx::WAIT_NS)) {
                    record_error(a.err, abort_flag, 14);
                    break;
                }
                fence_after_sync();
                const uint32_t tb =
                    tmem_base + (uint32_t)(abuf * mx::BUF) + ((uint32_t)(qd * 32) << 16);
                const int ct = cm.ct_base + 2 * ctp + (int)rank;
                epilogue_unit<S, SMALL>(cm, a.R_e, tb, rt, (int64_t)ct * mx::BM + qd * 32 + lane);
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(mapa_shared(smem_u32(&tempty[abuf]), 0));
                abuf ^= 1;
                if (abuf == 0) aphase ^= 1;
            }
        };
        if (a.small_sums) role(std::true_type{});
        else role(std::false_type{});
    }
    __syncthreads();
    cluster_sync();  // no CTA leaves while its peer may still signal it or use its TMEM
    if (warp == 0) {
        __syncwarp();
        fence_after_sync();
        tmem_dealloc2(tmem_base, 2 * mx::BUF);
    }
}

// ----------------------------------------------------------------------------
// Host side.
// ----------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool tmap_bf16_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer,
                  uint32_t box_inner, uint32_t box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Pipeline stages that fit the shared-memory budget for a tile of N = R*S limb rows
// (a CTA pair holds half of the limb tile per CTA).
int stage_count(int N, int N_e, bool pair) {
    const int NB = pair ? std::max(N, N_e) / 2 : std::max(N, N_e);
    const int per = mx::BM * mx::BK * 2 + NB * mx::BK * 2;
    return std::min(8, mx::SMEM_BUDGET / per);
}

size_t smem_bytes(int N, int N_e, bool pair, int stages) {
    const int NB = pair ? std::max(N, N_e) / 2 : std::max(N, N_e);
    return (size_t)stages * (mx::BM * mx::BK * 2 + NB * mx::BK * 2) + 1024 + 256;
}

}  // namespace

int mixed_radix(int64_t n) {
    for (int B = 9; B >= 7; --B)
        if (n < (int64_t(1) << (24 - B))) return B;
    return 0;
}

// UMMA N of the linear tile: a multiple of 32 (so each CTA of a pair holds whole
// 8-row swizzle groups of it) and at least 32.
int mixed_linear_n(int S, int R_e) { return (int)std::max<int64_t>(32, round_up((int64_t)S * R_e, 32)); }

cudaError_t mixed_layout(MixedDev& m, int64_t n, int S, int R_e, int64_t m_blk) {
    m.S = S;
    m.n = n;
    m.radix = mixed_radix(n);
    if (m.cfg_radix > 0 && 9 - m.cfg_radix < m.radix) m.radix = std::max(7, 9 - m.cfg_radix);
    // Tile height: as many rows as S limbs fit in N = 256. The S x R_e linear rows go to a
    // separate tile per SNP tile (N_e columns over every k), or, when asked (tile_cfg bit
    // 17) and at least 16 rows remain, ride in every row tile on its own k-range at the
    // cost of R_e fewer rows per tile.
    m.R_e = R_e;
    m.N_e = mixed_linear_n(S, R_e);
    const int r_fused = (mx::NT - S * R_e) / S;
    m.fused = m.cfg_fuse && r_fused >= 16;
    m.R = m.fused ? r_fused : mx::rows_max(S);
    // or (tile_cfg bit 21) the linear rows are R_e more rows after row n: they take the
    // last rows of the last row tile, which spans every k already (at most half a tile)
    m.ztail = !m.fused && m.cfg_ztail && 2 * R_e <= m.R;
    m.NT = mx::NT;
    m.pair = !m.cfg_single_cta;
    m.n_rt = (int)ceil_div(n + (m.ztail ? R_e : 0), m.R);
    m.n_pad = round_up(n, 64);
    m.rows_total = (int64_t)m.n_rt * m.NT + (m.fused || m.ztail ? 0 : m.N_e);
    m.mb_pad_max = round_up(m_blk, 2 * mx::BM);
    m.ldp = round_up(m_blk, 32);
    return cudaSuccess;
}

cudaError_t mixed_prepare(MixedDev& m, const double* W, int64_t ldw, const double* Z,
                          cudaStream_t s, int64_t* launches) {
    cudaError_t e = launch_limb_split(m, W, ldw, Z, s, launches);
    if (e != cudaSuccess) return e;
    // tensor maps over the fixed buffers
    const int N = m.NT;
    if (!tmap_bf16_2d(&m.tmX, m.Xb, (uint64_t)m.n_pad, (uint64_t)m.mb_pad_max, mx::BK, mx::BM) ||
        !tmap_bf16_2d(&m.tmW, m.WL, (uint64_t)m.n_pad, (uint64_t)m.rows_total, mx::BK, (uint32_t)N) ||
        !tmap_bf16_2d(&m.tmE, m.WL, (uint64_t)m.n_pad, (uint64_t)m.rows_total, mx::BK,
                      (uint32_t)m.N_e) ||
        !tmap_bf16_2d(&m.tmWh, m.WL, (uint64_t)m.n_pad, (uint64_t)m.rows_total, mx::BK,
                      (uint32_t)(N / 2)) ||
        !tmap_bf16_2d(&m.tmEh, m.WL, (uint64_t)m.n_pad, (uint64_t)m.rows_total, mx::BK,
                      (uint32_t)(m.N_e / 2)))
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

// The cohort constants of a launch over SNPs [snp0, mb) (snp0 a multiple of 256).
static CohortMx make_cohort(const MixedDev& m, int64_t mb, bool pair, int64_t snp0 = 0) {
    CohortMx c;
    c.n_rt = m.n_rt;
    c.n_ct = (int)ceil_div(mb - snp0, pair ? 2 * mx::BM : mx::BM);  // SNP tiles, or pairs
    c.ct_base = (int)(snp0 / mx::BM);
    c.n_kc_full = (int)(m.n_pad / mx::BK);
    const int64_t per_tile = (pair ? 2ll : 1ll) * mx::BM * m.n_pad * 2;  // BF16 dosages
    const int64_t budget = (int64_t)std::max(1, m.cfg_group_mb) << 20;
    c.group = (int)std::max<int64_t>(1, std::min<int64_t>(c.n_ct, budget / per_tile));
    c.mb = mb;
    c.ldp = m.ldp;
    c.unit_base = 0;
    c.extra = (m.fused || m.ztail) ? 0 : 1;
    c.ztail = m.ztail ? 1 : 0;
    c.radix = m.radix;
    c.small_sums = ((int64_t)m.n << m.radix) < (1ll << 22) ? 1 : 0;
    c.R = m.R;
    c.off = m.row_off();
    c.E_w = m.E;
    c.E_e = m.E + m.n_rt;
    c.sq_part = m.sq_part;
    c.lin = m.lin;
    return c;
}

static MixedArgs make_args(const MixedDev& m, int64_t mb, bool pair, int64_t snp0) {
    MixedArgs a;
    a.c = make_cohort(m, mb, pair, snp0);
    a.R_e = m.R_e;
    a.N_e = m.N_e;
    a.stages = stage_count(m.NT, m.N_e, pair);
    if (m.cfg_stages >= 2) a.stages = std::min(a.stages, m.cfg_stages);
    a.n_units = a.c.n_ct * (a.c.n_rt + a.c.extra);
    a.err = m.err;
    a.small_sums = a.c.small_sums;
    return a;
}

template <int S>
static cudaError_t launch_single_t(const MixedDev& m, int64_t mb, int64_t snp0, int num_sms,
                                   cudaStream_t s) {
    SrcOne src;
    src.tmX = m.tmX;
    src.tmW = m.tmW;
    src.tmE = m.tmE;
    src.a = make_args(m, mb, false, snp0);
    const size_t smem = smem_bytes(mx::NT, m.N_e, false, src.a.stages);
    cudaError_t e = cudaFuncSetAttribute(k_block_mixed<S, SrcOne>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(num_sms, src.a.n_units));
    k_block_mixed<S, SrcOne><<<grid, 256, smem, s>>>(src);
    return cudaGetLastError();
}

// Persistent launch of the CTA-pair kernel: clusters of 2 CTAs, as many as can be resident
// at once, at most one per unit.
template <class Src>
static cudaError_t launch_clusters(void (*kernel)(Src), const Src& src, size_t smem, int n_units,
                                   int num_sms, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // as many CTA pairs as can be resident at once (persistent), at most one per unit
    cfg.gridDim = dim3((unsigned)(2 * std::max(1, num_sms / 2)), 1, 1);
    int clusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorLaunchOutOfResources;
    clusters = std::min(clusters, std::max(1, num_sms / 2));
    clusters = std::min(clusters, n_units);
    cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
    e = cudaLaunchKernelEx(&cfg, kernel, src);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int S>
static cudaError_t launch_pair_t(const MixedDev& m, int64_t mb, int64_t snp0, int num_sms,
                                 cudaStream_t s) {
    static_assert(mx::NT % 32 == 0, "CTA pairs need N a multiple of 32");
    SrcOne src;
    src.tmX = m.tmX;
    src.tmW = m.tmWh;  // each CTA of a pair loads half of the limb tile
    src.tmE = m.tmEh;
    src.a = make_args(m, mb, true, snp0);
    const size_t smem = smem_bytes(mx::NT, m.N_e, true, src.a.stages);
    cudaError_t e = cudaFuncSetAttribute(k_block_mixed2<S, SrcOne>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_clusters(k_block_mixed2<S, SrcOne>, src, smem, src.a.n_units, num_sms, s);
}

// The limb counts a kernel is compiled for (the tile height is a run-time value).
#define GWAS_MIXED_LIMBS(X) X(2) X(3) X(4) X(5)

cudaError_t launch_block_mixed(const MixedDev& m, int64_t mb, int num_sms, cudaStream_t s,
                               int64_t snp0) {
    if (mb < 1 || mb > m.mb_pad_max || snp0 < 0 || snp0 >= mb || snp0 % (2 * mx::BM) != 0)
        return cudaErrorInvalidValue;
#define GWAS_TRY(SS)                                                          \
    if (m.S == SS)                                                            \
        return m.pair ? launch_pair_t<SS>(m, mb, snp0, num_sms, s)           \
                      : launch_single_t<SS>(m, mb, snp0, num_sms, s);
    GWAS_MIXED_LIMBS(GWAS_TRY)
#undef GWAS_TRY
    return cudaErrorInvalidValue;
}

bool mixed_shape_built(const MixedDev& m) {
#define GWAS_HAS(SS) \
    if (m.S == SS) return m.R >= 16 && m.R * SS + (m.fused ? SS * m.R_e : 0) <= mx::NT;
    GWAS_MIXED_LIMBS(GWAS_HAS)
#undef GWAS_HAS
    return false;
}

// ---- batched cohorts: one persistent launch over a device table of cohorts ----------

int mixed_stage_count(const MixedDev& m) {
    int st = stage_count(m.NT, m.N_e, m.pair);
    if (m.cfg_stages >= 2) st = std::min(st, m.cfg_stages);
    return st;
}

CohortMx mixed_cohort_entry(const MixedDev& m, int64_t mb, int64_t unit_base) {
    CohortMx c = make_cohort(m, mb, m.pair);
    c.unit_base = unit_base;
    return c;
}

int64_t mixed_cohort_units(const MixedDev& m, int64_t mb) {
    const CohortMx c = make_cohort(m, mb, m.pair);
    return (int64_t)c.n_ct * (c.n_rt + c.extra);
}

int64_t mixed_cohort_work(const MixedDev& m, int64_t mb) {
    const CohortMx c = make_cohort(m, mb, m.pair);
    int64_t chunks = 0;  // k-chunks of one SNP tile over its row tiles (as the kernel runs them)
    for (int rt = 0; rt < c.n_rt; ++rt)
        chunks += std::min<int64_t>(ceil_div((int64_t)(rt + 1) * c.R - c.off, mx::BK), c.n_kc_full);
    if (c.extra) chunks += ceil_div((int64_t)c.n_kc_full * m.N_e, mx::NT);
    return (int64_t)c.n_ct * chunks;
}

template <int S>
static cudaError_t batch_prepare_t(int N_e, int stages, bool pair) {
    const size_t smem = smem_bytes(mx::NT, N_e, pair, stages);
    if (pair)
        return cudaFuncSetAttribute(k_block_mixed2<S, SrcBatch>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaFuncSetAttribute(k_block_mixed<S, SrcBatch>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// One grouped launch over a table of cohorts. The map table holds three maps per cohort:
// dosages, limb row tiles, linear tile (half-height limb boxes for CTA pairs).
template <int S>
static cudaError_t batch_launch_t(const CohortMx* tab, const CUtensorMap* maps, int n_cohorts,
                                  int n_units, int R_e, int N_e, int stages, bool pair, int* err,
                                  bool small_sums, int num_sms, cudaStream_t s) {
    SrcBatch src;
    src.tab = tab;
    src.maps = maps;
    src.n_cohorts = n_cohorts;
    src.a = MixedArgs{};
    src.a.R_e = R_e;
    src.a.N_e = N_e;
    src.a.stages = stages;
    src.a.n_units = n_units;
    src.a.err = err;
    src.a.small_sums = small_sums ? 1 : 0;
    const size_t smem = smem_bytes(mx::NT, N_e, pair, stages);
    if (pair) return launch_clusters(k_block_mixed2<S, SrcBatch>, src, smem, n_units, num_sms, s);
    const int grid = std::max(1, std::min(num_sms, n_units));
    k_block_mixed<S, SrcBatch><<<grid, 256, smem, s>>>(src);
    return cudaGetLastError();
}

cudaError_t mixed_batch_prepare(const MixedDev& m, int stages) {
#define GWAS_TRY(SS) \
    if (m.S == SS) return batch_prepare_t<SS>(m.N_e, stages, m.pair);
    GWAS_MIXED_LIMBS(GWAS_TRY)
#undef GWAS_TRY
    return cudaErrorInvalidValue;
}

cudaError_t launch_block_mixed_batch(const CohortMx* tab, const CUtensorMap* maps, int n_cohorts,
                                     int64_t n_units, const MixedDev& m, int stages, int* err,
                                     bool small_sums, int num_sms, cudaStream_t s) {
    if (n_units <= 0) return cudaSuccess;
    if (n_units > 0x7fffffffLL) return cudaErrorInvalidValue;
#define GWAS_TRY(SS)                                                                     \
    if (m.S == SS)                                                                       \
        return batch_launch_t<SS>(tab, maps, n_cohorts, (int)n_units, m.R_e, m.N_e, stages, \
                                  m.pair, err, small_sums, num_sms, s);
    GWAS_MIXED_LIMBS(GWAS_TRY)
#undef GWAS_TRY
    return cudaErrorInvalidValue;
}

}  // namespace gwas
