// Host-side launchers of the engine's CUDA kernels (internal; not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gwas {

// ---- factor path (factor.cu) ------------------------------------------------

// M := sigma2 (h Phi + (1-h) I) from the lower triangle of Phi (is_phi), or a copy
// of the lower triangle of M; the strict upper triangle of the output is zeroed.
cudaError_t launch_build_M(const double* src, int64_t lds, double* M, int64_t ldm, int64_t n,
                           int is_phi, double h, double sigma2, cudaStream_t s);

// Blocked right-looking Cholesky of the lower triangle of A (n x n, col-major) in
// place, 64-wide blocks. Writes D_k = L_kk^{-1} of every diagonal block into Dinv
// (nt blocks of 64 x 64, col-major, zero padded) and the first non-positive pivot
// (global index) into *d_info (left untouched when the factorisation succeeds).
// Returns the number of kernels launched through *launches.
//
// With a lookahead stream (CholLookahead::panel non-null, created with a higher priority
// than s), each panel's factorisation and the update of the next panel's columns run on
// it, beside the update of the columns right of the next panel on s; the same tiles are
// computed in the same order as without it, so the factor is bitwise the same. s waits
// for the panel stream before the function returns.
struct CholLookahead {
    cudaStream_t panel = nullptr;
    cudaEvent_t ev[3] = {};  // start, panel factored, trailing update done
};
cudaError_t cholesky_blocked(double* A, int64_t lda, int64_t n, double* Dinv, int* d_info,
                             cudaStream_t s, int64_t* launches,
                             const CholLookahead* la = nullptr);

// W := L^{-1} (lower triangular, zeros above the diagonal) by the recursive block
// formula [[L11,0],[L21,L22]]^{-1} = [[W11,0],[-W22 L21 W11, W22]], with the
// diagonal 64 x 64 inverses taken from Dinv, evaluated level by level (two batched
// launches per level). tmp needs ceil(n/2/64)*64 squared doubles.
cudaError_t trtri_lower(const double* L, int64_t ldl, int64_t n, const double* Dinv, double* W,
                        int64_t ldw, double* tmp, cudaStream_t s, int64_t* launches);

// Generic FP64 GEMM: C := alpha op(A) op(B) + beta C, op(A) M x K, op(B) K x N.
struct GemmF64 {
    int64_t M = 0, N = 0, K = 0;
    const double* A = nullptr; int64_t lda = 0; bool transA = false;
    const double* B = nullptr; int64_t ldb = 0; bool transB = false;
    double* C = nullptr; int64_t ldc = 0;
    double alpha = 1.0, beta = 0.0;
    bool a_lower = false;  // op(A) square lower triangular: k runs to the row tile's end
    bool a_upper = false;  // op(A) square upper triangular: k starts at the row tile
    bool b_lower = false;  // op(B) square lower triangular: k starts at the column tile
    bool c_lower = false;  // compute only output tiles on or below the diagonal
};
cudaError_t gemm_f64(const GemmF64& g, cudaStream_t s);

// ---- per-block hot path (block_fp64.cu, snp_solve.cu) -------------------------

// Everything a block kernel needs about the cohort (device pointers).
struct CohortDev {
    int64_t n = 0;
    int q = 0;            // p - 1 fixed covariates
    int t = 0;            // phenotypes
    const double* W = nullptr;     // L^{-1}, n x n col-major, ld = ldw
    int64_t ldw = 0;
    const double* XLbar = nullptr; // n x q, ld = n
    const double* Ybar = nullptr;  // n x t, ld = n
    const double* S_TL = nullptr;  // q x q, ld = q
    const double* bbar_T = nullptr;// q x t, ld = q
    bool dense = false;            // W is a full (not lower-triangular) matrix
    // The all-ones SNP is collinear with X_L (decided once in FP64 by gwas_factor): a
    // SNP whose dosages are all equal (bad-flag bit 1, set by the mixed path's dosage
    // conversion) then gets status 1 without relying on the limb arithmetic's pivot.
    bool ones_singular = false;
};

// Per-SNP dosage flags (the `bad` arrays): bit 0 = a dosage outside {0,1,2} (status 2);
// bit 1 = every dosage equal (mixed path only).
constexpr uint8_t FLAG_BAD_DOSAGE = 1, FLAG_CONSTANT = 2;

// Number of per-SNP reduction values: q (S_BL) + 1 (S_BR) + t (bbar_B).
__host__ __device__ inline int n_red(const CohortDev& c) { return c.q + 1 + c.t; }

// FP64 path: for each (64-row tile r, 64-SNP tile) computes Xbar = W[r-tile, :] X
// and its row-tile partial sums of Xbar^T [Xbar_L | Xbar | Ybar] into
// part[(rt * nred + v) * ldp + snp]. Also writes bad[snp] (1 = dosage outside {0,1,2}).
cudaError_t launch_block_fp64(const CohortDev& c, const int8_t* X, int64_t ldx, int64_t mb,
                              double* part, int64_t ldp, uint8_t* bad, cudaStream_t s);

// Sums the n_tiles row-tile partials of every value of each SNP in a fixed order and
// writes the total over the first partial (row tile 0).
cudaError_t launch_reduce_fp64(const CohortDev& c, double* part, int64_t ldp, int n_tiles,
                               int64_t mb, cudaStream_t s);

// Reduces the row-tile partials (as launch_reduce_fp64: the totals replace row tile 0),
// assembles S_i and bbar_i (Algorithm 1), solves by p x p Cholesky, writes b, wald (may
// be null), status, and cov (may be null: mb x p x p, S_i^{-1} of every SNP).
cudaError_t launch_snp_solve(const CohortDev& c, double* part, int64_t ldp, int n_tiles,
                             const uint8_t* bad, int64_t mb, double* b, double* wald,
                             uint8_t* status, cudaStream_t s, double* cov = nullptr);

// ---- mixed-precision hot path (block_mixed.cu) ----------------------------------

// Per-cohort constants of a mixed launch (one entry per cohort of a batched launch).
struct CohortMx {
    int n_rt;           // row tiles of L^{-1}
    int n_ct;           // SNP tiles (of 128; of 256 in the CTA-pair kernel)
    int n_kc_full;      // k chunks covering n
    int group;          // SNP tiles per L2 group
    int64_t mb;         // SNPs
    int64_t ldp;        // leading dimension of sq_part / lin
    int64_t unit_base;  // first unit of this cohort in a batched launch
    int extra;          // 1: a separate linear tile per SNP tile; 0: linear rows fused
    int radix;          // bits per limb B: limbs in [-2^(B-1), 2^(B-1)]
    int R;              // rows of L^{-1} per row tile (limb i, l in column i*S + l)
    int off;            // n_rt R - n: row tile rt holds rows rt R - off .. (rt + 1) R - off
    int ct_base;        // first 128-SNP tile of the launch (its SNPs start at 128 ct_base)
    int small_sums;     // 1: n 2^B < 2^22, so every limb sum in TMEM is below 2^22
    int ztail;          // 1: the R_e linear rows are the last rows of the last row tile
    const int* E_w;     // exponent per row tile
    const int* E_e;     // exponent per linear row (fused: per (row tile, linear row))
    double* sq_part;    // [n_rt][ldp]
    double* lin;        // [R_e][ldp]; fused: [n_rt][R_e][ldp]
};

// Device buffers and tensor maps of the BF16-limb path for one cohort.
struct MixedDev {
    int S = 3;                  // BF16 limbs per element of L^{-1} and Z
    int radix = 9;              // bits per limb: 9 for n < 2^15, 8 for n < 2^16, 7 for n < 2^17
    int64_t n = 0;
    int R = 64;                 // rows of L^{-1} per tile (S R <= 256)
    int NT = 256;               // UMMA N of a row tile: its S R limb rows (row i's limbs
                                // side by side), fused linear rows, zero rows up to 256
    bool fused = false;         // linear rows ride in the spare N of every row tile
    bool ztail = false;         // linear rows are R_e extra rows at the end of the last row
                                // tile (over every k, one exponent each); no linear tile
    bool pair = true;           // CTA-pair kernel (cta_group::2) instead of one CTA per tile
    int n_rt = 0;               // R-row tiles of L^{-1}
    int64_t n_pad = 0;          // n rounded up to 64 (k extent of every BF16 row)
    int R_e = 0;                // linear rows q + t (Z = L^{-T} [Xbar_L | Ybar])
    int N_e = 0;                // UMMA N of the linear tile (S * R_e rounded up to 16)
    int64_t rows_total = 0;     // rows of WL: n_rt * NT (+ N_e for a separate linear tile)
    int64_t mb_pad_max = 0;     // rows of Xb
    int64_t ldp = 0;            // leading dimension of sq_part / lin
    uint16_t* WL = nullptr;     // BF16 limbs, [rows_total][n_pad], k contiguous
    unsigned long long* bits = nullptr;  // max |.| per row tile / linear row (FP64 bits)
    int* E = nullptr;           // exponents: n_rt row tiles, then the linear rows
    uint16_t* Xb = nullptr;     // BF16 dosages, [mb_pad_max][n_pad]
    double* sq_part = nullptr;  // [n_rt][ldp] row-tile partials of S_BRi
    double* lin = nullptr;      // [lin_tiles][R_e][ldp] S_BLi (q rows) then bbar_Bi (t rows)
    int* err = nullptr;         // kernel wait-timeout code (0 = none)
    int cfg_stages = 0;         // pipeline stages (0 = as many as fit)
    int cfg_group_mb = 40;      // MB of BF16 dosages per L2 group of SNP tiles
    bool cfg_single_cta = false;  // force one CTA per 128-SNP tile
    bool cfg_pair = false;        // force CTA pairs
    bool cfg_fuse = false;        // fuse the linear rows into the limb tiles (lower R)
    bool cfg_ztail = false;       // linear rows at the end of the last row tile (bit 21)
    int cfg_radix = 0;            // bits per limb at most 9 - cfg_radix (tile_cfg bits 15-16)
    int lin_tiles() const { return fused ? n_rt : 1; }
    // rows of padding before row 0: the row tiles end at row n (at row n + R_e with the
    // linear rows as the last rows), so the first is the short one
    int row_off() const { return (int)((int64_t)n_rt * R - n - (ztail ? R_e : 0)); }
    int n_exp() const { return n_rt + (fused ? n_rt * R_e : R_e); }
    CUtensorMap tmX, tmW, tmE;  // TMA maps of Xb, WL (row tiles), WL (linear tile)
    CUtensorMap tmWh, tmEh;     // the same WL maps with half-height boxes (CTA pairs)
};

int mixed_linear_n(int S, int R_e);
// Bits per limb B for n: the FP32 sums of n products |A_l x| <= 2^B stay below 2^24
// (exact) while n < 2^(24-B); 0 when n is too large for any supported B (>= 7).
int mixed_radix(int64_t n);
// true when a kernel for m's (S, R, NT, pair) layout is compiled in
bool mixed_shape_built(const MixedDev& m);
cudaError_t mixed_layout(MixedDev& m, int64_t n, int S, int R_e, int64_t m_blk);
// Exponents and BF16 limbs of W = L^{-1} (lower triangle) and Z (n x R_e) into m.WL / m.E
// (limbs.cu).
cudaError_t launch_limb_split(MixedDev& m, const double* W, int64_t ldw, const double* Z,
                              cudaStream_t s, int64_t* launches);
// launch_limb_split, then the tensor maps over m's buffers.
cudaError_t mixed_prepare(MixedDev& m, const double* W, int64_t ldw, const double* Z,
                          cudaStream_t s, int64_t* launches);
// Dosages of SNPs [snp0, mb) (n x mb int8, column-major) -> BF16 rows of m.Xb and their
// bad-dosage flags (limbs.cu).
cudaError_t launch_geno_bf16(const MixedDev& m, const int8_t* X, int64_t ldx, int64_t mb,
                             uint8_t* bad, cudaStream_t s, int64_t snp0 = 0);
// The tcgen05 kernel over SNPs [snp0, mb) (snp0 a multiple of 256): row-tile partials of
// S_BRi into m.sq_part, S_BLi / bbar_Bi into m.lin (columns snp0 .. mb-1).
cudaError_t launch_block_mixed(const MixedDev& m, int64_t mb, int num_sms, cudaStream_t s,
                               int64_t snp0 = 0);
// p x p solves of SNPs [snp0, mb) from the mixed partial layout (b, wald, status, cov and
// bad index SNPs of the whole block).
cudaError_t launch_snp_solve_mixed(const CohortDev& c, const MixedDev& m, const uint8_t* bad,
                                   int64_t mb, double* b, double* wald, uint8_t* status,
                                   cudaStream_t s, double* cov = nullptr, int64_t snp0 = 0);

// Batched cohorts: one grouped launch of the layout's kernel variant (CTA pairs over
// 256-SNP tiles, or one CTA per 128-SNP tile) over a device table of cohorts.
int mixed_stage_count(const MixedDev& m);
CohortMx mixed_cohort_entry(const MixedDev& m, int64_t mb, int64_t unit_base);
int64_t mixed_cohort_units(const MixedDev& m, int64_t mb);
// Tensor work of a cohort's units in full-width k-chunks (the linear tile at its width).
int64_t mixed_cohort_work(const MixedDev& m, int64_t mb);
cudaError_t mixed_batch_prepare(const MixedDev& m, int stages);
// small_sums: every cohort of the table has CohortMx::small_sums set (the faster exact
// conversion of the limb sums); otherwise all take the general one.
cudaError_t launch_block_mixed_batch(const CohortMx* tab, const CUtensorMap* maps, int n_cohorts,
                                     int64_t n_units, const MixedDev& m, int stages, int* err,
                                     bool small_sums, int num_sms, cudaStream_t s);

// ---- batched FP64 path, dosage conversion and p x p solves (batch.cu) ------------------

// One cohort of a batched FP64 / conversion / solve launch.
struct BatchJob {
    CohortDev c;
    const int8_t* X = nullptr;   // n x mb dosages (device), ld = n
    int64_t mb = 0;
    int64_t snp_base = 0;        // first SNP of this cohort in the batch's SNP numbering
    int64_t unit_base = 0;       // first FP64 unit of this cohort
    int n_rt64 = 0, n_ct64 = 0;  // FP64 tiles (64 rows, 64 SNPs)
    double* part = nullptr;      // FP64 partials [n_rt64][p+t][ldp]
    int64_t ldp = 0;
    uint8_t* bad = nullptr;
    uint16_t* Xb = nullptr;      // mixed: BF16 rows [mb_pad][n_pad]
    int64_t n_pad = 0;
    int convert = 1;             // mixed: 0 = Xb and bad are an earlier job's (same dosages)
    const double* sq_part = nullptr;  // mixed partials
    const double* lin = nullptr;
    int n_tiles_mx = 0;
    int lin_tiles = 1;
    double* b = nullptr;
    double* wald = nullptr;
    uint8_t* status = nullptr;
};

cudaError_t launch_block_fp64_batch(const BatchJob* jobs, int n_jobs, int64_t n_units,
                                    cudaStream_t s);
cudaError_t launch_geno_bf16_batch(const BatchJob* jobs, int n_jobs, int64_t n_snps,
                                   cudaStream_t s);
// p: the jobs' common q + 1; max_nred: the largest q + 1 + t over the jobs.
cudaError_t launch_snp_solve_batch(const BatchJob* jobs, int n_jobs, int64_t n_snps, int p,
                                   int max_nred, bool mixed, cudaStream_t s);

// ---- REML and db/dh (reml.cu) -----------------------------------------------------------

// Sum of log L_ii (ld = ldl) into *out (one block, fixed order).
cudaError_t launch_logdiag(const double* L, int64_t ldl, int64_t n, double* out, cudaStream_t s);
// out[0] = sum_ij A_ij B_ij, out[1] = sum_i A_ii for n x n column-major A, B (ld); the
// partial sums use part[0 .. 2*ceil(n/256)) and are added in a fixed order.
cudaError_t launch_frob_trace(const double* A, const double* B, int64_t ld, int64_t n,
                              double* part, double* out, cudaStream_t s);

// Inputs of the REML assembly (all device pointers; column-major, small).
struct RemlDev {
    int64_t n = 0;
    int q = 0, t = 0, j = 0;       // phenotype column j of Y
    double h = 0, sigma2 = 0;
    int profile = 0;               // 1: evaluate at the profiled sigma^2
    const double* S_TL = nullptr;  // q x q
    const double* bbar_T = nullptr;// q x t
    const double* G1 = nullptr;    // Zc^T Zc,      (q+t) x (q+t), Zc = M^-1 [X_L | Y]
    const double* G2 = nullptr;    // Zc^T Phi Zc (identity = 1: Zc^T [X_L | Y]), (q+t) x (q+t)
    const double* yy = nullptr;    // ybar_j^T ybar_j
    const double* logdet_M = nullptr;
    const double* frob = nullptr;  // [<M^-1, Phi>, tr M^-1] (identity = 1: [|L^-1|_F^2, *])
    // 1: Phi enters only through M = sigma2 (h Phi + (1-h) I), h > 0: Phi Zc =
    // ([X_L | Y] / sigma2 - (1-h) Zc) / h and <M^-1, Phi> = (n / sigma2 - (1-h) tr M^-1) / h
    // with tr M^-1 = |L^-1|_F^2, so neither Phi nor M^-1 is formed
    int identity = 0;
    double* out = nullptr;         // 8 doubles, see gwas_reml_result
};
cudaError_t launch_reml_assemble(const RemlDev& r, cudaStream_t s);

// db_i/dh from the forward partials (S_i, bbar_i) and the adjoint partials
// (g_iL = X_L^T M^-2 x_i, g_ii = |M^-1 x_i|^2, g_iy = Y^T M^-2 x_i), both in the FP64
// partial layout, and the Gram matrix G1 = Zc^T Zc. scale = sigma2 / h. part_fwd holds
// the totals in row tile 0 (left there by launch_snp_solve); part_adj is reduced here.
cudaError_t launch_dbdh(const CohortDev& c, const double* part_fwd, double* part_adj,
                        int64_t ldp, int n_tiles, const double* G1, double scale,
                        const uint8_t* bad, int64_t mb, double* dbdh, cudaStream_t s);

// ---- 2-bit packed genotypes (packed.cu) -------------------------------------------------
// Xp: mb columns of ceil(n/4) bytes (4 calls per byte, individual k in bits 2(k%4)..+1
// of byte k/4); call c becomes dosage code[c]. X: n x mb int8, ld = n.
cudaError_t launch_unpack_2bit(const uint8_t* Xp, int64_t n, int64_t mb, const int8_t code[4],
                               int8_t* X, cudaStream_t s);

// ---- utilities (util.cu) ---------------------------------------------------------------
cudaError_t launch_fill_dosages(int8_t* X, int64_t count, uint64_t seed, cudaStream_t s);

}  // namespace gwas
