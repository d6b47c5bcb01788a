/*
 * gwas.h -- C ABI of the GB300 mixed-model GWAS GLS engine.
 *
 * The engine solves, for every SNP i of a cohort of n individuals, the
 * generalized least-squares problem of Eq. (1) (Section 1):
 *
 *     b_i = (X_i^T M^{-1} X_i)^{-1} X_i^T M^{-1} y,   X_i = [X_L | x_i],
 *
 * with X_L the n x (p-1) fixed covariates shared by all SNPs, x_i the SNP's
 * n dosages, and M the n x n SPD covariance matrix. It follows the reduction of
 * Section 2 (Cholesky L L^T := M, Xbar := L^{-1} X, then a p x p Cholesky solve
 * of S_i b_i = bbar_i), with the i-independent work hoisted out of the SNP loop
 * as in Algorithm 1 (Section 2.1) and the SNPs streamed in blocks as in
 * Algorithm 2 (Section 3).
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major with leading dimension = number of rows.
 *   - Genotypes are int8 dosages in {0, 1, 2}, one SNP per column, so each SNP's
 *     n dosages are contiguous (the paper's blocks of contiguous vectors X_blk).
 *   - Outputs per block of mb SNPs and t phenotypes:
 *       b      double[mb * t * p], SNP-major: b[(i*t + j)*p + c] is coefficient c
 *              (c = p-1 is the SNP effect) of SNP i for phenotype j;
 *       wald   double[mb * t] or NULL: wald[i*t + j] = b_{i,p}^2 / (S_i^{-1})_{pp};
 *       status uint8_t[mb]: 0 ok, 1 singular S_i (b and wald set to NaN),
 *              2 a dosage outside {0,1,2} (b and wald set to NaN).
 *   - The caller owns every buffer it passes; the library owns all device memory
 *     it allocates (L, L^{-1}, Xbar_L, Ybar, device slots, scratch).
 *   - Every call returns a gwas_status; nothing aborts or throws across the ABI.
 *     gwas_last_error() describes the most recent failure of a context.
 *   - A context is bound to one CUDA device and is not thread-safe.
 *
 * Typical use (host buffers; error checks omitted):
 *
 *     gwas_opts o;  gwas_default_opts(&o);      // o.precision = GWAS_PREC_MIXED, ...
 *     gwas_ctx* ctx;  gwas_init(n, p, t, &o, &ctx);
 *     gwas_factor(ctx, Phi, 1, h, sigma2, XL, Y);    // once per cohort
 *     for (each block of mb <= o.m_blk SNPs)         // page-locked X for overlap
 *         gwas_solve_block(ctx, X_blk, mb, b_blk, wald_blk, status_blk);
 *     gwas_sync(ctx, -1);                            // all outputs are now in place
 *     gwas_finalize(ctx);
 */
#ifndef GWAS_GB300_H
#define GWAS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gwas_ctx gwas_ctx;     /* opaque: one cohort                      */
typedef struct gwas_batch gwas_batch; /* opaque: many cohorts solved together    */

typedef enum {
    GWAS_OK = 0,
    GWAS_ERR_ARG = 1,         /* invalid argument (size, NULL pointer, option)      */
    GWAS_ERR_NOT_SPD = 2,     /* M is not SPD; gwas_error_index() = failing pivot   */
    GWAS_ERR_CUDA = 3,        /* a CUDA runtime call failed                          */
    GWAS_ERR_OOM = 4,         /* device or pinned-host allocation failed             */
    GWAS_ERR_TIMEOUT = 5,     /* gwas_sync gave up waiting; work is still in flight  */
    GWAS_ERR_STATE = 6,       /* call out of order (e.g. solve before factor)        */
    GWAS_ERR_UNSUPPORTED = 7, /* option combination not built                        */
    GWAS_ERR_TOO_LARGE = 8    /* gwas_solve_block_noalloc: sizes exceed its scratch   */
} gwas_status;

typedef enum {
    GWAS_PREC_FP64 = 0,  /* every step in FP64                                        */
    GWAS_PREC_MIXED = 1  /* L^{-1} x_i on BF16 tensor cores as exact limb products,
                            everything else FP64                                      */
} gwas_precision;

typedef struct {
    int precision; /* gwas_precision                                                  */
    int m_blk;     /* largest block of SNPs one solve call may pass (device slot size) */
    int n_limbs;   /* GWAS_PREC_MIXED: BF16 limbs L^{-1} is split into (2..5); each adds
                      9 bits (8 for n >= 32768, 7 for n >= 65536): with 9-bit limbs 3
                      keep b within ~1e-8 of FP64, 5 within ~1e-13. n < 131072.        */
    int tile_cfg;  /* -1 = library default; for GWAS_PREC_MIXED, bits 0-3 = pipeline
                      stages (2..8, 0 = as many as fit), bits 4-11 = MB of BF16 dosages
                      per L2 group of SNP tiles (0 = 40), bit 12 = one CTA per 128-SNP
                      tile instead of CTA pairs (cta_group::2, the default), bit 13 =
                      CTA pairs, bit 17 = fuse the linear rows into the spare N of every
                      limb tile (fewer rows of L^{-1} per tile) instead of a separate
                      linear tile (the default; bit 14 also selects it and overrides
                      bit 17); bits 15-16 = r caps the bits per limb at 9 - r (the
                      default takes 9 bits for n < 32768, 8 for n < 65536, 7 for
                      n < 131072, the most for which the FP32 sums of limb products stay
                      exact); bits 18-20 (batches only) = the number of parts, 1..7, a
                      mixed batch's cohorts are split into (0 = 6; see gwas_batch_init);
                      bit 21 = the linear rows as R_e = q + t more rows at the end of the
                      last limb tile, which spans every k (no separate linear tile;
                      taken when R_e is at most half a tile and bit 17 is not set)      */
    int device;    /* CUDA device ordinal                                             */
    int timing;    /* 1 = record CUDA events around each dominant-kernel launch       */
    int use_graph; /* batches: 1 = capture the batched solve in a CUDA graph and
                      replay it while its pointers and sizes stay the same            */
} gwas_opts;

/* Per-context counters (gwas_get_stats). Times are CUDA-event milliseconds. */
typedef struct {
    int64_t blocks;            /* solve calls completed                               */
    int64_t snps;              /* SNPs solved                                         */
    int64_t kernel_launches;   /* kernels this library launched for solve calls      */
    int64_t trsm_launches;     /* launches of the dominant (L^{-1} X_blk) kernel      */
    double trsm_ms;            /* summed event time of those launches (timing = 1)    */
    int64_t h2d_bytes;         /* host->device bytes copied by solve calls            */
    int64_t d2h_bytes;         /* device->host bytes copied by solve calls            */
    double factor_ms;          /* event time of the last gwas_factor                  */
    int64_t factor_launches;   /* kernels launched by the last gwas_factor            */
    double factor_upload_ms;   /* of factor_ms: the copies of Phi (or M), X_L and Y   */
} gwas_stats;

/* Result of gwas_autotune. */
typedef struct {
    int tile_cfg;        /* fastest tile configuration (see gwas_opts.tile_cfg)          */
    int64_t m_blk;       /* SNPs per block at which it was fastest                       */
    double ms_per_snp;   /* device time per SNP of the whole block path at that setting  */
    double snps_per_s;
    int candidates;      /* (tile_cfg, block size) pairs timed                            */
} gwas_tune;

/* Result of gwas_reml (REML of the null model y = X_L beta + e, e ~ N(0, M)). */
typedef struct {
    double loglik;      /* l = -1/2[(n-q) log 2pi + log|M| + log|X_L^T M^-1 X_L| + y^T P y]  */
    double dl_dh;       /* dl/dh at (h, sigma2)                                           */
    double dl_dsigma2;  /* dl/dsigma2 at (h, sigma2)                                      */
    double sigma2_hat;  /* sigma2 maximising l at this h: sigma2 y^T P y / (n - q)         */
    double yPy;         /* y^T P y                                                        */
    double logdet_M;    /* log|M|                                                         */
    double logdet_A;    /* log|X_L^T M^-1 X_L|                                            */
    double sigma2;      /* the sigma2 the values refer to (sigma2_hat when profiled)      */
} gwas_reml_result;

/* Fill *opts with defaults: FP64, m_blk 16384, 3 limbs, default tiles, device 0,
 * no timing events, CUDA graphs on. */
void gwas_default_opts(gwas_opts* opts);

/*
 * Create a context for n individuals, p columns per design matrix (p-1 fixed
 * covariates + 1 SNP; 2 <= p <= 20, Section 1) and t phenotype columns sharing
 * one M (1 <= t <= 64). Allocates every device buffer up front; sizes:
 * about 2 n^2 doubles (L and L^{-1}) plus the SNP slots (2 * n * m_blk bytes)
 * plus O(n (p + t)) and O(m_blk (p + t) n / 64) scratch doubles.
 * Errors: GWAS_ERR_ARG, GWAS_ERR_CUDA, GWAS_ERR_OOM. *out is NULL on failure.
 */
gwas_status gwas_init(int64_t n, int p, int t, const gwas_opts* opts, gwas_ctx** out);

/*
 * Per-cohort setup, Algorithm 1 before its loop (Section 2.1):
 *   M := sigma2 * (h * Phi + (1 - h) * I)   if is_phi != 0 (M_or_Phi holds Phi),
 *   M := M_or_Phi                           otherwise;
 *   L L^T := M (FP64 Cholesky), L^{-1} formed explicitly in FP64,
 *   Xbar_L := L^{-1} X_L, Ybar := L^{-1} Y,
 *   S_TL := Xbar_L^T Xbar_L, bbar_T := Xbar_L^T Ybar.
 * M_or_Phi: n x n column-major (only the lower triangle is read); XL: n x (p-1);
 * Y: n x t. Each pointer may be host or device memory (any address the CUDA
 * runtime can copy from). Blocks until the setup is complete.
 * Errors: GWAS_ERR_NOT_SPD (gwas_error_index() = first non-positive pivot),
 * GWAS_ERR_ARG (NULL pointer, 0 <= h <= 1 and sigma2 > 0 violated with is_phi),
 * GWAS_ERR_CUDA.
 */
gwas_status gwas_factor(gwas_ctx* ctx, const double* M_or_Phi, int is_phi, double h,
                        double sigma2, const double* XL, const double* Y);

/*
 * One block of Algorithm 2's loop (Section 3): copy X (n x mb int8, HOST memory,
 * pinned for full overlap) into a device slot, compute Xbar_blk := L^{-1} X_blk
 * fused with the per-SNP reductions S_BLi, S_BRi, bbar_Bi and the p x p solve,
 * and copy b, wald (may be NULL) and status back into the caller's HOST buffers.
 * Asynchronous: returns once the work is queued. Two slots alternate, so the
 * copy of one block overlaps the compute of the previous one. The caller must not
 * modify X nor read b/wald/status before gwas_sync() returns GWAS_OK.
 * 1 <= mb <= m_blk. Errors: GWAS_ERR_ARG, GWAS_ERR_STATE (no factor), GWAS_ERR_CUDA.
 */
gwas_status gwas_solve_block(gwas_ctx* ctx, const int8_t* X, int64_t mb, double* b,
                             double* wald, uint8_t* status);

/*
 * As gwas_solve_block with every pointer in DEVICE memory of the context's device
 * (no copies). X must stay valid and unmodified, and the outputs unread, until the
 * work completes (gwas_sync, or stream order on gwas_stream()).
 */
gwas_status gwas_solve_block_device(gwas_ctx* ctx, const int8_t* X, int64_t mb, double* b,
                                    double* wald, uint8_t* status);

/*
 * As gwas_solve_block_device, and also S_i^{-1} = (X_i^T M^{-1} X_i)^{-1} of every SNP into
 * cov (DEVICE, mb x p x p float64, SNP-major, each matrix column-major and written in
 * full; NaN unless status is 0). S_i^{-1} is the covariance of b_i (sigma^2 is inside M):
 * the p x p matrix generated beside b_i (Section 3); wald = b_ip^2 / (S_i^{-1})_pp. It is
 * formed from the same p x p Cholesky factor as b_i. Errors as gwas_solve_block_device,
 * GWAS_ERR_ARG for a NULL cov.
 */
gwas_status gwas_solve_block_cov_device(gwas_ctx* ctx, const int8_t* X, int64_t mb, double* b,
                                        double* wald, uint8_t* status, double* cov);

/*
 * 2-bit packed genotype calls (the paper streams FP64 genotypes; this packs four calls
 * per byte, so a block's host -> device copy is n/4 bytes per SNP instead of n). Xp
 * holds mb SNP columns of ceil(n/4) bytes each; individual k of a column sits in bits
 * 2(k%4) and 2(k%4)+1 of byte k/4 (the unused bits of a column's last byte are
 * ignored). A call c in {0,1,2,3} stands for dosage code[c]; a code outside {0,1,2}
 * marks a missing or invalid call and gives the SNP status 2 with NaN outputs, like a
 * bad int8 dosage (e.g. {0,1,2,-1} for calls that are dosages, or {2,-1,1,0} for a
 * SNP-major PLINK .bed block with the dosage of its first allele). code: host array of
 * 4 int8, read during the call. The calls are unpacked on the GPU into the int8 layout
 * of gwas_solve_block, after which everything is identical, so results equal those of
 * gwas_solve_block on the unpacked dosages bit for bit.
 * gwas_solve_block_packed: Xp and the outputs in HOST memory, asynchronous and double
 * buffered as gwas_solve_block. gwas_solve_block_packed_device: every pointer in DEVICE
 * memory, ordered on gwas_stream() as gwas_solve_block_device; the unpacked block goes to
 * a device buffer of n x m_blk bytes allocated on first use.
 * Errors: GWAS_ERR_ARG (NULL pointer or code, mb out of 1..m_blk), GWAS_ERR_STATE (no
 * factor), GWAS_ERR_OOM, GWAS_ERR_CUDA.
 */
gwas_status gwas_solve_block_packed(gwas_ctx* ctx, const uint8_t* Xp, int64_t mb,
                                    const int8_t* code, double* b, double* wald,
                                    uint8_t* status);
gwas_status gwas_solve_block_packed_device(gwas_ctx* ctx, const uint8_t* Xp, int64_t mb,
                                           const int8_t* code, double* b, double* wald,
                                           uint8_t* status);

/*
 * Algorithm 2 end to end on host memory: m SNPs (n x m int8, column-major) in
 * blocks of m_blk, double-buffered, then gwas_sync(-1). Outputs as above with m
 * in place of mb. Errors as gwas_solve_block.
 */
gwas_status gwas_solve_all(gwas_ctx* ctx, const int8_t* X, int64_t m, double* b,
                           double* wald, uint8_t* status);

/*
 * Wait until host-path block number `block` (0-based count of the gwas_solve_block and
 * gwas_solve_block_packed calls made on this context) has completed: its input buffer may
 * be reused and its b / wald / status read. A streaming caller can recycle its pinned host
 * buffers this way while later blocks are in flight (Algorithm 2's double buffering).
 * timeout_ms < 0 waits without limit. Errors: GWAS_ERR_ARG (no such block yet),
 * GWAS_ERR_TIMEOUT, GWAS_ERR_CUDA.
 */
gwas_status gwas_wait_block(gwas_ctx* ctx, int64_t block, int timeout_ms);

/* Page-locked host memory for streaming buffers (cudaHostAlloc, portable); *out = NULL
 * for bytes = 0. gwas_host_free(NULL) is allowed. Errors: GWAS_ERR_ARG, GWAS_ERR_OOM
 * (alloc), GWAS_ERR_CUDA (free). */
gwas_status gwas_host_alloc(size_t bytes, void** out);
gwas_status gwas_host_free(void* p);

/*
 * Wait for all queued work of the context. timeout_ms < 0 waits without limit;
 * otherwise polls and returns GWAS_ERR_TIMEOUT after about timeout_ms (the work
 * stays queued and a later gwas_sync may still succeed). Never hangs the host
 * when a limit is given.
 */
gwas_status gwas_sync(gwas_ctx* ctx, int timeout_ms);

/* Free every resource of the context; ctx is invalid afterwards. NULL is allowed. */
gwas_status gwas_finalize(gwas_ctx* ctx);

/* Text of the last error of ctx ("" if none); owned by ctx. */
const char* gwas_last_error(const gwas_ctx* ctx);

/* Failing pivot index after GWAS_ERR_NOT_SPD, else -1. */
int64_t gwas_error_index(const gwas_ctx* ctx);

/* Counters since gwas_init or the last gwas_reset_stats (waits for queued work). */
gwas_status gwas_get_stats(gwas_ctx* ctx, gwas_stats* out);
gwas_status gwas_reset_stats(gwas_ctx* ctx);

/* The context's compute stream, as a cudaStream_t cast to void*. */
void* gwas_stream(const gwas_ctx* ctx);

/*
 * REML log-likelihood of phenotype column `pheno` and its gradient with respect to h and
 * sigma2, for M = sigma2 (h Phi + (1 - h) I). The paper takes M as given (Section 1);
 * this is the standard variance-component likelihood behind it, with its hand-derived
 * adjoint: the derivative of l with respect to M is -1/2 (P - P y y^T P), P =
 * M^-1 - M^-1 X_L (X_L^T M^-1 X_L)^-1 X_L^T M^-1, contracted with dM/dh = sigma2 (Phi - I)
 * and dM/dsigma2 = M / sigma2. Runs gwas_factor(ctx, Phi, 1, h, sigma2, XL, Y) first, then
 * the small Gram matrices of Z = M^-1 [X_L | Y] on the GPU. For h >= 1e-2 the traces
 * use Phi = (M / sigma2 - (1 - h) I) / h and tr M^-1 = |L^-1|_F^2 (no n x n product
 * beyond the factor); below it M^-1 = L^-T L^-1 is formed and Phi read directly.
 * Phi: the FULL n x n symmetric matrix (both triangles are read), host or device. With
 * profile != 0 every value is reported at sigma2 = sigma2_hat(h) (so dl/dh is the
 * derivative of the profiled likelihood). Afterwards the context is ready for
 * gwas_solve_block_grad_device at this (h, sigma2). Synchronous.
 * Errors: as gwas_factor; GWAS_ERR_ARG (pheno out of range).
 */
gwas_status gwas_reml(gwas_ctx* ctx, const double* Phi, double h, double sigma2, const double* XL,
                      const double* Y, int pheno, int profile, gwas_reml_result* out);

/*
 * gwas_solve_block_device plus db_i/dh for every SNP and phenotype: differentiating the
 * normal equations of Eq. (1) in h gives db_i/dh = (sigma2/h) S_i^-1 X_i^T M^-2 r_i with
 * r_i = y - X_i b_i (h > 0). The per-SNP products M^-1 x_i are recomputed from the
 * dosages by a second pass of the FP64 block kernel with M^-1 in place of L^-1.
 * dbdh: DEVICE double[mb * t * p], laid out like b (NaN where status != 0).
 * Needs a GWAS_PREC_FP64 context and a preceding gwas_reml (h > 0).
 * Errors: GWAS_ERR_STATE, GWAS_ERR_UNSUPPORTED (mixed context), GWAS_ERR_ARG, GWAS_ERR_CUDA.
 */
gwas_status gwas_solve_block_grad_device(gwas_ctx* ctx, const int8_t* X, int64_t mb, double* b,
                                         double* wald, uint8_t* status, double* dbdh);

/*
 * Change the kernel tile configuration of a context (see gwas_opts.tile_cfg). For a
 * GWAS_PREC_MIXED context whose limb tile height changes, the BF16 limbs are re-split
 * from the FP64 L^{-1} kept by gwas_factor (no new factorisation). Synchronises the
 * context. Errors: GWAS_ERR_ARG, GWAS_ERR_CUDA, GWAS_ERR_OOM, GWAS_ERR_UNSUPPORTED (no kernel
 * is built for the layout the bits select; the previous configuration stays).
 */
gwas_status gwas_set_tile_cfg(gwas_ctx* ctx, int tile_cfg);

/*
 * Autotuner: on a factored context, time the whole block path (dosage conversion,
 * dominant kernel, p x p solves) for every candidate tile configuration (mixed: one
 * CTA or CTA pairs, fused or separate linear rows, pipeline stages, L2 group size) and
 * block size (4096, 8192, 16384 and mb_max SNPs, up to m_blk) with CUDA events, `reps`
 * launches each; time the four fastest again (three interleaved rounds of 2 x reps
 * launches, best round each); keep the fastest of those on the context and report it
 * in *out. X: n x mb_max DEVICE
 * dosages to time with, or NULL for synthetic ones (timing does not depend on the
 * values). Allocates temporary device memory; synchronises the context; does not add
 * to the context's counters. Errors: GWAS_ERR_STATE (no factor), GWAS_ERR_CUDA.
 */
gwas_status gwas_autotune(gwas_ctx* ctx, const int8_t* X, int64_t mb_max, int reps,
                          gwas_tune* out);

/* ---------------------------------------------------------------------------------
 * Batches of cohorts. Many independent cohorts (each its own n, M, X_L and Y with t
 * phenotype columns; the same p, t and options for all) are solved together: every
 * cohort is factored once (as gwas_factor), and one batched solve runs ONE grouped
 * launch of the block kernel over all cohorts' work units, so cohorts of uneven n
 * share the GPU without a launch per cohort. With opts.use_graph the launches of a
 * batched solve are captured once into a CUDA graph and replayed while the pointers
 * and sizes passed in stay the same. This is Eq. (1) for each (cohort, SNP, phenotype);
 * several phenotypes sharing one M are the one-M case of the multi-trait problem in
 * the paper's outlook (Section 5).
 * --------------------------------------------------------------------------------- */

/* Create a batch of n_cohorts contexts with sizes n[c] (host array). opts->m_blk is the
 * largest number of SNPs per cohort in one batched solve. Every cohort takes
 * opts->tile_cfg: GWAS_PREC_MIXED batches run the CTA-pair kernel variant unless bit 12
 * forces one CTA per 128-SNP tile. A mixed batch of several cohorts is solved in parts
 * (contiguous cohort ranges of about equal work, tile_cfg bits 18-20, default 6) on two
 * streams, each part's dosage conversion beside the previous part's block kernel.
 * Errors as gwas_init. */
gwas_status gwas_batch_init(int n_cohorts, const int64_t* n, int p, int t, const gwas_opts* opts,
                            gwas_batch** out);

/* gwas_factor for cohort `cohort` of the batch (same arguments and errors). */
gwas_status gwas_batch_factor(gwas_batch* b, int cohort, const double* M_or_Phi, int is_phi,
                              double h, double sigma2, const double* XL, const double* Y);

/* One batched solve. X, mb, b, wald, status are HOST arrays with one entry per cohort;
 * the entries X[c] (n[c] x mb[c] int8 dosages), b[c], wald[c] (may be NULL, or wald
 * itself NULL), status[c] are DEVICE pointers laid out as in gwas_solve_block_device.
 * 1 <= mb[c] <= m_blk. Asynchronous on gwas_batch_stream(); the device tables behind
 * the launch are rebuilt (synchronously) when the pointers or sizes change.
 * Errors: GWAS_ERR_ARG, GWAS_ERR_STATE (a cohort not factored), GWAS_ERR_CUDA. */
gwas_status gwas_batch_solve_device(gwas_batch* b, const int8_t* const* X, const int64_t* mb,
                                    double* const* bo, double* const* wald,
                                    uint8_t* const* status);

/* Wait for the batch's queued work (timeout_ms < 0: no limit; else GWAS_ERR_TIMEOUT). */
gwas_status gwas_batch_sync(gwas_batch* b, int timeout_ms);

/* Counters summed over the batch's solves (factor_* summed over cohorts). */
gwas_status gwas_batch_get_stats(gwas_batch* b, gwas_stats* out);
gwas_status gwas_batch_reset_stats(gwas_batch* b);

/* Free the batch and every cohort context in it. NULL is allowed. */
gwas_status gwas_batch_finalize(gwas_batch* b);

/* Text of the batch's last error ("" if none). */
const char* gwas_batch_last_error(const gwas_batch* b);

/* The batch's stream, as a cudaStream_t cast to void*. */
void* gwas_batch_stream(const gwas_batch* b);

/*
 * Self-test of the bounded waits used by the pipeline kernels (the paper has no
 * counterpart): one GPU thread waits on an mbarrier phase that never completes, with a
 * limit of timeout_ms (1..10000). Returns GWAS_ERR_TIMEOUT when the wait gave up as it
 * must (the expected outcome; *waited_ms = device time spent waiting), GWAS_OK if it
 * completed, GWAS_ERR_CUDA/GWAS_ERR_ARG otherwise. The device stays usable afterwards.
 */
gwas_status gwas_selftest_wait(int device, int timeout_ms, double* waited_ms);

/*
 * Measured FP64 multiply-add rate of a device (the paper has no counterpart): the
 * roofline denominator of the FP64 block kernel, which is bound by the FP64 FMA pipe.
 * Times the block kernel's FP64 inner loop on shared-memory operands alone (256 threads
 * per CTA, each a 4 x 4 register tile of fma over 16-deep chunks; 2, 4 and 8 CTAs per
 * SM, ~0.12 s per launch, best of two launches after a warm-up) and returns the best
 * rate in *tflops (2 flops per fma). Synchronous, about 1.2 s; allocates a few hundred
 * kB of device memory. Errors: GWAS_ERR_ARG (NULL tflops), GWAS_ERR_CUDA.
 */
gwas_status gwas_fp64_fma_rate(int device, double* tflops);

/*
 * Allocation-free FP64 block solve. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they call in -- their
 * GPU memory is already fully reserved by another allocator (a framework's caching
 * allocator, or a fixed per-process budget), or they run a latency-sensitive serving
 * loop in which cudaMalloc/cudaFree, which may synchronise the device, are not
 * acceptable. It allocates nothing and needs no context: it runs the FP64 block
 * kernels of gwas_solve_block_device on the caller's buffers, and their scratch lives
 * in one fixed 16 MiB array in device global memory that belongs to the library image
 * (every GPU that loads the library holds it until the process exits).
 *
 * Everything is DEVICE memory of the CURRENT device, column-major:
 *   Linv    n x n lower-triangular L^{-1} with zeros above the diagonal, ld = ld_linv >= n;
 *   XLbar   n x (p-1) = L^{-1} X_L;  Ybar n x t = L^{-1} Y  (ld = n);
 *   S_TL    (p-1) x (p-1) = XLbar^T XLbar;  bbar_T (p-1) x t = XLbar^T Ybar;
 *   X       n x mb int8 dosages;  b, wald (may be NULL), status as in gwas_solve_block.
 * Runs on `stream` (a cudaStream_t; NULL = the default stream) and returns once the
 * work is queued; the caller synchronises.
 * Scratch limit: ceil(n/64) * (p+t) * round_up(mb,32) * 8 bytes, rounded up to 256,
 * plus round_up(mb,256) must not exceed 16 MiB (16,777,216 bytes); otherwise the call
 * returns GWAS_ERR_TOO_LARGE before launching anything (at n = 10,000, p = 4, t = 1 that
 * is about 2,600 SNPs per call). The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream
 * capture. All calls share the one array and it keeps the last call's contents
 * (nothing in it needs to start at zero): calls that overlap on the GPU -- on
 * different streams, or from different threads -- race on it and must be serialised
 * by the caller. Before launching, the call checks (cudaPointerGetAttributes, which
 * allocates nothing) that the first and last byte of every buffer lie in device or
 * managed memory of the current device; host memory, another device's memory or an
 * unknown address is GWAS_ERR_ARG. Errors: GWAS_ERR_ARG, GWAS_ERR_TOO_LARGE, GWAS_ERR_CUDA.
 */
gwas_status gwas_solve_block_noalloc(int64_t n, int p, int t, const double* Linv,
                                     int64_t ld_linv, const double* XLbar, const double* Ybar,
                                     const double* S_TL, const double* bbar_T, const int8_t* X,
                                     int64_t mb, double* b, double* wald, uint8_t* status,
                                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GWAS_GB300_H */
