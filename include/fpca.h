/*
 * fpca.h -- C ABI of the GB300 (sm_103a) binned local linear FPCA smoother.
 *
 * The library estimates the mean mu(t) and the 2d-dimensional covariance
 * surface Gamma(s,t) of functional data observed on a d-dimensional domain
 * (Chen & Jiang, "Multi-dimensional Functional Principal Component
 * Analysis"): binning (Section 3.2), the local linear smoothers Eq. (2.3) and
 * Eq. (2.4), matrixisation (Section 3.1, Eq. 3.1) and the random-projection
 * eigendecomposition (Section 3.4).
 *
 * Conventions (every entry point)
 *  - Array arguments are DEVICE pointers allocated and owned by the caller,
 *    unless the comment says "host".  The library never frees them.
 *  - Work is queued on the context's CUDA stream and returns before it
 *    finishes; results are valid after fpca_sync() or a later stream sync.
 *  - Argument checks are synchronous: a bad argument returns
 *    FPCA_E_INVALID_ARG (or FPCA_E_UNSUPPORTED for a valid but unbuilt
 *    combination) with a message in fpca_last_error(); nothing is launched.
 *  - Device-side failures (a bounded wait that ran out, a CUDA launch
 *    error) are recorded in a device error word and returned by the next
 *    fpca_sync(): FPCA_E_TIMEOUT or FPCA_E_CUDA.
 *  - Nothing aborts, exits or throws across this interface.
 *  - A singular local system is not an error: it is reported per output
 *    point in a status array (FPCA_PT_*).
 *
 * Grid: d in {1,2,3}; bins [k/M, (k+1)/M) per axis (last bin closed),
 * centres (k + 1/2)/M, flattened in C order (axis 0 slowest).  P = prod M_k.
 * The covariance grid is P x P, row = s, column = t.
 */
#ifndef FPCA_H
#define FPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FPCA_OK = 0,
  FPCA_E_INVALID_ARG = 1,
  FPCA_E_UNSUPPORTED = 2,
  FPCA_E_CUDA = 3,
  FPCA_E_OOM = 4,
  FPCA_E_TIMEOUT = 5,
  FPCA_E_NUMERIC = 6
} fpca_status;

/* Arithmetic of a stage.
 *  F64   FP64 throughout (CUDA cores).
 *  F32   FP32 moment sums, FP32 local solve; a point whose FP32 pivot ratio
 *        falls below 1e-2 is solved again in float-float arithmetic (pairs of
 *        FP32 numbers, about 48 significant bits).
 *  F32C  as F32 with Kahan-compensated moment sums.
 *  BF16  binning products on tcgen05 tensor cores, BF16 operands, FP32
 *        accumulation in tensor memory; pair counts stay exact integers. */
typedef enum { FPCA_F64 = 0, FPCA_F32 = 1, FPCA_BF16 = 2, FPCA_F32C = 4 } fpca_prec;

/* Per-point status of a local fit (uint8 arrays). */
enum { FPCA_PT_OK = 0, FPCA_PT_FALLBACK = 1, FPCA_PT_EMPTY = 2 };

/* Data layouts. */
enum { FPCA_DENSE = 0, FPCA_SPARSE = 1 };
/* Covariance responses: residual products R R with R = Y - mu_hat
 * (Gamma_hat = b0), or raw products Y Y as printed in Eq. (2.4)
 * (Gamma_hat = b0 - mu_hat(s) mu_hat(t)). */
enum { FPCA_COV_RESIDUAL = 0, FPCA_COV_RAW = 1 };

typedef struct {
  int d;      /* 1..3 */
  int m[3];   /* bins per axis (entries beyond d ignored) */
} fpca_grid;

/* Observations, Eq. (2.2): Y_ij = X_i(t_ij) + eps_ij.
 *  Dense (functional data on the grid nodes): y is n x P row-major, FP64
 *    (y_prec = FPCA_F64) or FP32 (FPCA_F32); mask is n x P uint8 (1 =
 *    observed) or NULL for fully observed data.
 *  Sparse (longitudinal data): subject i owns observations
 *    offs[i] .. offs[i+1]-1; t is N x d FP64 locations in [0,1]^d, y is N
 *    FP64 values.  Locations are binned by floor(t M) clamped to M-1. */
typedef struct {
  int layout;              /* FPCA_DENSE or FPCA_SPARSE */
  int n;                   /* subjects */
  const void* y;
  int y_prec;
  const uint8_t* mask;     /* dense only, may be NULL */
  const int64_t* offs;     /* sparse only: n + 1 entries */
  const double* t;         /* sparse only: N x d */
} fpca_data;

/* Covariance bins of Eq. (2.4), fold-major: F = max(nfold, 1) slices of
 * P x P, slice f holding the pairs of subjects in fold f.  Element type of
 * w, v, q: double when prec == FPCA_F64, float otherwise. */
typedef struct {
  int nfold;
  int prec;
  const int32_t* cnt;      /* F x P x P pair counts, exact */
  const void* w;           /* sum of subject weights 1/(N_i(N_i-1)) */
  const void* v;           /* sum of weighted response products */
  const void* q;           /* sum of weighted squared products (CV), or NULL */
  int asym;                /* 0: cnt, w, v, q are symmetric in (s, t), as fpca_bin_cov
                              makes them, and the smoother may evaluate t >= s only
                              and mirror; nonzero: arbitrary bins, every pair fitted */
} fpca_covbins;

typedef struct fpca_ctx fpca_ctx;

/* Context: binds a device and a stream (NULL = the legacy default stream)
 * and owns a workspace that grows on demand.  Returns FPCA_E_CUDA if the
 * device cannot be used and FPCA_E_UNSUPPORTED if it is not sm_103. */
fpca_status fpca_create(fpca_ctx** ctx, int device, void* cuda_stream);
void fpca_destroy(fpca_ctx* ctx);
fpca_status fpca_set_stream(fpca_ctx* ctx, void* cuda_stream);
/* Text of the last error on this context ("" if none); owned by ctx. */
const char* fpca_last_error(const fpca_ctx* ctx);
/* Waits for the stream and returns the first recorded device-side error. */
fpca_status fpca_sync(fpca_ctx* ctx);
/* Number of kernels this context has launched so far (host counter). */
uint64_t fpca_launch_count(const fpca_ctx* ctx);

/* Arithmetic-throughput probe: launches `blocks` blocks of 256 threads that
 * each run 8 independent FMA chains for 16 * iters rounds (fp64 = 0: paired FP32
 * FMAs, two per instruction; fp64 != 0: FP64 FMAs) and writes to *flops (host)
 * the floating-point operations the launch performs (2 per FMA).  The caller
 * times the launch on the context's stream (CUDA events) to measure the FP32 or
 * FP64 FMA peak of the device; with blocks a few times the SM count the FMA pipes,
 * not latency, bind. */
fpca_status fpca_alu_probe(fpca_ctx* ctx, int fp64, int blocks, int iters, double* flops);

/* Choice of the t-side moment sweep of the FP32 d = 2 covariance smoother
 * (fpca_smooth_cov_project with FPCA_F32 / FPCA_F32C):
 *  0  automatic (default): the candidates built for the grid and windows are
 *     timed once per (grid, windows, precision) on the context's stream and the
 *     fastest is remembered in the context;
 *  1  the scalar sweep (every t-plane layout and window);
 *  2  the packed-pair sweep where it is built (t-planes 32 or 64 wide, the
 *     same window on both t axes), else the scalar one.
 * All choices compute the same sums in the same order per output up to the
 * grouping of the FP32 partial sums, within the stated FP32 tolerance. */
fpca_status fpca_set_sweep_kernel(fpca_ctx* ctx, int kernel);

/* Schedule of the K-fold CV grid of the FP32 d = 2 covariance smoother
 * (fpca_smooth_cov_project with cv != NULL, fold bins, symmetric bins, no raw
 * mean, t-planes 8, 16, 32 or 64 wide).
 *  0  item by item: each (bandwidth, fold) item's t-side runs right after its
 *     s-side, with the sweep kernel fpca_set_sweep_kernel selects;
 *  1  batched: the s-side passes of every item run first, each into arrays of
 *     its own (40 P^2 bytes per item in the context's workspace), then ONE
 *     persistent launch of the scalar t-side sweep takes the tiles of all items
 *     from a shared counter and scores each against its held-out fold;
 *  2  automatic (default): on the first call for a (grid, folds, precision,
 *     number of bandwidths, and whether the widest window's tile leaves room
 *     for two batched CTAs per SM), the two schedules are timed on the
 *     context's stream (after one untimed item-by-item pass) and the faster is
 *     remembered in the context.
 * Batched falls back to item by item when the items' arrays do not fit in 80%
 * of the free device memory, when the widest window's tile exceeds the shared
 * memory, or when sweep kernel 2 is forced.  Both compute the same fits and CV
 * terms (the same sums per point, FP32 tolerance). */
fpca_status fpca_set_cv_batch(fpca_ctx* ctx, int batch);

/* Self-check of the device-side failure detection.  Launches one thread
 * that waits on an on-chip barrier (an mbarrier expecting one arrival) with
 * the bounded wait every waiting kernel of this library uses.  arrive != 0:
 * the barrier is completed first and the next fpca_sync() returns FPCA_OK.
 * arrive == 0: nothing completes it, the wait gives up after its limit
 * (about 2 s of GPU time) and the next fpca_sync() returns FPCA_E_TIMEOUT;
 * the kernel exits normally, so the context and the GPU stay usable and
 * the following fpca_sync() returns FPCA_OK again. */
fpca_status fpca_check_wait(fpca_ctx* ctx, int arrive);

/* CUDA graphs of call sequences.  fpca_graph_begin starts capturing the
 * context's stream (which must be a created stream, not the legacy default
 * stream; kernel timing must be off); the calls that follow are recorded, not
 * run; fpca_graph_end closes the capture and returns an instantiated graph that
 * fpca_graph_launch replays on the context's stream with the same device
 * pointers and scalars (the caller keeps the buffers alive and rewrites their
 * contents between launches).  Calls that read results back to the host, grow
 * the workspace, time an autotuner's candidates or copy from host memory cannot
 * be captured: they return FPCA_E_UNSUPPORTED, and fpca_graph_end then returns
 * FPCA_E_UNSUPPORTED without a graph.  So run a sequence once before capturing
 * it (the workspace grows and the autotuners decide on that first run).
 * fpca_graph_launches gives the number of kernels in a graph (added to the
 * context's launch count at every launch).  Argument errors during capture are
 * reported as outside it; device errors surface at fpca_sync after a launch. */
typedef struct fpca_graph fpca_graph;
fpca_status fpca_graph_begin(fpca_ctx* ctx);
fpca_status fpca_graph_end(fpca_ctx* ctx, fpca_graph** graph);
fpca_status fpca_graph_launch(fpca_ctx* ctx, const fpca_graph* graph);
uint64_t fpca_graph_launches(const fpca_graph* graph);
void fpca_graph_destroy(fpca_graph* graph);

/* Kernel timing (off by default).  When enabled, a CUDA event is recorded on
 * the context stream at the start of every entry point and after every
 * kernel launch; a kernel's time is the interval between its event and the
 * previous one (so a stream memset or host gap before a kernel is counted
 * with it).  fpca_profile_enable clears the totals.  fpca_profile_count
 * waits for the stream, folds finished intervals into per-kernel-name totals
 * and returns the number of names; fpca_profile_entry reads entry i (name
 * owned by ctx, valid until the next fpca_profile_count). */
fpca_status fpca_profile_enable(fpca_ctx* ctx, int enable);
int fpca_profile_count(fpca_ctx* ctx);
fpca_status fpca_profile_entry(fpca_ctx* ctx, int i, const char** name, double* total_ms,
                               uint64_t* launches);

/* Mean bins with the 1/N_i weights of Eq. (2.3) (Section 3.2 binning).
 * Outputs (length P each): cnt = observations per bin (exact);
 * w = sum_i n_ib / N_i; v = sum_i sum_{j in b} Y_ij / N_i;
 * v2 = sum_i sum_{j in b} Y_ij^2 / N_i (may be NULL).  Subjects with
 * N_i = 0 are skipped. */
fpca_status fpca_bin_mean(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                          int32_t* cnt, double* w, double* v, double* v2);

/* Local linear mean, Eq. (2.3), at every bin centre from the mean bins, with
 * the product Epanechnikov kernel and bandwidths h[0..d-1] (host).  The
 * kernel's support is |c - x| < h per axis; a point whose window holds
 * fewer than d+1 non-empty bins, or whose normal matrix has a Cholesky pivot
 * at most 1e-9 of its diagonal (natural variable order), gets the local
 * constant fit and FPCA_PT_FALLBACK; a window without weight gets NaN and
 * FPCA_PT_EMPTY.  FP64 throughout.  mu, status: length P. */
fpca_status fpca_smooth_mean(fpca_ctx* ctx, const fpca_grid* grid, const int32_t* cnt,
                             const double* w, const double* v, const double* h,
                             double* mu, uint8_t* status);

/* Cross-validation score of the mean smoother, Eq. (2.3) (Section 3.3
 * selects bandwidths by cross-validation), for nh bandwidth vectors h (host,
 * nh x d): subjects are split into nfold folds by fold[i] (device int32,
 * length n, values 0..nfold-1); for fold f the mean is fitted on the mean bins
 * of the other folds and scored on fold f's observations at their bin centres
 * with the weights 1/N_i: sum (1/N_i)(Y_ij - mu_hat(c))^2 over held-out
 * observations whose fit is not EMPTY, divided by their weight sum; +inf when
 * EMPTY fits hold more than 1% of the held-out weight.  Scattered data only
 * (FPCA_SPARSE; gridded data can be listed as points at the node centres);
 * FP64 throughout.  cv: nh device doubles out. */
fpca_status fpca_smooth_mean_cv(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                                const int32_t* fold, int nfold, const double* h, int nh,
                                double* cv);

/* Covariance bins of Eq. (2.4) over ordered pairs j != l of one subject,
 * subject weight 1/(N_i(N_i - 1)) (subjects with N_i < 2 skipped).
 *  mu: the fitted mean at the bin centres (length P, FP64).
 *  mode: FPCA_COV_RESIDUAL (products of Y - mu) or FPCA_COV_RAW (Y Y).
 *  Dense data: C = M'M, W = M' diag(w) M, V = R' diag(w) R with the p == q
 *   entries (only j == l pairs) set to zero.  prec FPCA_F64 uses FP64
 *   CUDA-core products (w, v double); FPCA_BF16 uses tcgen05 tensor cores
 *   with BF16 operands and FP32 accumulation (w, v float); counts are exact
 *   for n < 2^24.  FPCA_F32 uses FP32 CUDA-core products (w, v, q float; the
 *   terms w_i R R and their sums rounded to FP32) and is the one dense
 *   precision that takes fold/nfold and q, with the meaning they have for
 *   sparse data; FPCA_F64 and FPCA_BF16 need fold = NULL, nfold = 0, q = NULL.
 *  Sparse data: integer-exact pair scatter; FPCA_F64 or FPCA_F32 sums.
 *   fold (length n, values 0..nfold-1) splits the pairs into nfold slices;
 *   q (may be NULL) receives sum w (R R)^2 for cross-validation.
 * cnt, w, v, q are F x P x P (F = max(nfold, 1)) and are overwritten. */
fpca_status fpca_bin_cov(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                         const double* mu, int prec, int mode,
                         const int32_t* fold, int nfold,
                         int32_t* cnt, void* w, void* v, void* q);

/* Local linear covariance surface, Eq. (2.4), at every pair of bin centres,
 * for nh bandwidths h (host, nh x d), and what the eigen step needs from it.
 * Built for d <= 2 and m[k] <= 64 (the P x P surface is materialised); d = 3
 * grids return FPCA_E_UNSUPPORTED here and use the factored entry points
 * (fpca_bin_cov_factor, fpca_smooth_cov_apply) instead.
 *  bins: from fpca_bin_cov; all folds are pooled for the fit.
 *  prec: FPCA_F64, FPCA_F32 or FPCA_F32C (see fpca_prec).
 *  mu_raw: for raw-mode bins, the fitted mean (Gamma_hat = b0 - mu mu);
 *   NULL for residual-mode bins (Gamma_hat = b0).
 *  gamma (optional): nh x P x P, double for FPCA_F64 else float; NaN where
 *   EMPTY, the local constant fit where FALLBACK.
 *  status (optional): nh x P x P uint8, rules as in fpca_smooth_mean with
 *   2d+1 unknowns.
 *  omega/l/y (optional, all or none): y = G Omega, nh x P x l float, with
 *   G = Gamma_hat (EMPTY points counted as zero; no symmetrisation and no
 *   domain mask), omega P x l float, l <= 64 -- the first product of the
 *   random projection (Section 3.4) taken while each row of Gamma_hat is
 *   still on chip.
 *  cv (optional, bins->nfold >= 2, bins->q given, residual mode): nh
 *   doubles, the subject-level K-fold CV score of each bandwidth: for fold f
 *   the surface is fitted on the pooled bins minus fold f's bins and scored
 *   on fold f's held-out products at the bin centres, sum (Q_f - 2 G V_f +
 *   G^2 W_f) over non-EMPTY points divided by their held-out weight; +inf
 *   when EMPTY points hold more than 1% of the held-out weight
 *   (Section 3.3 selects bandwidths by cross-validation).
 * At least one output must be given. */
fpca_status fpca_smooth_cov_project(fpca_ctx* ctx, const fpca_grid* grid,
                                    const fpca_covbins* bins, const double* h, int nh,
                                    int prec, const double* mu_raw,
                                    const float* omega, int l,
                                    void* gamma, uint8_t* status, float* y, double* cv);

/* Eigenpairs of the matrixised covariance (Section 3.1, Eq. 3.1):
 * Sigma = (G + G')/2 with NaN entries and rows/columns outside the domain
 * set to zero; lambda = theta dV, phi = psi / sqrt(dV), dV = 1/P; each
 * eigenvector's largest-magnitude entry made positive; FVE_k =
 * sum_{j<=k} lambda_j / (trace(Sigma) dV).
 *  gamma: P x P, double (gamma_prec FPCA_F64) or float (FPCA_F32).
 *  domain: P int32 mean-bin counts from fpca_bin_mean (a node is inside
 *   Omega when its count is > 0), or NULL for the whole box.
 *  full = 1: all eigenpairs of Sigma itself (gamma FP64, P <= 1024), of which the
 *   leading k are returned: two-sided block Jacobi in FP32 (blocks of 16 indices,
 *   each round's block pairs diagonalised side by side, the rotations applied
 *   across the GPU), then three Ogita-Aishima refinement steps in FP64 on the
 *   FP64 matrix (each squares the error: eigenpairs to about FP64 accuracy).
 *  full = 0: random projection (Section 3.4) with the caller's Gaussian
 *   test matrix omega (P x l float, k < l <= 64): Y = Sigma Omega, power_iters
 *   rounds of Q = orth(Y), Y = Sigma Q, then Q = orth(Y), B = Q' Sigma Q and
 *   the eigenpairs of B (Rayleigh-Ritz): FP32 Jacobi refined by two
 *   Ogita-Aishima steps (float-float, about 1e-14, for l <= 32; FP64 beyond).
 *   The products Sigma X are FP32 with the partial sums of the k ranges
 *   added in a fixed order (the result does not depend on scheduling).
 *   orth is Cholesky QR (one pass between power iterations, two at the end)
 *   on a compensated FP32 Gram matrix with the Cholesky factor and its
 *   inverse in float-float (about 48 bits).
 * Outputs (device, FP64): evals k, evecs P x k (column-major: vector j at
 * evecs + j*P), fve k (may be NULL). */
fpca_status fpca_rproj_eig(fpca_ctx* ctx, const fpca_grid* grid, const void* gamma,
                           int gamma_prec, const int32_t* domain,
                           const float* omega, int l, int k, int power_iters, int full,
                           double* evals, double* evecs, double* fve);

/* Learned bandwidth proposal.  Section 3.3 selects bandwidths by
 * cross-validation over candidates and calls grid search expensive; this
 * network maps a 32-number summary of a dataset's bins (fpca_bw_features)
 * to the CV-optimal log bandwidths [log h_mu (3), log h_Gamma (3)], so that
 * one smoothing pass plus a CV check can replace the grid.
 * Architecture 32 -> 256 -> 256 -> 256 -> 6, exact GELU after each hidden
 * layer; weights used in FP16 (rounded from the FP32 master copy), FP32
 * accumulation.  Parameter vector (device float, fpca_bw_param_count()
 * entries): for each layer W (fan_in x fan_out, row-major) then b. */
int64_t fpca_bw_param_count(void);
/* Initial parameters (device float, fpca_bw_param_count() entries): every
 * weight of a layer with fan_in inputs drawn from N(0, 2 / fan_in) (He
 * initialisation), biases zero.  The draws come from a counter-based generator
 * (splitmix64 of (seed, parameter index), Box-Muller), so the same seed gives
 * the same parameters on any device and any stream. */
fpca_status fpca_bw_mlp_init(fpca_ctx* ctx, uint64_t seed, float* params);
/* Save (save != 0) or load the trained network to or from the file `path`
 * (host string): the parameter vector and, when the pointers are not NULL,
 * the 32 feature means and 32 feature scales used to standardise the input
 * (device float arrays; on save a NULL pointer writes zeros, on load a NULL
 * pointer skips them).  The file holds an 8-byte tag, the parameter count and
 * the values in the byte order of the host.  Loading a file of another
 * layout returns FPCA_E_INVALID_ARG and leaves the arrays unchanged.
 * Synchronises the context's stream. */
fpca_status fpca_bw_mlp_io(fpca_ctx* ctx, float* params, float* feat_mu, float* feat_sd,
                           const char* path, int save);
/* out (B x 6) = network(feat (B x 32)); all device float. */
fpca_status fpca_bw_predict(fpca_ctx* ctx, const float* params, const float* feat, int B,
                            float* out);
/* One training step on a batch: loss = sum m (out - target)^2 / sum m over
 * the B x 6 entries with tmask (uint8) set; the gradient of the loss by
 * manual backward; if step >= 1, one AdamW update (beta 0.9/0.999, eps
 * 1e-8, bias correction for update number `step`, decoupled weight decay wd)
 * of params with moments adam_m, adam_v (device float, zero initially).
 * step = 0 computes loss and gradient only.  loss (device float) and
 * grad_out (param_count floats) may be NULL. */
fpca_status fpca_bw_train_step(fpca_ctx* ctx, float* params, float* adam_m, float* adam_v,
                               int step, const float* feat, const float* target,
                               const uint8_t* tmask, int B, float lr, float wd, float* loss,
                               float* grad_out);

/* The network's input: 32 summary numbers of one dataset (device float
 * feat[32]) from its observations (for the per-subject counts N_i), its mean
 * bins (cnt, w, v, v2 as produced by fpca_bin_mean; v2 may be NULL) and its
 * covariance bins (fold slices are pooled).  Features, in order: d; log n; log
 * mean N_i; std/mean N_i; log min N_i; log max N_i; log(1 + mean bin count);
 * var/mean^2 and skewness of bin counts; fraction of empty bins; log mean
 * within-bin variance v2/w - (v/w)^2; log variance of the binned mean v/w;
 * log mean squared 2nd difference of v/w along axes 0..2 and 1st difference
 * along axes 0..1, relative to that variance; 0; log roughness of the
 * covariance raw means V/W along s_1 and along the (s_1, t_1) diagonal,
 * relative to their variance; log(1 + mean pair count); fraction of
 * covariance bins with a pair; log 1/M_k (k < d); zeros.  Non-empty means
 * w > 0; sums in FP64. */
fpca_status fpca_bw_features(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                             const int32_t* cnt, const double* w, const double* v,
                             const double* v2, const fpca_covbins* bins, float* feat);

/* Mean bins of gridded data without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- code whose device memory is owned by another
 * allocator (a framework's caching pool or a fixed arena), code running
 * where allocation is not allowed, or hosts that forbid libraries from
 * allocating behind their back.  It needs no fpca_ctx (creating one
 * allocates) and computes the mean bins of fpca_bin_mean for FPCA_DENSE data,
 * on the given stream (NULL = legacy default stream) of the current device:
 * the counts are bit-identical; w, v and v2 are the same sums added in another
 * order (one FP64 chain per bin instead of float-float slices and an FP64
 * tree), so they agree to about 1e-13 relative, not bit for bit.
 *
 *  y: n x P row-major, FP64 (y_prec FPCA_F64) or FP32 (FPCA_F32); mask: n x P
 *  uint8 or NULL; outputs cnt, w, v (and v2 unless NULL) of length P.  All
 *  are caller-owned device pointers.
 *
 * Scratch: the per-subject counts N_i live in a file-scope __device__ array
 * of 2^20 int32 (4 MiB) that every GPU loading the library holds until the
 * process exits.  n > 2^20 returns FPCA_E_UNSUPPORTED without launching.
 * Each call overwrites entries 0..n-1 before reading them, so nothing needs
 * to start at zero; all calls share the array, so calls that overlap on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.  The first call on a device looks up the array's device address
 * with that device current (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The address is remembered with the unique id of
 * the device's context and looked up again when that changes (after a
 * cudaDeviceReset, the first call after it does the lookup again and should
 * likewise come before any capture).  Errors: FPCA_E_INVALID_ARG for bad
 * arguments, FPCA_E_CUDA for a failed lookup or launch. */
fpca_status fpca_bin_mean_static(void* cuda_stream, int n, int P, const void* y, int y_prec,
                                 const uint8_t* mask, int32_t* cnt, double* w, double* v,
                                 double* v2);

/* ---- trust-region bandwidth search (Section 3.3) ----------------------------
 *
 * Section 3.3 replaces the grid search by a derivative-free trust-region
 * method (Marazzi and Nocedal) whose local quadratic model is fitted by
 * least-squares regression, since the CV score is noisy.  Built for d <= 2 on
 * the CV of fpca_smooth_cov_project (bins with nfold >= 2 and q; prec as
 * there).  The reading of each step (variables log h, box trust region, 3^d
 * sample stencil, exact box-constrained model minimiser, ratio test, best point
 * evaluated) is documented with the implementation and mirrored by the FP64
 * oracle.  Host-driven: each iteration launches the CV of its new sample
 * bandwidths and reads the scores back (synchronising the stream).
 *  h0        host, d doubles: the starting bandwidths (e.g. the learned proposal);
 *            their CV score must be finite.
 *  opt       NULL for the defaults {0.4, 0.01, 1.0, 0.02, 0.6, 20}.
 *  h_best    host, d doubles out; cv_best, n_evals host out (may be NULL).
 *  trace     host, trace_cap x (d + 1) doubles out (may be NULL): every
 *            evaluated bandwidth vector and its CV score in evaluation order. */
typedef struct {
  double delta0, delta_min, delta_max;  /* trust-region half-width in log h */
  double h_lo, h_hi;                    /* bounds of every bandwidth */
  int max_iter;
} fpca_tr_options;

fpca_status fpca_bw_trust_region(fpca_ctx* ctx, const fpca_grid* grid, const fpca_covbins* bins,
                                 int prec, const double* h0, const fpca_tr_options* opt,
                                 double* h_best, double* cv_best, int* n_evals, double* trace,
                                 int trace_cap);

/* ---- noise variance (Eq. 2.5-2.6) ------------------------------------------
 *
 * sigma2_hat(t) = b0(t) - Gamma_hat(t, t) - mu_hat(t)^2 at every grid node, where
 * b0 is the local linear fit of Eq. (2.5) to the squared observations (the mean
 * smoother of Eq. 2.3 applied to the bins cnt, w, v2 of fpca_bin_mean, bandwidth h,
 * FP64).  The paper prints "+ mu_hat mu_hat"; since E[Y^2] = Gamma + sigma^2 + mu^2
 * the mean term is subtracted.  Eq. (2.6) integrates over Omega; the integral is
 * divided by |Omega| (the mean over the domain nodes) so that a constant sigma^2
 * is recovered on any domain.
 *  cnt, w, v2   P mean bins (fpca_bin_mean; v2 = sum Y^2 / N_i).
 *  h            host, d doubles (h_sigma).
 *  mu           P doubles, the mean fit.
 *  gdiag        Gamma_hat(t, t): element p at gdiag + p * gdiag_stride (FP64 or FP32
 *               per gdiag_prec) -- the diagonal of a P x P surface (stride P + 1) or
 *               a length-P vector (stride 1).
 *  domain       P int32 (e.g. the mean-bin counts; > 0 = inside Omega) or NULL (all).
 *  sigma2_t     P doubles out (NaN where the b0 fit is EMPTY); status P uint8 out
 *               (FPCA_PT_*) or NULL; sigma2 one double out (the average) or NULL. */
fpca_status fpca_sigma2(fpca_ctx* ctx, const fpca_grid* grid, const int32_t* cnt, const double* w,
                        const double* v2, const double* h, const double* mu, const void* gdiag,
                        int gdiag_prec, long long gdiag_stride, const int32_t* domain,
                        double* sigma2_t, uint8_t* status, double* sigma2);

/* ---- principal component scores (Section 2.1, Eq. 2.7) ----------------------
 *
 * Functions known on the grid (mu, phi_l) are read at an observation through the
 * bin that holds it (the binning of Section 3.2).  evals (L doubles) and evecs
 * (P x L column-major, phi_l at evecs + l * P, the normalisation of
 * fpca_rproj_eig: sum_p phi_l(p)^2 / P = 1) are device arrays; 1 <= L <= 16.
 * scores is n x L row-major device doubles, overwritten.
 *
 * fpca_scores_pace: the conditional expectation of Eq. (2.7),
 *   A_i = Lambda Phi_i' (Phi_i Lambda Phi_i' + sigma^2 I)^{-1} (Y_i - mu(t_i)),
 * evaluated through the push-through identity as the L x L system
 *   (sigma^2 Lambda^{-1} + Phi_i' Phi_i) A_i = Phi_i' (Y_i - mu(t_i))
 * (sums in compensated FP32 -- error-free products and additions on
 * float-float inputs, about FP64 accuracy -- then an FP64 Cholesky).  Gridded
 * data (mask or all nodes) and
 * scattered data (offs, t) are both accepted.  A subject without observations
 * gets A_i = 0 (the prior mean).  sigma2 is ONE device double (e.g. the output
 * of fpca_sigma2, so no host round trip separates the two calls); it must be
 * >= 0 and every evals[l] > 0 (with sigma2 == 0 the system is singular for a
 * subject with fewer than L observations).  A negative or NaN sigma2, a
 * non-positive evals[l] or a non-positive pivot writes NaN scores for the
 * subject and makes fpca_sync() return FPCA_E_NUMERIC.
 *
 * fpca_scores_integral: the integral of (Y_i - mu) phi_l over Omega as the
 * Riemann sum over the subject's observed nodes, cell volume dV = 1/P (gridded
 * data only; compensated FP32 sums, about FP64 accuracy).
 *
 * fpca_reconstruct: X_i(t_p) = mu(t_p) + sum_l A_il phi_l(t_p) at every node,
 * n x P row-major FP32 out (compensated sum, rounded once; n < 2^20).
 *
 * Each of the three splits mu and the first L eigenfunctions into float-float
 * in the context's workspace first (which may synchronise the stream the first
 * time it grows). */
fpca_status fpca_scores_pace(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                             const double* mu, const double* evals, const double* evecs, int L,
                             const double* sigma2, double* scores);
fpca_status fpca_scores_integral(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                                 const double* mu, const double* evecs, int L, double* scores);
fpca_status fpca_reconstruct(fpca_ctx* ctx, const fpca_grid* grid, const double* mu,
                             const double* evecs, int L, const double* scores, int n,
                             float* xhat);

/* MISE of a reconstruction (Section 4, Simulation I): (1/n) sum_i of the
 * integral over Omega of (xhat_i - x_i)^2, as the Riemann sum over all P grid
 * nodes with dV = 1/P.  xhat: n x P FP32 (fpca_reconstruct); x: n x P, FP64
 * (x_prec FPCA_F64) or FP32 (FPCA_F32), e.g. the noise-free curves of a
 * simulation; mise: one device double out.  Compensated FP32 sums per thread,
 * FP64 trees across threads and blocks (deterministic). */
fpca_status fpca_mise(fpca_ctx* ctx, const fpca_grid* grid, const float* xhat, const void* x,
                      int x_prec, int n, double* mise);

/* ---- d = 3: covariance smoothing fused into its projection ----------------
 *
 * For a 32 x 32 x 32 grid the covariance grid has P^2 = 1.07e9 points; these
 * entry points smooth it (Eq. 2.4 with the Section 3.2 binning) and apply it
 * to a block of vectors without forming the P x P bins or the P x P surface,
 * for the random projection of Section 3.4.
 *
 * Scope: d = 3, every subject observed at every grid node (dense layout,
 * mask NULL), 2 <= M_k <= 64, residual mode, the same bandwidth vector h for
 * s and t with 1..4 kernel taps per axis (taps = #{k >= 1 : k/(h_k M_k) < 1};
 * the shared-memory staging of the near-diagonal tile pairs holds at most 4).
 * Other inputs return FPCA_E_UNSUPPORTED.
 *
 * Arithmetic: residuals R~ = (Y - mu_hat)/sqrt(n) in BF16 for the tensor-core
 * products (FP32 accumulation), FP32 elsewhere; per-point local solves in
 * FP32 (an ill-conditioned one makes fpca_sync() return FPCA_E_NUMERIC);
 * Rayleigh-Ritz as fpca_rproj_eig (l = 64: FP32 Jacobi, FP64 refinement).
 * For fully observed data every local system is regular (status FPCA_PT_OK
 * at every point), so no status array is produced.
 */

/* Bytes of the factored covariance bins of n subjects on `grid` (0 if the
 * grid is not 3-dimensional).  Host function, no device work. */
size_t fpca_cov_factor_bytes(const fpca_grid* grid, int n);

/* Covariance bins of fully observed gridded data in factored form (Eq. 2.4,
 * Section 3.2): the bins are W[p,q] = sum_i w_i (p != q) and
 * V[p,q] = sum_i w_i R_ip R_iq with the diagonal p == q dropped, so the
 * n x P residual matrix R = Y - mu_hat determines them; it is stored (with
 * its node-wise sums of squares) instead of the P x P arrays.
 *  data   dense layout, mask NULL, y n x P (F32 or F64), n >= 2.
 *  mu     P doubles, the mean fit at the nodes (fpca_smooth_mean).
 *  factor device buffer of at least fpca_cov_factor_bytes(grid, n) bytes,
 *         overwritten; opaque, read by the calls below with the same grid
 *         and n. */
fpca_status fpca_bin_cov_factor(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                                const double* mu, void* factor, size_t factor_bytes);

/* y = Gamma_hat x: the covariance surface of Eq. (2.4) at bandwidth h (host,
 * 3 doubles), residual mode, matrixised as in Section 3.1 (row = s, column
 * = t, nodes in C order), times the P x l block x.
 *  x, y   P x l floats, row-major (row = node), 1 <= l <= 64. */
fpca_status fpca_smooth_cov_apply(fpca_ctx* ctx, const fpca_grid* grid, const void* factor,
                                  int n, const double* h, const float* x, int l, float* y);

/* Gamma_hat at the output pairs of ntiles tile pairs (for checking): tiles
 * (HOST, ntiles x 6 int32) holds per tile the s-box corner (multiples of
 * 4, 4, 8) and the t-box corner (multiples of 4, 4, 4); out (device,
 * ntiles x 128 x 64 floats) receives Gamma_hat(s, t) for the 4 x 4 x 8 s-box
 * (C order) against the 4 x 4 x 4 t-box (C order), NaN where a node lies off
 * the grid.  Synchronises the context's stream before returning. */
fpca_status fpca_smooth_cov_tiles(fpca_ctx* ctx, const fpca_grid* grid, const void* factor,
                                  int n, const double* h, int ntiles, const int32_t* tiles,
                                  float* out);

/* Gamma_hat(t, t) at every node (P doubles, device) from the factored bins at
 * bandwidth h: the diagonal of the surface that fpca_smooth_cov_apply applies,
 * e.g. for fpca_sigma2 (stride 1). */
fpca_status fpca_smooth_cov_diag(fpca_ctx* ctx, const fpca_grid* grid, const void* factor, int n,
                                 const double* h, double* diag);

/* Random projection of Section 3.4 on the fused operator: Y = Gamma_hat Omega,
 * power_iters re-orthonormalised power steps, Rayleigh-Ritz on l columns
 * (FP32 Jacobi with two refinement steps, as fpca_rproj_eig), rescaling
 * lambda = theta dV, phi = psi / sqrt(dV) (dV = 1/P), sign and
 * FVE (trace of Gamma_hat from its diagonal) as fpca_rproj_eig.
 *  omega  P x l floats (device), k < l <= 64.
 *  evals k, evecs P x k column-major (vector j at evecs + j*P), fve k (may
 *  be NULL): device doubles. */
fpca_status fpca_rproj_eig_factor(fpca_ctx* ctx, const fpca_grid* grid, const void* factor,
                                  int n, const double* h, const float* omega, int l, int k,
                                  int power_iters, double* evals, double* evecs, double* fve);

#ifdef __cplusplus
}
#endif

#endif /* FPCA_H */
