/*
 * pt.h -- C ABI of the GB300 max-null permutation-testing library (libpt.so).
 *
 * What it computes (arXiv 1703.01506):
 *   - the permutation testing matrix T (relabellings x voxels) of voxel-wise
 *     pooled-variance two-sample t statistics (Sec. 2.1, Eq. (5)), reduced to
 *     the max-null distribution m_i = max_j T[i][j] (Sec. 2; Alg. 1), plus the
 *     per-voxel uncorrected exceedance counts #{i : T[i][j] >= t_obs[j]};
 *   - the same max-null recovered by RapidPT (Alg. 2, Sec. 4): full rows for
 *     n_train training relabellings, a tracked rank-r subspace, and for every
 *     later relabelling only a sampled subset of voxels.
 *
 * Conventions shared by every entry point:
 *   - All array arguments are caller-owned pointers to DEVICE memory of the
 *     current CUDA device unless the comment says "host". The library never
 *     frees them and never keeps them beyond the call (pt_prepare copies what
 *     it needs; the caller may free X and mask after it returns).
 *   - Work is enqueued on the stream given to pt_prepare. Compute entry points
 *     return once their kernels are enqueued; outputs are valid after the
 *     stream is synchronised. Errors found by the kernels themselves (an input
 *     row that is not a permutation, a bounded wait that expired) are reported
 *     by the next pt_sync on that context.
 *   - Scalar arguments are validated on the host before any launch; an invalid
 *     one returns PT_ERR_INVALID and enqueues nothing.
 *   - Voxel order is the raster order of the mask ("masked order"); v below is
 *     the number of mask voxels. Group 1 is the first n1 entries of each
 *     relabelling row. The observed labelling is the identity (subjects
 *     0..n1-1 in group 1) and is not part of `perms`.
 *   - A voxel whose n values are all equal has no t statistic: it is left out
 *     of every maximum and its count is 0.
 *   - No C++ exception crosses this boundary and nothing here calls exit().
 *     Functions are safe to call from several host threads on distinct
 *     contexts; a single context must not be used concurrently.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt_ctx pt_ctx; /* opaque; owns all device workspaces */

typedef enum {
  PT_OK = 0,
  PT_ERR_INVALID = 1,     /* bad argument or bad input data */
  PT_ERR_NOMEM = 2,       /* device allocation failed */
  PT_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
  PT_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired */
  PT_ERR_UNSUPPORTED = 5  /* valid request the library cannot serve here (e.g. no sm_103 device) */
} pt_status;

/* Arithmetic of the contraction S1 = L . Xn (labels exact in every mode). */
typedef enum {
  PT_PREC_FP32 = 0,    /* plain FP32 CUDA-core (SIMT) kernel */
  PT_PREC_BF16X2 = 1,  /* tcgen05 tensor cores, data split hi+lo in BF16, FP32 accumulate */
  PT_PREC_BF16X3 = 2,  /* tcgen05 tensor cores, data split hi+mid+lo in BF16, FP32 accumulate */
  PT_PREC_FP16X2 = 3   /* tcgen05 tensor cores, data scaled by 2^15 and split hi+lo in FP16
                          (~22 significant bits), labels in FP16, FP32 accumulate */
} pt_precision;

typedef struct {
  int32_t precision; /* pt_precision; default PT_PREC_BF16X3 */
  int32_t two_sided; /* 0 (default): statistic t; 1: statistic |t| (max |t|, counts |t|>=|t_obs|) */
  int32_t accumulate_counts; /* 0 (default): counts = this call's exceedances; 1: counts +=
                                this call's (a run split into relabelling chunks, resumed
                                from a checkpoint or sharded, sums its counts in place) */
} pt_naive_opts;

/* Fills *o with the defaults above. */
void pt_naive_opts_default(pt_naive_opts* o);

/*
 * pt_prepare -- per-voxel centring and moments (the one-time O(n v) step that
 * precedes Alg. 1 / Alg. 2).
 *   X      : device, float32, n x n_grid row-major (row s = subject s over the
 *            whole grid; the "n rows and v columns" data matrix of Sec. 5.3.1).
 *            May also be page-locked host memory that the device can address
 *            (cudaHostAlloc / cudaHostRegister): the kernels then read it over
 *            the host link directly, and only the values of mask voxels.
 *   n      : subjects, 3 <= n <= 1024.
 *   n_grid : columns of X (grid voxels), 1 <= n_grid < 2^31.
 *   mask   : device (or device-addressable page-locked host) memory, uint8,
 *            n_grid entries, nonzero = in the brain; NULL means every grid voxel.
 *   n1     : size of group 1, 1 <= n1 <= n-1 (group 2 has n - n1).
 *   stream : cudaStream_t to run on (NULL = legacy default stream).
 *   out    : host; receives the new context (unchanged on failure).
 * Per voxel it computes, in FP64, the mean and total sum of squares SS of the
 * n values, and stores the centred data scaled to unit norm,
 * Xn[j][s] = (x_s - mean_j) / sqrt(SS_j), in FP32 and as BF16 pieces; and the
 * observed statistic t_obs (identity labelling). It waits on the stream
 * while it runs (to size its buffers from the mask and valid-voxel counts and
 * to report bad input); X and mask are no longer read once it returns, and
 * its last kernel may still be running (stream order covers every later call).
 * Errors: PT_ERR_INVALID for bad sizes or a NaN/Inf in a mask voxel,
 * PT_ERR_NOMEM, PT_ERR_CUDA.
 */
pt_status pt_prepare(const float* X, int32_t n, int64_t n_grid, const uint8_t* mask,
                     int32_t n1, void* stream, pt_ctx** out);

/*
 * pt_prepare_glm -- pt_prepare for the two-group statistic with nuisance
 * covariates (the general-contrast form of the per-voxel statistic that Alg. 1
 * takes as input; Sec. 3.2 instantiates it as the two-sample t of Eq. (5)).
 * For a relabelling with group-1 indicator l the statistic is the least-squares
 * t of beta in  y = beta l + [1, Z] gamma + e  (intercept always added): the
 * group column is relabelled, every subject keeps its covariate values. With
 * q = 0 it is the pooled t of pt_prepare.
 *   X, n, n_grid, mask, n1, stream, out : as pt_prepare.
 *   Z : host, float64, n x q row-major (subject s's covariates in row s); NULL if q = 0.
 *   q : 0 <= q <= 16 and q <= n - 3 (the fit keeps n - q - 2 >= 1 degrees of freedom).
 * Computes in FP64 an orthonormal basis of [1, Z], each voxel's residual on it
 * (a voxel whose residual vanishes, e.g. constant, has no statistic), and the
 * observed statistic (pt_t_obs). Contexts from here run pt_maxnull_naive(_ex)
 * and pt_autotune_naive on the tensor-core precisions (PT_PREC_FP32, RapidPT
 * and the batched call return PT_ERR_UNSUPPORTED), pt_fwer_pvalues, pt_t_obs and
 * pt_maxnull_anova (the F of a factor with these covariates).
 * A relabelling whose group column lies in the span of [1, Z] makes the next
 * pt_sync return PT_ERR_INVALID.
 * Errors: as pt_prepare, and PT_ERR_INVALID for NaN/Inf in Z, [1, Z] without
 * full column rank, or an observed group column in its span.
 */
pt_status pt_prepare_glm(const float* X, int32_t n, int64_t n_grid, const uint8_t* mask,
                         int32_t n1, const double* Z, int32_t q, void* stream, pt_ctx** out);

/*
 * pt_maxnull_naive -- NaivePT (Alg. 1) with default options.
 *   perms   : device, int32, P x n row-major; each row a permutation of 0..n-1.
 *   P       : relabellings, 1 <= P <= 2^31 - 1.
 *   maxnull : device, float32[P]: m_i = max_j t[i][j] (Alg. 1 "Max").
 *   argmax  : device, int32[P]: masked-order voxel of m_i, smallest index on
 *             ties; -1 when the context has no voxel with a defined t.
 *   counts  : device, uint32[v]: #{i : t[i][j] >= t_obs[j]}; may be NULL.
 * T is never written to memory. A row that is not a permutation makes the
 * next pt_sync return PT_ERR_INVALID (outputs then undefined).
 */
pt_status pt_maxnull_naive(pt_ctx* ctx, const int32_t* perms, int64_t P, float* maxnull,
                           int32_t* argmax, uint32_t* counts);

/* pt_maxnull_naive with explicit options (opts NULL = defaults). */
pt_status pt_maxnull_naive_ex(pt_ctx* ctx, const int32_t* perms, int64_t P,
                              const pt_naive_opts* opts, float* maxnull, int32_t* argmax,
                              uint32_t* counts);

/*
 * pt_maxnull_naive_batched -- NaivePT (Alg. 1) for several independent
 * studies in one call: per study i, exactly what pt_maxnull_naive_ex computes
 * for (ctxs[i], perms[i], P[i]) into maxnull[i], argmax[i], counts[i]. The
 * paper runs one study at a time (Sec. 5); batching only packs the studies'
 * (relabelling block x voxel tile) work into one persistent tensor-core launch
 * per launch class (voxel tile, k-steps per label stage; see pt_tc_config), so
 * small studies share the GPU instead of each leaving SMs idle.
 *   ctxs      : host array of n_studies distinct contexts, all on one device.
 *               Work runs on ctxs[0]'s stream; every context's own stream is
 *               synchronised once when the batch is (re)planned.
 *   n_studies : 1 <= n_studies <= 4096.
 *   perms, P, maxnull, argmax, counts : host arrays of n_studies entries with
 *               the meaning of pt_maxnull_naive's arguments (device buffers);
 *               counts may be NULL, as may any counts[i].
 *   opts      : precision must be a tensor-core one (PT_PREC_BF16X2, _BF16X3 or
 *               _FP16X2; PT_ERR_UNSUPPORTED for FP32); two_sided applies to all.
 * The first call with a given set of arguments plans the launch (host work and
 * one synchronisation), captures it in a CUDA graph and runs the graph; a
 * later call with the same contexts, buffers and sizes replays that graph
 * without host work. One graph is cached per process; pt_destroy of a member
 * context drops it. Errors: PT_ERR_INVALID (NULL entries, P out of range, a
 * context listed twice, contexts on different devices), PT_ERR_UNSUPPORTED,
 * PT_ERR_NOMEM, PT_ERR_CUDA. A row of perms[i] that is not a permutation
 * sets the error flag of ctxs[i]: after pt_sync(ctxs[0]), pt_sync(ctxs[i])
 * returns PT_ERR_INVALID.
 */
pt_status pt_maxnull_naive_batched(pt_ctx* const* ctxs, int32_t n_studies,
                                   const int32_t* const* perms, const int64_t* P,
                                   const pt_naive_opts* opts, float* const* maxnull,
                                   int32_t* const* argmax, uint32_t* const* counts);

/* ------------------------------------------------------------------------- */
/* RapidPT (Alg. 2; Sec. 4.1 training, Sec. 4.2 recovery)                     */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t precision;    /* contraction of the training rows (pt_precision); default BF16X3 */
  int32_t train_passes; /* passes over the training columns; default 1 (Alg. 2's single
                           loop; Sec. 4.1 allows "multiple passes") */
  int32_t qr_every;     /* re-orthonormalise U (FP64-factorised QR) every this many steps;
                           default 100 */
  int32_t admm_iters;   /* iterations of each l1 weight solve; default 30 */
  float admm_rho;       /* ADMM penalty rho; default 2 */
  float step;           /* geodesic step: theta = step * atan(||r|| / ||w||); default 1 */
  int32_t shift_mode;   /* 0: mu = largest training residual (Alg. 2 as printed);
                           1 (default): mu = mean shift of the maximum (Sec. 4.1) */
  uint64_t seed;        /* key of the Philox4x32-10 draws; default 1 */
  float rec_step;       /* U during recovery: 0 (default) frozen, as Alg. 2 prints it;
                           > 0: after each recovery relabelling's maximum is formed, U takes
                           the training step (geodesic, theta = rec_step * atan(||r||/||w||))
                           towards that relabelling's fit residual on its samples, in row
                           order, with QR every qr_every such steps (recovery becomes
                           sequential: one step and one reconstruction per relabelling) */
} pt_rapid_opts;

typedef struct {
  double sigma;         /* std of the sampled training residuals */
  double mu;            /* shift added to every recovered maximum */
  int64_t m_per_perm;   /* sampled voxels per relabelling, ceil(sample_rate * v_valid) */
  int64_t train_steps;  /* subspace-tracking steps taken (train_passes * n_train) */
} pt_rapid_info;

/* Fills *o with the defaults above (one training pass, QR every 100 steps,
 * 30 ADMM iterations at rho = 2, step 1, shift_mode 1, seed 1, BF16X3, U frozen
 * during recovery). */
void pt_rapid_opts_default(pt_rapid_opts* o);

/*
 * pt_maxnull_rapid -- RapidPT max-null (Alg. 2).
 *   perms, P   : device int32 P x n relabellings; rows 0..n_train-1 train.
 *   rank       : r, 1 <= r <= min(n, 128).
 *   sample_rate: eta in (0, 1]; m = ceil(eta * v_valid) >= r voxels are drawn
 *                (i.i.d. uniform, Alg. 2 "UNIF[1, v]") per relabelling. The m
 *                sampled rows of U (4 m r bytes) and one r x r matrix per CTA must
 *                fit the shared memory of a 16-CTA cluster: m <= 13,280 at r = 50,
 *                4,480 at r = 100, 2,144 at r = 128; larger requests return
 *                PT_ERR_UNSUPPORTED before any work.
 *   n_train    : l, 1 <= l < P.
 *   maxnull    : device float32[P]; rows < l: exact maxima of the training rows
 *                (statistic recomputed in FP64); rows >= l: max_j (U w + s)_j + mu.
 *   counts     : device uint32[v] or NULL: exceedances t >= t_obs over the l
 *                training rows (the only rows computed in full).
 *   info       : host, or NULL: sigma, mu, m, steps.
 * One-sided statistic only. Synchronises the stream; a bad relabelling row makes
 * the next pt_sync return PT_ERR_INVALID.
 */
pt_status pt_maxnull_rapid(pt_ctx* ctx, const int32_t* perms, int64_t P, int32_t rank,
                           double sample_rate, int32_t n_train, const pt_rapid_opts* opts,
                           float* maxnull, uint32_t* counts, pt_rapid_info* info);

/*
 * pt_rapid_train -- the training phase alone (Sec. 4.1) on relabellings 0..n_train-1.
 *   U_out    : device float32 v_valid x rank (row j = voxel j in the compact order of
 *              voxels with a defined t), or NULL.
 *   train_max: device float32[n_train] or NULL (exact training maxima).
 *   counts   : device uint32[v] or NULL (as pt_maxnull_rapid).
 *   w_hist   : device float32[train_steps][rank] or NULL: weights of every step.
 *   info     : host or NULL.
 * Synchronises the stream.
 */
pt_status pt_rapid_train(pt_ctx* ctx, const int32_t* perms, int32_t n_train, int32_t rank,
                         double sample_rate, const pt_rapid_opts* opts, float* U_out,
                         float* train_max, uint32_t* counts, float* w_hist,
                         pt_rapid_info* info);

/*
 * pt_rapid_recover -- the recovery phase alone (Sec. 4.2) for rows
 * first_row..P-1 of perms with a given basis U (v_valid x rank, device), sigma and
 * mu. Draws are keyed by the row index, so ranges can be split across calls or
 * devices with identical results (with opts->rec_step = 0; with U updates the
 * rows depend on the rows before them and the given U is the state at first_row).
 *   maxnull: device float32[P - first_row].  W_out: device float32[P - first_row][rank]
 *   or NULL (weights). Synchronises the stream.
 */
pt_status pt_rapid_recover(pt_ctx* ctx, const int32_t* perms, int64_t P, int64_t first_row,
                           const float* U, int32_t rank, double sample_rate, double sigma,
                           double mu, const pt_rapid_opts* opts, float* maxnull, float* W_out);

/*
 * pt_sync -- wait for the context's stream and report errors the kernels
 * raised since the previous pt_sync (PT_ERR_INVALID for a bad relabelling
 * row, PT_ERR_TIMEOUT for an expired device wait), then clear them.
 */
pt_status pt_sync(pt_ctx* ctx);

/*
 * pt_t_rows -- rows of the permutation testing matrix T (Sec. 2.1): the pooled
 * t of Eq. 5 at every mask voxel under each of P relabellings, written out
 * (NaivePT never forms T; this call is for inspection and for RapidPT's
 * training rows, whose kernels it shares).
 *   perms     : device, int32, P x n (as pt_maxnull_naive), 1 <= P <= 2^31 - 1.
 *   precision : PT_PREC_FP32 (CUDA cores) or PT_PREC_BF16X2 / _BF16X3 / _FP16X2
 *               (tensor cores).
 *   T         : device, float32, P x v row-major in masked order; NaN where the
 *               voxel has no statistic. P * v * 4 bytes, caller-owned.
 * t is formed in FP32 from the FP32 accumulator u as sqrt(k(n-2)) u / sqrt(1 - k u^2).
 * Asynchronous on the context's stream; invalid rows make the next pt_sync
 * return PT_ERR_INVALID. PT_ERR_UNSUPPORTED for a context with covariates.
 */
pt_status pt_t_rows(pt_ctx* ctx, const int32_t* perms, int64_t P, int32_t precision, float* T);

/*
 * pt_maxnull_anova -- NaivePT (Alg. 1) with the one-way F of g groups as the
 * voxel statistic (Alg. 1's "stat" input with several group columns; g = 2 gives
 * F = t^2 of Eq. 5): F = (SS_between / (g-1)) / (SS_within / (n-g)).
 *   perms       : device int32 P x n; positions [0, n_1) of a row form group 1,
 *                 [n_1, n_1 + n_2) group 2, ...; the observed labelling is the identity.
 *   group_sizes : host int32[g], each >= 1, summing to the context's n; 2 <= g <= 16, n > g.
 *   precision   : as pt_naive_opts (the g - 1 group sums come from the same contraction).
 *   maxnull, argmax : device float32[P] / int32[P]: max over voxels of F (the winner's F
 *                 recomputed in FP64 from the input values) and its masked voxel index.
 *   counts      : device uint32[v] or NULL: #{i : F_ij >= F_obs_j}.
 * With a context from pt_prepare_glm (covariates Z, intercept added) the statistic is the
 * factor's F in  y = E beta + [1, Z] gamma + e  (E: indicators of groups 1..g-1 of the
 * relabelling; every subject keeps its covariate values):
 *   F = ((RSS_reduced - RSS_full) / (g-1)) / (RSS_full / (n - g - q)),
 * formed from the g - 1 group sums of each voxel's unit-norm residual on [1, Z] and, per
 * relabelling, (E^T (I - H) E)^-1 in FP64 (H the projector on [1, Z]); BF16X2 / BF16X3
 * only (PT_ERR_UNSUPPORTED otherwise), n - g - q >= 1. A relabelling whose group columns
 * are not independent of [1, Z] makes the next pt_sync return PT_ERR_INVALID.
 * The context's n1 plays no part. Synchronous; a bad relabelling row makes the next
 * pt_sync return PT_ERR_INVALID.
 */
pt_status pt_maxnull_anova(pt_ctx* ctx, const int32_t* perms, int64_t P,
                           const int32_t* group_sizes, int32_t g, int32_t precision,
                           float* maxnull, int32_t* argmax, uint32_t* counts);

/*
 * Cluster-level summaries (the cluster tables of Sec. 6, Figs. 8-9, and the
 * permutation distribution of the largest cluster, the cluster-level
 * counterpart of the max-null of Sec. 2). A mask voxel is active when its t
 * reaches tau; clusters are connected sets of active voxels on the grid.
 *   tau          : cluster-forming threshold on t (finite).
 *   dims         : host int32[3] (d0, d1, d2), d0 * d1 * d2 = n_grid; grid index
 *                  g = (i0 * d1 + i1) * d2 + i2 (C order, as X's columns).
 *   connectivity : 6 (faces), 18 (faces, edges) or 26 (faces, edges, corners).
 * The plain two-sample t only (PT_ERR_UNSUPPORTED with covariates).
 *
 * pt_cluster_maxnull -- maxsize[i] (device int32[P]) = size of the largest
 *   cluster of relabelling i (0 when no voxel is active). perms as
 *   pt_maxnull_naive; precision as pt_naive_opts. A batch of relabellings at a
 *   time, the contraction writes one bit per relabelling and voxel (t >= tau)
 *   and the components are found over the active voxels (about 2 GB of device
 *   workspace, of which only the active voxels' entries are touched). Synchronous.
 * pt_cluster_observed -- the observed map's clusters, in masked order:
 *   label[j] (device int32[v]) = masked index of the smallest voxel of j's
 *   cluster, or -1; size[j] (device int32[v]) = that cluster's size, or 0.
 *   The cluster-level FWER p-value of a cluster of size k is
 *   (1 + #{i : maxsize[i] >= k}) / (P + 1). Synchronous.
 */
pt_status pt_cluster_maxnull(pt_ctx* ctx, const int32_t* perms, int64_t P, double tau,
                             const int32_t* dims, int32_t connectivity, int32_t precision,
                             int32_t* maxsize);
pt_status pt_cluster_observed(pt_ctx* ctx, double tau, const int32_t* dims, int32_t connectivity,
                              int32_t* label, int32_t* size);

/* t_obs: device float32[v]: observed statistic per voxel (NaN where undefined).
 * Enqueued on the context's stream. */
pt_status pt_t_obs(pt_ctx* ctx, float* t_obs);

/*
 * pt_fwer_pvalues -- FWER-corrected p-value of every mask voxel from a
 * max-null (Sec. 2: the share of the permutation distribution of the maximum
 * statistic at or above the voxel's observed statistic; the observed
 * labelling counts as one of the P + 1):
 *   p_j = (1 + #{i : maxnull_i >= T_j}) / (P + 1),  T_j = t_obs_j (|t_obs_j| if two_sided),
 * compared as float32 values.
 *   maxnull : device, float32[P] (from pt_maxnull_naive / _rapid with the same sidedness).
 *   p_out   : device, float32[v] in masked order; NaN where the voxel has no t.
 * Asynchronous on the context's stream. The smallest attainable value is 1/(P + 1).
 */
pt_status pt_fwer_pvalues(pt_ctx* ctx, const float* maxnull, int64_t P, int32_t two_sided,
                          float* p_out);

/* ------------------------------------------------------------------------- */
/* Launch configuration of the tensor-core NaivePT kernel and its autotuner.  */
/* The paper has no GPU kernel; these entry points only choose how the fused  */
/* contraction of Alg. 1 is cut into work: the outputs do not depend on the   */
/* configuration (every T entry is summed over the same data pieces and       */
/* subjects in the same order whatever the ring shape or the block split).    */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t voxel_tile;   /* voxels per work tile: 256, 128, 96 or 64, fixed by n (the largest
                           whose data pieces fit in shared memory beside a label ring deep
                           enough to hide the label loads, else beside 4 stages; they stay
                           there while the relabellings stream). It also fixes how the
                           pieces' partial sums are combined, so a configuration must keep
                           it. */
  int32_t stages;       /* depth of the shared-memory ring of label stages, 2..32 (limited by
                           what fits beside the data tile) */
  int32_t ksteps_per_stage; /* k-steps (128 relabellings x 16 subjects, 4 KB) per stage and per
                           ring wait: 1, 2, 4 or 8 */
  int32_t items_per_sm; /* single-study launches split each voxel tile's relabelling blocks
                           until there are at least this many work items per SM, 1..64 */
} pt_tc_config;

/*
 * pt_autotune_naive -- times candidate launch configurations of the fused
 * tensor-core kernel on this problem (ctx's data, these relabellings, the
 * options' precision and sidedness): k-steps per stage (1, 2, 4, 8) x ring
 * depths of 8, 16 and 32 k-steps at eight work items per SM, then block splits
 * of 1, 2 and 4 items per SM for the best;
 * each candidate runs twice and its faster run counts. The fastest is recorded
 * in the process-wide table under the shape key (padded n, precision,
 * sidedness, half-octave buckets of the voxel count and of P), where later
 * pt_maxnull_naive(_ex) and pt_maxnull_naive_batched calls of the same key
 * find it. Shapes without an entry use the default: the largest stage (8, 4, 2
 * or 1 k-steps) of which two fit, a ring of about 16 k-steps, 8 items per SM.
 *   perms, P : as pt_maxnull_naive (device). opts: precision BF16X2 or BF16X3
 *              (PT_ERR_INVALID otherwise); NULL = defaults.
 *   chosen   : host, or NULL: the recorded configuration.
 *   chosen_ms: host, or NULL: its kernel time in ms (CUDA events).
 * Synchronous; computes no outputs. Errors: PT_ERR_INVALID (bad arguments or a
 * row that is not a permutation), PT_ERR_UNSUPPORTED, PT_ERR_NOMEM, PT_ERR_CUDA,
 * PT_ERR_TIMEOUT.
 */
pt_status pt_autotune_naive(pt_ctx* ctx, const int32_t* perms, int64_t P,
                            const pt_naive_opts* opts, pt_tc_config* chosen, double* chosen_ms);

/* pt_autotune_naive for every distinct shape key among the studies of a
 * batched call (arguments as pt_maxnull_naive_batched); a cached batched graph
 * is dropped so that the next batched call plans with the new entries. */
pt_status pt_autotune_naive_batched(pt_ctx* const* ctxs, int32_t n_studies,
                                    const int32_t* const* perms, const int64_t* P,
                                    const pt_naive_opts* opts);

/* The configuration a reduce call would use for n subjects, v voxels with a
 * defined t and P relabellings (host only, no CUDA call): returns 1 when the
 * table has an entry (copied to *out), 0 when it has none (*out = the
 * default), -1 for bad arguments or an n no tile fits. */
int32_t pt_tune_lookup(int32_t n, int32_t precision, int32_t two_sided, int64_t v, int64_t P,
                       pt_tc_config* out);

/* Records cfg for the shape key of (n, precision, two_sided, v, P) without
 * timing. PT_ERR_INVALID if the configuration does not fit that n or names
 * another voxel tile than the one n fixes. */
pt_status pt_tune_set(int32_t n, int32_t precision, int32_t two_sided, int64_t v, int64_t P,
                      const pt_tc_config* cfg);

/* Writes the table to a text file (a header line, then one line per key with
 * its configuration and measured ms), or merges such a file into the table;
 * a malformed file or an entry that does not fit its n leaves the table as
 * it was and returns PT_ERR_INVALID. pt_tune_clear empties the table. */
pt_status pt_tune_save(const char* path);
pt_status pt_tune_load(const char* path);
void pt_tune_clear(void);

/* grid_index: device int64[v]: grid column of each masked-order voxel. */
pt_status pt_voxel_grid_index(pt_ctx* ctx, int64_t* grid_index);

/* Number of mask voxels (v, the length of counts and of the masked-order maps),
 * and of those with a defined statistic; -1 if ctx is NULL. */
int64_t pt_num_voxels(const pt_ctx* ctx);
int64_t pt_num_valid_voxels(const pt_ctx* ctx);

/* Text of the last failure on ctx (or, for ctx NULL, of the last failure of a
 * call without a context on this thread, e.g. pt_prepare). Never NULL. */
const char* pt_last_error(const pt_ctx* ctx);

/*
 * Profiling of the dominant kernel. When enabled, every compute call records a
 * pair of CUDA events on the context's stream around the launch of its main
 * contraction kernel. pt_profile_read waits for the last timed launch (not for
 * later work on the stream) and returns (host outputs) the summed device time
 * in ms and the number of timed launches since the previous read, then resets
 * both.
 */
pt_status pt_profile_enable(pt_ctx* ctx, int32_t on);
pt_status pt_profile_read(pt_ctx* ctx, double* total_ms, int64_t* launches);

/* Number of kernels this library has launched in this process (all contexts). */
int64_t pt_kernel_launch_count(void);

/* ------------------------------------------------------------------------- */
/* Failure handling checks (no counterpart in the paper). Failures are made on */
/* the host or by a wait that runs out of time; nothing here faults the GPU.  */
/* ------------------------------------------------------------------------- */

/*
 * pt_debug_fail_allocations -- after `after` more device allocations by this
 * library (its caching allocator's requests, cache hits included) every later
 * one fails, so the calls that need memory return PT_ERR_NOMEM; after < 0
 * switches the injection off. Process-wide; for tests of the error paths.
 */
void pt_debug_fail_allocations(int64_t after);

/*
 * pt_debug_device_reset -- cudaDeviceReset() on the calling thread's current
 * device, through the library's own CUDA runtime: every allocation and module
 * of this process on that device is released and the primary context starts
 * afresh at its next use. Only for tests that check a call still works after
 * such a reset; no pt_ctx may be alive. Returns PT_ERR_CUDA on failure.
 */
pt_status pt_debug_device_reset(void);

/*
 * pt_selftest_bounded_wait -- runs, on ctx's stream, the library's bounded
 * device-side wait on an mbarrier phase that nothing completes, with a limit of
 * limit_ms (1 <= limit_ms <= 2000): the kernel gives up, records the timeout in
 * ctx's status word and returns. The next pt_sync returns PT_ERR_TIMEOUT and
 * clears it; the context stays usable. Asynchronous.
 */
pt_status pt_selftest_bounded_wait(pt_ctx* ctx, int32_t limit_ms);

/*
 * pt_maxnull_naive_noalloc -- NaivePT (FP32 CUDA-core contraction) for callers
 * that cannot allocate device memory. The paper has no counterpart: this entry
 * point exists for callers that must not call cudaMalloc (code running inside
 * another runtime's memory pool, or under a fixed memory budget after
 * start-up). It allocates nothing: all intermediate buffers live in one static
 * device array of 64 MiB that every GPU loading this library holds until the
 * process exits.
 *   X       : device, float32, n x v row-major (every column is a voxel; no mask).
 *   n, n1   : as pt_prepare (3 <= n <= 1024, 1 <= n1 <= n-1); v >= 1.
 *   perms, P, maxnull, argmax, counts : as pt_maxnull_naive (argmax is the
 *             column of X; counts may be NULL). perms holds P x n entries,
 *             maxnull and argmax P each, counts v.
 *   two_sided: 0 statistic t, 1 statistic |t|.
 *   stream  : cudaStream_t to run on (NULL = legacy default stream).
 * Synchronous: it reads two status words back to the host and waits on the
 * stream during the work and at its end. Returns PT_ERR_INVALID for a bad
 * argument, NaN/Inf in X, a row that
 * is not a permutation, or a problem whose buffers exceed the 64 MiB array
 * (the message gives the bytes needed). Each call looks up the array's device
 * address (cudaGetSymbolAddress) in the context current at the call, so it is
 * valid in any context on the device, including the primary context after
 * cudaDeviceReset. Calls share the array: calls that overlap on the GPU race
 * and must be serialised by the caller.
 */
pt_status pt_maxnull_naive_noalloc(const float* X, int32_t n, int64_t v, int32_t n1,
                                   const int32_t* perms, int64_t P, int32_t two_sided,
                                   float* maxnull, int32_t* argmax, uint32_t* counts,
                                   void* stream);

/* Frees the context's device memory (returned to the library's cache). NULL ok.
 * Does not wait for work the context has queued: its blocks are handed out
 * again only after an event recorded on its stream at this call has completed,
 * so a context created next on the same stream may be prepared at once. A
 * context that took part in the cached pt_maxnull_naive_batched graph is waited
 * for (the device is synchronised) before its memory is returned. Results the
 * queued work writes into caller buffers still arrive in stream order. */
void pt_destroy(pt_ctx* ctx);

/* Returns every cached device block to the driver (cudaFree), after waiting for
 * the work of destroyed contexts whose blocks are still held back. */
void pt_release_cached_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* PT_H */
