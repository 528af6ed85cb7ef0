/*
 * dpmm.h -- C ABI of the GB300 (sm_103a) sweep library for the sub-cluster
 * split/merge Dirichlet-process mixture sampler (Dinari, Zamir, Fisher III,
 * Freifeld, arXiv 2204.08988; sampler of Chang & Fisher III, NIPS 2013).
 *
 * One context holds one chain: the data X (N points of dimension d), the labels
 * z (cluster) and zbar (sub-cluster l=0 / r=1), the sufficient statistics of the
 * K clusters and 2K sub-clusters, and the parameters drawn from them.  A sweep
 * (dpmm_sweep) is one iteration of Sec. 4.1: (a) weights, (b) sub-weights, (c)
 * cluster and (d) sub-cluster parameters, (e) labels, (f) sub-labels, the
 * sufficient statistics, then the split and merge proposals.  Every step runs on
 * the GPU; there is no CPU fallback: without a usable sm_103a device every call
 * that needs one returns DPMM_ECUDA.
 *
 * Conventions
 *  - The caller owns every buffer it passes; the library never keeps a caller
 *    pointer after a call returns, except that dpmm_update_data reads page-locked
 *    host input asynchronously, until the next synchronising call.  Host buffers
 *    are CPU memory (pageable or page-locked); where a call takes `on_device`, a
 *    non-zero value means the pointer is device memory of the context's device.
 *  - All work is ordered on the stream given to dpmm_set_options (default: the
 *    legacy default stream).  Calls that return data to the host synchronise that
 *    stream; dpmm_sweep does not.
 *  - Every call returns a status; dpmm_last_error gives the text of the last
 *    failure of that context.  No exception crosses the ABI.
 *  - Matrices are row-major.  Slot s = 3k + 0 is cluster k, 3k + 1 and 3k + 2
 *    its sub-clusters l and r.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 * (entity, sweep index, tag << 24 | block, problem); the layout is fixed, so a
 * chain is reproducible from (data, prior, options, seed) alone.
 */
#ifndef DPMM_H
#define DPMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpmm_ctx dpmm_ctx; /* opaque, library-owned */

typedef enum {
    DPMM_OK = 0,
    DPMM_EINVAL = 1,   /* bad argument (message says which) */
    DPMM_ENOMEM = 2,   /* device or host allocation failed */
    DPMM_ECUDA = 3,    /* CUDA runtime/driver error, or no usable sm_103a device */
    DPMM_ESTATE = 4,   /* call out of order (e.g. sweep before set_data) */
    DPMM_ENUMERIC = 5, /* NaN score or non-positive-definite scale seen on the device */
    DPMM_ETIMEOUT = 6  /* a bounded device wait gave up */
} dpmm_status;

/* Component family and conjugate prior (Sec. 2.2).
 * DPMM_PRIOR_NIW: Gaussian components, Normal-Inverse-Wishart prior
 *   NIW(mu, Sigma; kappa0, m0, nu0, Psi0) = N(mu; m0, Sigma/kappa0) W^-1(Sigma; nu0, Psi0),
 *   kappa0 > 0, nu0 > d - 1, Psi0 symmetric positive definite (d x d), m0 in R^d.
 * DPMM_PRIOR_DIRICHLET: multinomial components (count vectors), Dirichlet(beta)
 *   prior, beta_j > 0. */
typedef enum { DPMM_PRIOR_NIW = 0, DPMM_PRIOR_DIRICHLET = 1 } dpmm_prior_kind;

typedef struct {
    dpmm_prior_kind kind;
    double kappa0;       /* NIW */
    const double* m0;    /* NIW, d values */
    double nu0;          /* NIW */
    const double* psi0;  /* NIW, d x d */
    const double* beta;  /* Dirichlet, d values */
} dpmm_prior;

/* Element type of the data passed to dpmm_set_data. */
typedef enum { DPMM_F64 = 0, DPMM_F32 = 1, DPMM_BF16 = 2, DPMM_I32 = 3 } dpmm_dtype;

/* Arithmetic of the label step (e)-(f) and of the statistics.
 * FP64_PLAIN: everything in FP64 on CUDA cores (the parity path).
 * FP32: FP32 CUDA cores, FP64 combine of statistics.
 * TF32 / BF16: the cluster likelihoods as one tensor-core contraction
 *   (tcgen05, FP32 accumulation), the rest as FP32.  TF32: Gaussian, d <= 32;
 *   BF16: multinomial, d <= 256.
 * BF16X3: Gaussian, d <= 128: the cluster likelihoods as a tensor-core
 *   contraction with both operands split into two BF16 values (three products,
 *   about 16 significant bits per operand, FP32 accumulation); sub-labels and
 *   statistics as FP32.
 * Every reduced precision draws the parameters with an FP32 factorisation and
 * redoes a slot in FP64 when that factorisation loses too much to cancellation. */
typedef enum {
    DPMM_PREC_FP64_PLAIN = 0,
    DPMM_PREC_TF32 = 1,
    DPMM_PREC_BF16 = 2,
    DPMM_PREC_FP32 = 3,
    DPMM_PREC_BF16X3 = 4
} dpmm_prec;

/* Create a chain.  alpha > 0 is the DP concentration (Eq. DPLatentVar); d >= 1
 * the dimension (at most 160 for the NIW prior, 65536 for the Dirichlet prior;
 * multinomial data of more than 256 categories are held as compressed rows, see
 * dpmm_set_data_csr, run in FP32 or FP64_PLAIN and take K_max <= 256);
 * 1 <= K_max <= 1000 the capacity for clusters (a split that would exceed it is
 * rejected and counted, Sec. 4.1 "Propose and accept splits").
 * Errors: DPMM_EINVAL for invalid hyper-parameters or sizes (kappa0 <= 0,
 * nu0 <= d - 1, Psi0 not symmetric positive definite, beta_j <= 0, alpha <= 0, d or
 * K_max out of range), DPMM_ECUDA without a usable sm_103 device, DPMM_ENOMEM when
 * the device tables (O(K_max d^2) doubles) do not fit.  *out is NULL on error. */
dpmm_status dpmm_create(const dpmm_prior* prior, double alpha, int d, int K_max, dpmm_ctx** out);

/* Options; call before dpmm_set_data.  init_K: clusters at start (Sec. 3.4
 * examples start from 1); burn_out: sweeps a new cluster must complete before it
 * may be split (the examples pass 15); cuda_stream: a cudaStream_t or NULL. */
dpmm_status dpmm_set_options(dpmm_ctx* ctx, dpmm_prec prec, int init_K, int burn_out, void* cuda_stream);

/* Data (Sec. 2.2: the observations x_1..x_N the mixture is fitted to; Sec. 4.5: the
 * library holds them once on the device, O(d N) memory): N x d row-major of type dt.
 * The library copies and converts it into its
 * own device buffer (FP64 for FP64_PLAIN, FP32 for FP32/TF32/BF16X3, BF16 for BF16;
 * Gaussian data is centred by its mean, an exact reparameterisation undone in
 * every output).  X is device memory (on_device = 1) or host memory: page-locked
 * host memory is read in place by the conversion kernels, pageable memory is first
 * staged in device memory.  Resets the chain: the labels are drawn at the next sweep.
 * Errors: DPMM_EINVAL (N < 1, NULL X, type not allowed for the prior). */
dpmm_status dpmm_set_data(dpmm_ctx* ctx, const void* X, int64_t N, dpmm_dtype dt, int on_device);

/* Multinomial data of more than 256 categories as compressed rows (Sec. 5.3's
 * document-word data; such data are also taken by dpmm_set_data as dense counts and
 * compressed on the device): host arrays indptr[N + 1] (indptr[0] = 0, non-decreasing),
 * indices[nnz] (categories in [0, d), increasing within each row) and counts[nnz]
 * (in [0, 2^24)), nnz = indptr[N].  Copied; resets the chain like dpmm_set_data.  The
 * score of point i under cluster k is log pi_k + sum over its nonzeros of count x
 * log theta_kj, the same sum as over all d categories.  Errors: DPMM_EINVAL for a context
 * that does not hold compressed rows (Gaussian, or d <= 256) or malformed arrays. */
dpmm_status dpmm_set_data_csr(dpmm_ctx* ctx, const int64_t* indptr, const int32_t* indices, const int32_t* counts,
                              int64_t N);

/* Replace the values of the data (same N, d, dtype) and keep the chain's state.
 * Used for streaming data and for end-to-end timing with host-resident inputs.
 * Asynchronous on the context's stream: a host buffer must keep its values until
 * the next synchronising call (e.g. dpmm_get_labels). */
dpmm_status dpmm_update_data(dpmm_ctx* ctx, const void* X, dpmm_dtype dt, int on_device);

/* Stage the values of the next sweep's data (same N, d, dtype; host memory), for
 * streaming inputs: Sec. 4.5 keeps the data on the device, and new values must cross
 * the CPU-GPU link every step.  The copy runs on a copy-engine stream of the context's
 * own, so it overlaps the sweep in flight; the next dpmm_sweep (or dpmm_sweep_sharded)
 * waits for it and converts the staged values into the data before its first kernel,
 * exactly as dpmm_update_data would have.  A second call before that sweep replaces the
 * staged values; dpmm_update_data and dpmm_set_data discard them.  The device staging
 * buffer (the input's size) stays with the context until dpmm_destroy.  Page-locked
 * host memory is copied asynchronously and must keep its values until the next
 * synchronising call; pageable memory is copied before the call returns.  Not for
 * compressed rows.  Errors: DPMM_ESTATE without data, DPMM_EINVAL (NULL X, another
 * dtype, compressed rows), DPMM_ENOMEM (staging buffer). */
dpmm_status dpmm_stage_data(dpmm_ctx* ctx, const void* X, dpmm_dtype dt);

/* Run `iters` sweeps (Sec. 4.1) with Philox key `seed`.  The sweep counter
 * persists across calls, so two calls of 5 equal one call of 10.  Asynchronous on
 * the context's stream. */
dpmm_status dpmm_sweep(dpmm_ctx* ctx, int iters, uint64_t seed);

/* Problem id of this chain: the fourth word of every Philox counter (the paper's
 * counters name the point or cluster, the sweep and the draw; this word keeps the
 * random streams of independent chains apart, e.g. the problems of a batch).
 * Default 0.  Takes effect at the next kernel, also inside an already captured
 * sweep graph.  Synchronises. */
dpmm_status dpmm_set_problem(dpmm_ctx* ctx, uint32_t problem);

/* Batched sweeps of independent problems: `iters` sweeps of each of the n
 * contexts, interleaved (sweep t of every context before sweep t + 1), all with
 * Philox key `seed` (give each context its own problem id).  Each context's sweeps
 * are queued asynchronously on its own stream as a captured graph, so contexts with
 * distinct non-NULL streams run concurrently on the GPU and small problems fill it
 * together.  The paper runs one problem per call and has no counterpart; the result
 * of every context equals that of dpmm_sweep on it alone.  Returns the first
 * failing context's status (the remaining contexts of that round are not queued);
 * DPMM_EINVAL for a NULL array or entry, n < 0 or iters < 0. */
dpmm_status dpmm_sweep_batch(dpmm_ctx* const* ctxs, int n, int iters, uint64_t seed);

/* Point-sharded chains: the data of one chain split over several contexts (e.g. one per
 * GPU).  Every step of Sec. 4.1 that depends on all points reads only
 * the sufficient statistics (Sec. 4.4), so a shard needs its own points and the sum of all
 * shards' statistics.  dpmm_set_shard: this context's data are points [point_offset,
 * point_offset + N) of the whole data set; the random streams of its points are those of
 * their index in the whole set.  Call after dpmm_set_data.  dpmm_sweep_sharded: `iters`
 * sweeps of the chain whose points are held by the G contexts shards[0..G) (1 <= G <= 16,
 * shard s starting where shard s - 1 ends, all with the same prior, options and state).
 * After each shard's label step, and again after a relabelling, the shards' statistics are
 * summed in shard order and every shard receives the sum; every shard then draws the same
 * parameters and takes the same split/merge decisions.  Counts are exact in any order; FP64
 * sums differ from an unsharded chain's by rounding only.  The Gaussian reduced-precision
 * paths centre each context's data by its own mean and are refused (DPMM_EINVAL); the
 * FP64-plain and multinomial paths are supported.  Synchronises between its phases; a
 * sharded context must not be swept by dpmm_sweep alone.  Errors: DPMM_EINVAL (NULL or
 * mismatched shards, offsets that do not tile the points), DPMM_ESTATE (a shard without
 * data), DPMM_ECUDA. */
dpmm_status dpmm_set_shard(dpmm_ctx* ctx, int64_t point_offset);
dpmm_status dpmm_sweep_sharded(dpmm_ctx* const* shards, int G, int iters, uint64_t seed);

/* Checkpoint and resume.  A checkpoint holds everything the next sweep reads, taken
 * at a sweep boundary: K, the sweep counter, the problem id, the labels z and zbar,
 * the cluster ages (split eligibility, Sec. 3.4 burn_out), the sufficient-statistics
 * table with its per-cluster reference shift, and the last weights and split/merge
 * counters.  The parameters are redrawn from the statistics at every sweep (Sec. 4.1
 * steps (a)-(d)) and the random streams are counter-based, so loading a checkpoint
 * into a context with the same prior kind, d, N and data (dpmm_set_data first)
 * continues the chain exactly as if it had never stopped (default step mask).
 * The checkpoint is one host byte buffer of dpmm_checkpoint_size bytes (it grows
 * with K), owned by the caller.  Errors: DPMM_ESTATE without a chain (save) or data
 * (load); DPMM_EINVAL for a short buffer, a buffer that is not a checkpoint, one of
 * another prior, dimension or N, or labels out of range.  All three synchronise. */
dpmm_status dpmm_checkpoint_size(dpmm_ctx* ctx, size_t* bytes);
dpmm_status dpmm_save_checkpoint(dpmm_ctx* ctx, void* buf, size_t bytes);
dpmm_status dpmm_load_checkpoint(dpmm_ctx* ctx, const void* buf, size_t bytes);

/* Failure-detection check (no counterpart in the paper): runs one kernel whose
 * bounded mbarrier wait cannot complete (nothing arrives on the barrier), with the
 * same bounded wait every tensor-core kernel uses.  The wait gives up after its poll
 * or cycle limit (about one second) and the kernel records DPMM_ETIMEOUT in the
 * context's device error word, which this call reads and clears.  Returns
 * DPMM_ETIMEOUT when the mechanism works; the context stays usable.  Synchronises. */
dpmm_status dpmm_check_wait_timeout(dpmm_ctx* ctx);

/* The chain's current assignments (Sec. 2.3: the cluster labels z_i of Eq. DPLatentVar's
 * latent variables and the auxiliary sub-cluster labels zbar_i of the augmented space)
 * into caller-owned host arrays of length N (z in [0, K), zbar in {0,1}).  Either
 * pointer may be NULL.  Synchronises. */
dpmm_status dpmm_get_labels(dpmm_ctx* ctx, int32_t* z, uint8_t* zbar);

/* Sufficient statistics (Sec. 4.4) in the data's original coordinates, for the
 * 3K slots: n[3K], sx[3K x d] (sum of x), sxx[3K x d x d] (sum of x x^T, Gaussian
 * only; may be NULL) and the cluster weights pi_k[K] of the last sweep (may be
 * NULL).  Buffers must hold 3*K_max (resp. K_max) entries.  Synchronises. */
dpmm_status dpmm_get_stats(dpmm_ctx* ctx, int* K, int64_t* n, double* sx, double* sxx, double* weights);

/* Number of clusters and the sweep counter.  Synchronises. */
dpmm_status dpmm_get_info(dpmm_ctx* ctx, int* K, uint32_t* iter);

/* Last sweep's split/merge accounting: out[0] splits, out[1] merges, out[2] splits
 * rejected because K would exceed K_max, out[3] clusters emptied by the label step.
 * Synchronises. */
dpmm_status dpmm_get_counters(dpmm_ctx* ctx, int out[4]);

const char* dpmm_last_error(const dpmm_ctx* ctx);
void dpmm_destroy(dpmm_ctx* ctx);

/* ---- test hooks (used by the parity tests; not needed by an ordinary user) ---- */

/* Set the labels (host arrays, length N) and K; the statistics are recomputed. */
dpmm_status dpmm_set_state(dpmm_ctx* ctx, int K, const int32_t* z, const uint8_t* zbar);

/* Steps a sweep performs: bit 0 parameters (a)-(d), bit 1 labels (e)-(f) and
 * statistics, bit 2 splits and merges.  Default 7.  With bit 0 clear the label
 * step uses the parameters last drawn or set by dpmm_set_params. */
dpmm_status dpmm_set_step_mask(dpmm_ctx* ctx, unsigned mask);

/* Label-step kernel selection (Sec. 4.2, "Two kernels for optimization": the package
 * picks at run time between a hand-written kernel and a library matrix product, from d,
 * N and the GPU).  Here the two label-step kernels of a precision with tensor cores
 * (TF32 and BF16X3 Gaussian, BF16 multinomial) are the tcgen05 kernel and the FP32
 * CUDA-core kernel (the same Gumbel-max draws, scores in FP32 instead of TF32/BF16).
 * choice: DPMM_KERNEL_TENSOR (the default) or DPMM_KERNEL_CUDA_CORE pins one;
 * DPMM_KERNEL_AUTO times both at the next sweep that runs eagerly (the first after
 * this call or after new data): each runs three times on the context's data and
 * stream (CUDA events, the first run a warm-up), the faster is kept for the captured
 * sweep graph, and the choice is cached for the process under (device, prior kind,
 * precision, d, floor(log2 N), K_max), so a context with the same key takes it without
 * timing.  The label step is deterministic given the parameters and the sweep counter,
 * so the timing runs leave the chain as if the chosen kernel had run alone; which
 * kernel wins may differ between GPUs and runs, so pin one where bit-reproducibility
 * across machines matters.  Precisions without a tensor-core kernel keep their only
 * kernel.  Drops the captured graph.  Errors: DPMM_EINVAL for an unknown choice.
 * dpmm_get_kernel: *in_use = the kernel the label step runs (DPMM_KERNEL_TENSOR or
 * DPMM_KERNEL_CUDA_CORE); *ms_tensor, *ms_cuda_core = the timed milliseconds per
 * label step (the cached figures for a cache hit), or -1 when not timed; any output
 * may be NULL. */
typedef enum { DPMM_KERNEL_TENSOR = 0, DPMM_KERNEL_CUDA_CORE = 1, DPMM_KERNEL_AUTO = 2 } dpmm_kernel;
dpmm_status dpmm_set_kernel(dpmm_ctx* ctx, int choice);
dpmm_status dpmm_get_kernel(dpmm_ctx* ctx, int* in_use, float* ms_tensor, float* ms_cuda_core);

/* Parameters of the 3K slots (host arrays), in the data's original coordinates.
 * Gaussian: log weight logw[3K], mean mu[3K x d], precision factor W[3K x d x d]
 * (upper-triangular, Lambda = W W^T) and logdetW[3K] = sum_j log W_jj.
 * Multinomial: logw[3K] and logtheta[3K x d].  Unused pointers may be NULL on get;
 * on set they must match the prior's kind.  set overwrites K. */
dpmm_status dpmm_set_params(dpmm_ctx* ctx, int K, const double* logw, const double* mu, const double* W,
                            const double* logdetW, const double* logtheta);
dpmm_status dpmm_get_params(dpmm_ctx* ctx, double* logw, double* mu, double* W, double* logdetW,
                            double* logtheta);

/* The label step's cluster scores log pi_k + log f(x_i; theta_k) (before the Gumbel
 * perturbation) for the current parameters, computed by this precision's label
 * kernel, into a host array scores[N x K] (K from dpmm_get_info).  The chain's
 * labels are left as they were.  Synchronises. */
dpmm_status dpmm_label_scores(dpmm_ctx* ctx, double* scores);

/* Overwrite the sweep counter (so that a test can replay one sweep index). */
dpmm_status dpmm_set_iter(dpmm_ctx* ctx, uint32_t iter);

/* Kernel timing.  enable = 1 brackets every kernel launch of the sweep with CUDA
 * events on the context's stream; enable = 2 only the label-step kernel; 0 turns
 * it off.  While timing is on, sweeps are launched eagerly (no graph replay).  Each
 * call resets the records.  dpmm_get_profile returns, for up to `cap` entries, the
 * kernel name, its launches and summed device time (ms) since the reset, then one
 * entry "all_kernels" whose launch count is every kernel the library launched since
 * the reset (kernels of a replayed sweep graph included); *count is the number of
 * entries.  Synchronises. */
dpmm_status dpmm_profile(dpmm_ctx* ctx, int enable);
dpmm_status dpmm_get_profile(dpmm_ctx* ctx, int cap, const char** names, int* launches, double* ms, int* count);

/* ---- allocation-free statistics (no counterpart in the paper) ---- */

/* Sufficient statistics of given labels without allocating any memory.  The paper
 * has no counterpart.  It serves callers that cannot allocate device memory where they
 * need the statistics: applications that reserve the GPU's memory up front in their own
 * pool and forbid any later cudaMalloc (a serving process that owns all of HBM, a host
 * framework whose plug-ins must not allocate), and latency-critical code that must not
 * take the implicit device-wide synchronisation a cudaMalloc or cudaFree can cause.
 * The call makes no cudaMalloc, cudaFree or other allocating call.
 *
 * Inputs, all device memory of the current device: X (N x d row-major FP32), z[N]
 * in [0, K) and zbar[N] in {0, 1}.  Outputs, device memory of length 2K, 2K x d and
 * 2K x d x d: for sub-cluster slot 2k + h, n_out = count, sx_out = sum of x,
 * sxx_out = sum of x x^T over the points with (z, zbar) = (k, h), in FP64 (per-tile
 * FP32 sums added in FP64).  Points whose label is outside that range are ignored.
 * The call is asynchronous on `stream` (a cudaStream_t or NULL).
 *
 * Limits: 1 <= d <= 32, 1 <= K <= 16, N >= 1; anything else returns DPMM_EINVAL
 * before any work.  Scratch is a fixed 5.6 MiB array inside the library's device
 * image (held by every GPU that loads the library until the process exits).  The
 * first call on each device (and in each CUDA context) looks up the array's address
 * (cudaGetSymbolAddress) with that device current, so make that first call before any
 * stream capture.  After cudaDeviceReset the next call looks the address up again
 * only if the context handle changed; call it once outside any capture after a reset.
 * All calls on a device share the array and every call overwrites it (it keeps the
 * last call's contents; each call clears what it accumulates into): calls whose kernels
 * overlap on the GPU (other streams, other threads) race and give wrong results;
 * serialise them.  Returns DPMM_ECUDA when a launch fails. */
dpmm_status dpmm_suffstats_noalloc(const float* X, int64_t N, int d, const int32_t* z, const uint8_t* zbar,
                                   int K, double* n_out, double* sx_out, double* sxx_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DPMM_H */
