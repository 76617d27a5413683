/*
 * ls.h -- C ABI of libls, the GB300 (sm_103a) implementation of the Li & Stephens all-vs-all
 * hot path of the kalis paper (arXiv 2212.11403): forward and backward recursions over N
 * independent copying HMMs, posterior decoding and the local distance matrix.
 *
 * Conventions shared by every call
 *   - Loci are 0-based (the paper's variant l is locus l-1 here); haplotypes (recipients i,
 *     donors j) are 0-based.
 *   - Matrices are recipient-major: X[i*N + j] holds the paper's X_ji (the paper's column i,
 *     Sec. 2.1, stored contiguously).  A table over targets [t_from, t_to) stores row r for
 *     target t_from + r.
 *   - rho[l], l = 0..L-2, is the recombination probability of the interval between loci l and
 *     l+1; the forward step l -> l+1 and the backward step l+1 -> l both use it.
 *   - Pointers documented "device" must be CUDA device memory (e.g. a torch tensor's
 *     data_ptr()); "host" pointers are ordinary CPU memory.  The caller owns every pointer it
 *     passes; contexts and tables are owned by the library and freed by the matching destroy.
 *   - Every call that takes a stream enqueues its work on that stream (a cudaStream_t passed as
 *     ls_stream_t; NULL = the legacy default stream) and returns without waiting, unless stated.
 *   - Return value: LS_OK (0), a positive warning, or a negative error; on error nothing was
 *     enqueued and ls_last_error() (per calling thread) describes the cause.
 *   - Floating point: recurrences in FP32, per-target log scales in FP64.
 */
#ifndef LS_H
#define LS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------------------------- */
#define LS_OK 0
#define LS_WARN_UNDERFLOW 1      /* some target hit total underflow (App. A.3); see status_out */
#define LS_WARN_OVERFLOW 2       /* some target hit total overflow (App. A.3); see status_out  */
#define LS_ERR_ARG (-1)          /* bad argument (null pointer, size, range, invalid prior)     */
#define LS_ERR_PARAM_MISMATCH (-2) /* table propagated under another parameter set (Sec. 4.1.2) */
#define LS_ERR_DIRECTION (-3)    /* forward asked to move to an earlier locus, backward to later */
#define LS_ERR_LOCUS_MISMATCH (-4) /* forward and backward tables are not at the same locus     */
#define LS_ERR_RANGE (-5)        /* tables cover different targets / distance needs all targets */
#define LS_ERR_CUDA (-6)         /* a CUDA runtime call failed                                   */
#define LS_ERR_OOM (-7)          /* device memory allocation failed                              */
#define LS_ERR_STATE (-8)        /* parameters not set, or table not initialised                */
#define LS_ERR_DEVICE (-9)       /* a device-side wait ran out its time limit                    */
#define LS_ERR_UNSUPPORTED (-10) /* size or option outside what this build supports              */

/* per-target status bits written to status_out arrays */
#define LS_STATUS_UNDERFLOW 1u   /* a normaliser sum was 0 or subnormal                          */
#define LS_STATUS_OVERFLOW 2u    /* a normaliser sum was not finite                              */
#define LS_STATUS_TIMEOUT 4u     /* a device wait for staged haplotype rows ran out              */

#define LS_FWD 0
#define LS_BWD 1

typedef void* ls_stream_t; /* a cudaStream_t */
typedef struct ls_ctx ls_ctx;
typedef struct ls_table ls_table;
typedef struct ls_ckpt ls_ckpt;
typedef struct ls_mlp ls_mlp;

/* Library version and build description (arch, kernel variants).  Static string. */
const char* ls_version(void);

/* Text of the last error raised on the calling thread ("" if none).  Thread-local storage. */
const char* ls_last_error(void);

/* ---- haplotype cache (Sec. 3.2, Sec. 4.1.1: CacheHaplotypes / QueryCache / CacheSummary) --- */

/* Create a context holding one haplotype data set on the current CUDA device.
 * haps: host uint8 [L][N], variant-major, entries 0/1 (the paper's L x N matrix h, Sec. 2.1).
 * The data are packed on the device into variant-major rows of 32 haplotypes per uint32
 * (haplotype i in bit i%32 of word i/32, Sec. 4.1.1), each row padded to a 16-byte multiple with
 * at least one zero word.  Synchronous.  N >= 2, L >= 1.  *out receives the context. */
int ls_create(ls_ctx** out, const uint8_t* haps, int32_t N, int32_t L);

/* Same, from haplotypes already packed on the device: packed [L][row_words] uint32 in the layout
 * above (row_words >= ceil(N/32)); bits beyond N are ignored.  The data are copied.  Synchronous. */
int ls_create_packed(ls_ctx** out, const uint32_t* packed, int32_t N, int32_t L, int32_t row_words);

/* Free a context and everything it owns (tables created from it must be destroyed first). */
int ls_destroy(ls_ctx* ctx);

/* N, L, words per packed row, and device bytes held by the context (any pointer may be NULL). */
int ls_info(const ls_ctx* ctx, int32_t* N, int32_t* L, int32_t* row_words, size_t* device_bytes);

/* Read haplotypes back from the packed cache: out[a*nh + b] = h at locus loci[a], haplotype
 * haps[b].  All arrays host.  Synchronous. */
int ls_query(const ls_ctx* ctx, const int32_t* loci, int32_t nl, const int32_t* haps, int32_t nh, uint8_t* out);

/* Copy the packed cache to host memory out [L][row_words].  Synchronous. */
int ls_export_packed(const ls_ctx* ctx, uint32_t* out);

/* ---- parameters (Sec. 3.3 Parameters / CalcRho; Sec. 4.1.2) ---------------------------------- */

/* Eq. rho: rho_out[k] = 1 - exp(-Ne * m[k]^gamma), evaluated as -expm1(.).  m in Morgans.
 * Host arrays.  Errors on n < 0, a negative or non-finite m, Ne < 0 or gamma <= 0. */
int ls_calc_rho(const double* m, int32_t n, double Ne, double gamma, double* rho_out);

/* Set the model parameters of a context (Sec. 2.1): rho host double [L-1] with 0 <= rho <= 1;
 * mu host double [mu_len], mu_len 1 (scalar) or L, 0 <= mu <= 1/2; Pi NULL for the uniform
 * prior 1/(N-1), otherwise device float [N][N] recipient-major (Pi[i*N+j] = prior that recipient
 * i copies donor j) with a zero diagonal and rows summing to 1 within 1e-5 (copied).
 * Tables propagated under an earlier parameter set are refused afterwards
 * (LS_ERR_PARAM_MISMATCH).  *hash_out (may be NULL) receives the parameter fingerprint.
 * Synchronous. */
int ls_set_params(ls_ctx* ctx, const double* rho, const double* mu, int32_t mu_len, const float* Pi,
                  uint64_t* hash_out);

/* Storage format of a prior matrix (an option of this library; the paper's Pi is double).
 * LS_PRIOR_FP32 (the default): Pi as the caller's FP32 values.  LS_PRIOR_BF16: ls_set_params
 * rounds every entry of its copy of Pi to the nearest bfloat16 (ties to even) after validating
 * the caller's values, and all kernels then run with the rounded prior, whose rows sum to 1 only
 * within about 2^-9 per entry; the results are those of the rounded matrix.  A target's prior row
 * then fits on chip next to its state for N > 20480 (the large-N kernels keep it in shared memory
 * as bfloat16): a prior matrix with N in (20480, 106496] needs this format (LS_ERR_UNSUPPORTED from
 * the propagation calls otherwise).  Takes effect at the next ls_set_params and enters the
 * parameter fingerprint.  LS_ERR_ARG for another value. */
#define LS_PRIOR_FP32 0
#define LS_PRIOR_BF16 1
int ls_set_prior_format(ls_ctx* ctx, int32_t format);

/* ---- forward / backward tables (Sec. 3.4-3.5, Table tab:fwdbck) ----------------------------- */

/* Create a table (kind LS_FWD or LS_BWD) for targets [t_from, t_to), 0 <= t_from < t_to <= N.
 * The table is uninitialised (no locus): the first ls_forward initialises it at locus 0, the
 * first ls_backward at locus L-1 (Sec. 3.5).  Device memory: (t_to-t_from) * N floats plus one
 * double per target.  Requires parameters to be set. */
int ls_table_create(ls_ctx* ctx, int32_t kind, int32_t t_from, int32_t t_to, ls_table** out);

/* Free a table. */
int ls_table_destroy(ls_table* t);

/* CopyTable: deep copy src into dst (same kind and target range).  Enqueued on stream. */
int ls_table_copy(ls_table* dst, const ls_table* src, ls_stream_t stream);

/* ResetTable: mark the table uninitialised again (no device work). */
int ls_table_reset(ls_table* t);

/* kind, current locus (-1 if uninitialised), target range and parameter fingerprint. */
int ls_table_info(const ls_table* t, int32_t* kind, int32_t* locus, int32_t* t_from, int32_t* t_to,
                  uint64_t* hash);

/* Copy the table's contents to caller device memory: state [T][N] floats (forward: alpha of
 * Eq. fwd1; backward: beta of Eq. bck1, i.e. beta not pre-multiplied by theta) and logscale [T]
 * doubles (forward: log F at the current locus, Eq. F; backward: log G at the current locus,
 * Eq. G, with G = 1 at the last locus).  Either pointer may be NULL.  Enqueued on stream. */
int ls_table_read(const ls_table* t, float* state, double* logscale, ls_stream_t stream);

/* Sizes the propagation calls (ls_forward, ls_backward, ls_checkpoints, ls_run_all and their
 * callers) serve: the uniform prior for N up to 114688 (register-tile kernels to N = 20480, one
 * CTA per target to 57344, two-CTA clusters beyond); a prior matrix up to N = 20480 in either
 * prior format and up to N = 106496 in the BF16 format.  Beyond these the launch planner returns
 * LS_ERR_UNSUPPORTED before anything is enqueued. */

/* Forward (Eq. fwd0, fwd1): propagate fwd in place to locus to_locus >= its current locus
 * (an uninitialised table starts at locus 0).  If n_store > 0, alpha at each locus in
 * store_loci (host int32, strictly increasing, within (current, to_locus]) is written to
 * alpha_out (device float [n_store][T][N]).  status_out (device uint32 [T], may be NULL) is
 * OR-ed with per-target LS_STATUS_* bits.  Errors: LS_ERR_DIRECTION, LS_ERR_PARAM_MISMATCH. */
int ls_forward(ls_ctx* ctx, ls_table* fwd, int32_t to_locus, const int32_t* store_loci, int32_t n_store,
               float* alpha_out, uint32_t* status_out, ls_stream_t stream);

/* Backward (Eq. bck0, bck1): propagate bck in place to locus to_locus <= its current locus
 * (an uninitialised table starts at locus L-1).  store_loci strictly decreasing within
 * [to_locus, current); beta at those loci goes to beta_out [n_store][T][N].  Otherwise as
 * ls_forward. */
int ls_backward(ls_ctx* ctx, ls_table* bck, int32_t to_locus, const int32_t* store_loci, int32_t n_store,
                float* beta_out, uint32_t* status_out, ls_stream_t stream);

/* ---- forward checkpoints and replay ---------------------------------------------------------
 * The paper keeps one locus per table and resumes by propagating again (Sec. 3.5); to revisit
 * earlier loci without a full new pass, ls_checkpoints snapshots alpha at the K = ceil(log2(b-a+1))
 * recursive-bisection loci of [a, b]: c_0 = a and c_k = b - floor((b-a) / 2^k) for k = 1..K-1 (the
 * halving points, densest where a backward sweep starts).  A snapshot is the table's state
 * [T][N] and log F [T] at that locus.  LS_CKPT_F32 keeps alpha exactly; LS_CKPT_F16 stores, per
 * target, s = max_j alpha_j (float) and alpha_j / s rounded to nearest binary16: entries at or
 * above 2^-14 s keep a relative error of at most 2^-11, smaller ones an absolute error of at most
 * 2^-25 s (those below 2^-25 s become 0). */
#define LS_CKPT_F32 0
#define LS_CKPT_F16 1

/* Propagate fwd (an LS_FWD table at a locus <= a, or uninitialised) to locus b, taking the K
 * snapshots on the way; 0 <= a <= b < L.  *out receives a new checkpoint set owning
 * K * T * N * (4 or 2) bytes of device memory (+ K * T * 12 bytes).  status_out as ls_forward.
 * Errors: LS_ERR_DIRECTION (fwd beyond a), LS_ERR_PARAM_MISMATCH, LS_ERR_OOM. */
int ls_checkpoints(ls_ctx* ctx, ls_table* fwd, int32_t a, int32_t b, int32_t dtype, ls_ckpt** out,
                   uint32_t* status_out, ls_stream_t stream);

/* Number of snapshots, their loci (host int32 [K], may be NULL), dtype, target range and the
 * device bytes held. */
int ls_ckpt_info(const ls_ckpt* ck, int32_t* n, int32_t* loci, int32_t* dtype, int32_t* t_from, int32_t* t_to,
                 size_t* device_bytes);

/* Snapshot k decoded to FP32: alpha_out device float [T][N] and logF_out device double [T]
 * (either may be NULL).  Enqueued on stream. */
int ls_ckpt_read(const ls_ckpt* ck, int32_t k, float* alpha_out, double* logF_out, ls_stream_t stream);

/* Replay: set fwd (same context and target range as the checkpoints) to the snapshot with the
 * largest c_k <= locus, decoded to FP32, and propagate it forward to locus (c_0 <= locus < L),
 * whatever fwd held before.  Errors: LS_ERR_RANGE, LS_ERR_PARAM_MISMATCH (the parameters
 * changed since the checkpoints were taken). */
int ls_ckpt_replay(ls_ctx* ctx, const ls_ckpt* ck, ls_table* fwd, int32_t locus, uint32_t* status_out,
                   ls_stream_t stream);

/* Free a checkpoint set. */
int ls_ckpt_destroy(ls_ckpt* ck);

/* PostProbs (Eq. postprob): p_out device float [T][N], p_out[r*N+j] = posterior that target
 * t_from+r copies donor j; p = epsilon (DBL_EPSILON) for every donor if the normaliser is 0;
 * the diagonal is 0.  Both tables must cover the same targets and sit at the same locus
 * (LS_ERR_RANGE / LS_ERR_LOCUS_MISMATCH). */
int ls_posterior(ls_ctx* ctx, const ls_table* fwd, const ls_table* bck, float* p_out, ls_stream_t stream);

/* DistMat (Eq. distmat): d_out device float [N][N], d_ji = -(log(p_ji v eps) + log(p_ij v eps))/2,
 * d_ii = 0, eps = DBL_EPSILON.  Needs tables over all N targets (LS_ERR_RANGE otherwise). */
int ls_distance(ls_ctx* ctx, const ls_table* fwd, const ls_table* bck, float* d_out, ls_stream_t stream);

/* Fused all-vs-all pipeline: forward over all L loci, backward over all L loci, posterior and
 * distance at the D loci decode_loci (host int32, strictly increasing).  d_out [D][N][N] floats,
 * device or host memory (host: the result is copied back before the call returns).  pac_out
 * (host, may be NULL) receives the PAC log-likelihood sum_i log P(h_i | h_-i) (Sec. 1).
 * status_out (device uint32 [N], may be NULL) receives per-target status bits.  Uses library-
 * owned scratch of D*N*N floats (cached in the context).  Synchronous when pac_out is given or
 * d_out is host memory; returns LS_WARN_* when such a call saw underflow/overflow. */
int ls_run_all(ls_ctx* ctx, const int32_t* decode_loci, int32_t D, float* d_out, double* pac_out,
               uint32_t* status_out, ls_stream_t stream);

/* ---- adjoint: gradient of the PAC log-likelihood --------------------------------------------
 * The PAC log-likelihood of targets [t_from, t_to), sum_i log P(h_i | h_-i) (Sec. 1, Eq. F at the
 * last locus), and its gradient with respect to log mu (one scalar scale of every mu_l) and to
 * log rho on K groups of intervals: interval m (between loci m and m+1) belongs to group
 * interval_of[m] (host int32 [L-1], nondecreasing, in [0, K)), and dlogrho[k] is the derivative
 * with respect to a common log-scale of the rho_m of group k.  The paper defines no gradient;
 * this one is the score by the Fisher identity (posterior expectation of the complete-data score
 * of Eq. transition and App. A.3's emission), computed by two forward statistic passes and one
 * backward pass in FP32 with FP64 sums.  Outputs are host doubles (any may be NULL); dlogrho has
 * K entries, 0 for groups without intervals.  Device memory: (3 * (number of nonempty groups) + 2)
 * floats per target and donor, allocated for the call and freed before it returns; the targets
 * are processed in blocks whose scratch stays within 16 GiB (the environment variable
 * LS_GRAD_BUDGET_MB, a positive number of MiB, sets another ceiling; one target is the minimum).
 * Synchronous.  Requires the uniform prior (LS_ERR_UNSUPPORTED otherwise), rho < 1 and mu < 1.
 * Returns LS_WARN_* like ls_run_all. */
int ls_pac_grad(ls_ctx* ctx, int32_t t_from, int32_t t_to, const int32_t* interval_of, int32_t K,
                double* pac_out, double* dlogmu_out, double* dlogrho_out, ls_stream_t stream);

/* ---- learned sparse path: donor proposal, MLP, restricted recursions ------------------------
 * The paper runs every target against all N-1 donors.  This extension restricts target i in
 * window w (256 consecutive loci) to a proposed set S_i^w of K donors: stage 1 keeps the C donors
 * with the fewest mismatches over windows w-1..w+1, stage 2 scores them with a 3-layer MLP
 * (8 -> 256 -> 256 -> 1, ReLU) on the match fractions of windows w-3..w+3 and keeps the K best.
 * The recursions of Eq. fwd1 / Eq. bck1 then run over the sets (prior 1/(N-1) as in the dense
 * chain, continuation only for donors kept across a window change); the donors outside the set
 * are either one pooled state (pool = 1, the default of the Python binding: their mass stays in
 * the normalisers, leaving donors' mass joins the pool and entering donors start from its
 * average) or dropped (pool = 0).  Targets whose forward mass leaves the sets are recomputed
 * densely. */

/* Posterior rows (Eq. postprob) from caller-held alpha and beta rows of targets
 * [t_from, t_from+T): p_out device float [T][N].  Enqueued on stream. */
int ls_posterior_rows(ls_ctx* ctx, const float* alpha, const float* beta, int32_t t_from, int32_t T, float* p_out,
                      ls_stream_t stream);

/* Network parameters as one FP32 vector of LS_MLP_PARAMS floats: W1 [8][256] (input x unit; the
 * eighth input is always 0), b1 [256], W2 [256][256], b2 [256], w3 [256], b3.  params NULL gives
 * a He-uniform initialisation from seed.  The network lives on the current device. */
#define LS_MLP_PARAMS 68353
int ls_mlp_create(const float* params, uint64_t seed, ls_mlp** out);
int ls_mlp_destroy(ls_mlp* m);
int ls_mlp_get(const ls_mlp* m, float* params);
int ls_mlp_set(ls_mlp* m, const float* params);

/* Scores of n feature rows X (device float [n][8]) by the BF16 tensor-core inference kernel
 * (weights and hidden activations rounded to BF16, FP32 accumulation): scores device float [n].
 * Synchronous. */
int ls_mlp_forward(const ls_mlp* m, const float* X, int64_t n, float* scores, ls_stream_t stream);

/* FP32 gradient of the loss sum_r (s_r - y_r)^2 / (2n) over n rows (X [n][8], y [n], device) at
 * the current parameters: grad host float [LS_MLP_PARAMS] (may be NULL), loss host double.
 * Synchronous. */
int ls_mlp_grad(ls_mlp* m, const float* X, const float* y, int32_t n, float* grad, double* loss, ls_stream_t stream);

/* `steps` Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) on minibatches of `batch` rows drawn
 * with replacement by a seeded splitmix64 stream; loss_out = mean minibatch loss over the last
 * tenth of the steps.  Synchronous. */
int ls_mlp_train(ls_mlp* m, const float* X, const float* y, int64_t n, int32_t steps, int32_t batch, float lr,
                 uint64_t seed, double* loss_out, ls_stream_t stream);

/* Stage 1 of window w alone: cand_out device int32 [N][C] (ascending ids, -1 padding) and, if not
 * NULL, feat_out device float [N][C][8] (match fractions of windows w-3..w+3, then 0).
 * Synchronous. */
int ls_propose_window(ls_ctx* ctx, int32_t C, int32_t w, int32_t* cand_out, float* feat_out, ls_stream_t stream);

/* Training labels of the learned proposal (no counterpart in the paper): for the stage-1 candidates
 * cand (device int32 [N][C], as ls_propose_window writes them) and the dense posteriors P (device
 * float [N][N], row i the posterior of target i over donors at the window's middle locus, as
 * ls_posterior_rows writes them), y_out (device float [N][C]) receives
 * y = 1 + log10(max(p, 1e-12)) / 12 (1 for p = 1, 0 at 1e-12 and below), the network's regression
 * target; 0 where cand is -1 (padding) and NaN where an id is >= N.  N is the context's.
 * Synchronous. */
int ls_propose_labels(ls_ctx* ctx, const float* P, const int32_t* cand, int32_t C, float* y_out, ls_stream_t stream);

/* Donor sets for every window: idx_out device int32 [N][ceil(L/256)][K] in ascending id order.
 * With mlp NULL the K donors are stage 1's (C ignored); otherwise stage 1 keeps C (K <= C <= 2048)
 * and the network keeps the K best scores (ties to the lower id).  1 <= K <= 512.  Synchronous. */
int ls_propose(ls_ctx* ctx, int32_t C, int32_t K, const ls_mlp* mlp, int32_t* idx_out, ls_stream_t stream);

/* Sparse forward + backward over donor sets idx (device int32 [N][ceil(L/WS)][K], ascending ids,
 * -1 padding, never the target itself), posteriors and distances at the D decode loci.  Window w
 * runs on S^w (lookahead 0), S^w u S^{w+1} (1: every proposed donor has a window of history when
 * its own window starts) or S^{w-1} u S^w u S^{w+1} (2: proposed donors also stay a window
 * longer); (lookahead + 1) K <= 1536.  With pool = 1 the donors outside the set are carried as one
 * aggregate state with their average emission (allele counts of the locus minus the set's
 * matches), so the normalisers include their mass as in the dense chain; leaving donors' mass
 * joins it and entering donors start from its average.  The posterior at a decode locus is the
 * pooled chain's: normalised over the set and the pool state, every outside donor receiving an
 * equal share of the pool's posterior.
 * d_out device float [D][N][N], complete with pool = 1: d_ij of Eq. distmat from the two targets'
 * posteriors, where an outside donor's posterior is that estimated share; 0 on the diagonal.  With
 * pool = 0 entries with an outside donor on either side are NaN.  Targets whose largest forward
 * mass on donors leaving their set exceeds lost_tol (lost_tol < 0: never) get dense rows (requires
 * N within the dense kernels' range); *n_fallback_out receives their number.
 * trust_out (device uint32 [D][N][ceil(N/32)], may be NULL): bit j % 32 of word j / 32 of row i is 1
 * where d_ij needs no estimate and is within the error budget: both halves come from chain
 * posteriors (j in i's set and i in j's set, or dense rows) and either both targets have dense rows
 * or d_ij <= d_trust.  lost_out device float [N] (may be NULL) receives the lost mass per target;
 * pout_out device float [D][N] (may be NULL) the pooled chain's posterior mass on all outside donors
 * per decode locus and target (0 without a pool; fallback targets keep their sparse value);
 * pac_out the log-likelihood of the restricted chains.  Synchronous.  Uniform prior only. */
int ls_sparse_run_all(ls_ctx* ctx, const int32_t* idx, int32_t K, int32_t WS, int32_t lookahead, int32_t pool,
                      const int32_t* decode_loci, int32_t D, float* d_out, float lost_tol, float* lost_out,
                      double* pac_out, uint32_t* status_out, int32_t* n_fallback_out, float d_trust,
                      uint32_t* trust_out, float* pout_out, ls_stream_t stream);

/* ---- fused pipeline without allocation --------------------------------------------------- */

/* Largest N the allocation-free pipeline's scratch holds: a fixed area inside the library sized
 * for this many targets (LS_NOALLOC_MAX_N x 12 bytes plus a few words, about 768 KB, held by every
 * GPU that loads the library until the process exits).  An N within this bound that no compiled
 * propagation variant serves is refused by the launch planner (LS_ERR_UNSUPPORTED) before anything
 * is enqueued, as in ls_run_all. */
#define LS_NOALLOC_MAX_N 65536

/* The paper has no counterpart to this entry point.  Same computation as ls_run_all (forward and
 * backward over all loci, posterior and symmetrised distances at the D decode loci, the PAC
 * log-likelihood) for callers that must not allocate device memory while they run it: code that
 * is being captured into a CUDA graph (cudaMalloc is not allowed during stream capture), code
 * that lives inside a framework or serving loop owning a fixed device-memory budget, and code for
 * which cudaMalloc's implicit device synchronisation is unacceptable.  It allocates nothing: the
 * caller passes d_out (device float [D][N][N], required, no host buffer) and the optional outputs
 * as for ls_run_all; per-target log scales, status words, the error word and the PAC sum live in
 * the library's fixed scratch area.  The first call on each device looks up that area's device
 * address (cudaGetSymbolAddress) with the context's device current, so make the first call before
 * any stream capture.  All calls share the one area and reuse it: the call clears what must start
 * at zero, and calls whose GPU work overlaps (different streams, or different contexts on one
 * device running at once) race on it.  It launches exactly the kernels ls_run_all launches (the
 * same planner), on the caller's stream only.  N > LS_NOALLOC_MAX_N gives LS_ERR_UNSUPPORTED; D is
 * limited to 64 as for ls_run_all.  Synchronous when pac_out is given (it waits for the PAC sum and
 * returns LS_WARN_* like ls_run_all), asynchronous otherwise.  A device wait that ran out of time
 * is recorded in the scratch area and reported as LS_ERR_DEVICE by the next call that passes
 * pac_out (which then clears the record); calls without pac_out report no device error. */
int ls_run_all_noalloc(ls_ctx* ctx, const int32_t* decode_loci, int32_t D, float* d_out, double* pac_out,
                       uint32_t* status_out, ls_stream_t stream);

/* ---- profiling (tracing hook) ------------------------------------------------------------ */

/* Enable (1) or disable (0) phase timing of ls_run_all on this context.  When enabled, each
 * ls_run_all records CUDA events on its stream before and after its four phases. */
int ls_set_profiling(ls_ctx* ctx, int32_t enable);

/* Device durations of the phases of the last profiled ls_run_all, in milliseconds (ms [4]) and
 * the number of kernels each phase launched (launches [4], may be NULL): 0 forward propagation,
 * 1 backward propagation (with the in-place alpha*beta products at the decode loci), 2 posterior
 * normalisation into half distances, 3 symmetrisation.  Waits for the last recorded event. */
int ls_profile_read(ls_ctx* ctx, float* ms, int32_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* LS_H */
