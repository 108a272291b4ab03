/*
 * hawkes.h -- C ABI of libhawkes, a GB300 (sm_103a) implementation of the
 * spatiotemporal Hawkes log-likelihood of Holbrook, Ji & Suchard ("Bayesian
 * mitigation of spatial coarsening for a Hawkes model applied to gunfire,
 * wildfire and viral contagion") and of its gradients, together with the
 * HMC trajectory over event locations that calls them.
 *
 * Model (Section 2.1).  Events (x_n, t_n), x_n in R^D, t_n >= 0, n = 1..N.
 *   lambda_n = sum_{n'} mu_{nn'} + xi_{nn'}                         (Eq. (1))
 *   mu_{nn'} = mu0 / (tau_x^D tau_t) phi((x_n-x_n')/tau_x) phi((t_n-t_n')/tau_t) I[t_n != t_n']
 *   xi_{nn'} = theta omega / h^D exp(-omega (t_n-t_n')) phi((x_n-x_n')/h) I[t_n' < t_n]
 *   Lambda_n = mu0 [Phi((T-t_n)/tau_t) - Phi(-t_n/tau_t)] + theta [1 - exp(-omega (T-t_n))]
 *   ell      = sum_n log lambda_n - sum_n Lambda_n,  T = max_n t_n     (Eq. (1))
 * phi is the standard normal density (D-variate for space), Phi its CDF.
 * The location gradient is the one of Appendix A (its sigma_x is h):
 *   d ell/d x_n = sum_{n'} [ (mu_{nn'}/lambda_n + mu_{n'n}/lambda_n') / tau_x^2
 *                          + (xi_{nn'}/lambda_n + xi_{n'n}/lambda_n') / h^2 ] (x_n' - x_n)
 * The parameter gradient differentiates the same expressions with respect to
 * Theta = (mu0, tau_x, tau_t, theta, omega, h).
 *
 * Conventions shared by every entry point.
 *   - Arrays named t, X, grad, p, box_* are DEVICE pointers owned by the
 *     caller; X is row-major N x D (event n occupies X[n*D .. n*D+D-1]).
 *     Times need not be sorted; outputs follow the caller's event order.
 *   - hawkes_params and host-side index arrays are HOST pointers, read
 *     before the call returns.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream) and the call returns without waiting for it.  Scalar
 *     results are written to device memory.
 *   - The returned status reports argument errors found on the host.
 *     Errors found on the device (non-finite or negative inputs, a zero
 *     rate) are recorded in a sticky per-context
 *     device status; hawkes_ctx_sync_status() waits for the stream and
 *     returns it.  Outputs of a call that records a device error are NaN.
 *   - A context is used by one host thread at a time; calls that share a
 *     context must be issued on one stream, or ordered by the caller.
 *   - No C++ exception crosses this interface; hawkes_last_error() returns a
 *     message for the last failure on a context.
 */
#ifndef HAWKES_H
#define HAWKES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Theta of Section 2.1, in the paper's order.  All six must be finite and
 * strictly positive (omega, h and theta are stated as strictly positive in
 * Section 2.1; mu0 and the bandwidths carry truncated priors on (0, inf)). */
typedef struct {
    double mu0, tau_x, tau_t, theta, omega, h;
} hawkes_params;

typedef enum {
    /* FP32 pairwise kernel values and squared distances, compensated FP32
     * row sums, FP64 logs, integrated rate, reductions and HMC update. */
    HAWKES_PREC_MIXED = 0,
    /* Every operation in FP64. */
    HAWKES_PREC_FP64 = 1
} hawkes_precision;

/* Element type of an input array that may be given in either precision. */
typedef enum {
    HAWKES_F64 = 0, /* double */
    HAWKES_F32 = 1  /* float */
} hawkes_dtype;

typedef enum {
    HAWKES_OK = 0,
    HAWKES_ERR_INVALID_ARG = 1,  /* bad size, pointer, parameter or option   */
    HAWKES_ERR_ZERO_RATE = 2,    /* some lambda_n == 0: ell = -inf, grad NaN */
    HAWKES_ERR_CUDA = 3,         /* a CUDA runtime call failed               */
    /* 4 is unused: no kernel of the library waits on another CTA, stream or
     * device, so there is no device-side wait that could time out.         */
    HAWKES_ERR_OOM = 5,          /* device workspace could not be allocated  */
    HAWKES_ERR_INVALID_DATA = 6  /* non-finite X or t, or some t_n < 0       */
} hawkes_status;

typedef struct hawkes_ctx hawkes_ctx;
typedef void *hawkes_stream; /* cudaStream_t */

/* ------------------------------------------------------------ context -- */

/* Create a context on CUDA device `device` whose device workspace holds
 * mixed-precision problems of up to max_n events (summed over the sets of a
 * batch) in up to max_d <= 8 dimensions.  Larger calls grow the workspace on
 * demand, which allocates device memory at that call; so does the first
 * HAWKES_PREC_FP64 call.  The workspace is O(n): about 0.5 KB per event in
 * the arrays kept per event, plus the pair kernels' partial sums, which
 * take at most max(1 GiB, four slots) where a slot is (vpc + d) floats per
 * event on the mixed path (vpc = 1, 2 or 6 rate sums) and (6 + d) doubles on
 * the FP64 path (see HAWKES_OPT_PARTIAL_SLOTS).  On success *ctx owns the
 * workspace until hawkes_ctx_destroy. */
hawkes_status hawkes_ctx_create(hawkes_ctx **ctx, int32_t device, int64_t max_n, int32_t max_d);

/* Release a context and its device memory.  The caller must have finished
 * (synchronized) all work enqueued on it.  NULL is accepted. */
void hawkes_ctx_destroy(hawkes_ctx *ctx);

/* Message for the last failure on ctx ("" if none); valid until the next
 * call on ctx.  A NULL ctx returns the message of the last failed create. */
const char *hawkes_last_error(const hawkes_ctx *ctx);

/* Wait for `stream`, then return and clear the sticky device status of ctx
 * (HAWKES_OK if no device-side error was recorded since the last check). */
hawkes_status hawkes_ctx_sync_status(hawkes_ctx *ctx, hawkes_stream stream);

/* Tuning and profiling options (hawkes_ctx_set_option):
 *   HAWKES_OPT_BLOCK_WARPS   row groups of warps per CTA of the mixed pair
 *                            kernels, which set the pair block size (32 x
 *                            rows-per-lane x row groups events; 0 = tuned)
 *   HAWKES_OPT_COL_GROUPS    column groups of warps per CTA of the rate and
 *                            gradient passes, which split each pair block's
 *                            columns (1, 2 or 4, with row groups x column
 *                            groups <= 8; 0 = chosen per pass: the most that
 *                            keep blocks x warps within 48 per SM, so that
 *                            small problems still fill the SMs with warps)
 *   HAWKES_OPT_CTAS_PER_SM   persistent CTAs per SM (0 = occupancy limit)
 *   HAWKES_OPT_PROFILE       1: time every pair-kernel launch with events
 *   HAWKES_OPT_TIMES_SORTED  1: the caller promises t is non-decreasing and
 *                            the time sort is skipped (checked on device)
 *   HAWKES_OPT_MIXED_FIXUP_EXP  log2 of the rate threshold below which a
 *                            row of the mixed path is recomputed in FP64
 *                            (default -76, range [-120, 0])
 *   HAWKES_OPT_SKIP_FAR_BLOCKS  1: the mixed path skips pair blocks whose
 *                            time gap makes every kernel value underflow
 *                            FP32 (exponent <= -130 for both terms); their
 *                            contribution is exactly zero, so results are
 *                            bit-identical to the dense evaluation, but the
 *                            number of pairs evaluated depends on the data
 *                            (default 0: every pair is evaluated)
 *   HAWKES_OPT_FP64_ORDERED  1: the FP64 path evaluates every ordered pair
 *                            with CUDA's exp() in a few column splits;
 *                            0 (default): each unordered pair once, with a
 *                            table-driven FP64 exp2 (Tang's method)
 *   HAWKES_OPT_ONE_LAUNCH    1: a batch whose sets have several dimensions
 *                            runs each mixed pair pass as one persistent
 *                            launch over every set's pair blocks (each block
 *                            dispatched on its set's dimension; one shape and
 *                            the largest register count of all dimensions);
 *                            0 (default): one persistent launch per
 *                            dimension, the launches on forked streams so
 *                            that they overlap; results are the same within
 *                            the mixed tolerances (block sizes may differ)
 *   HAWKES_OPT_PARTIAL_SLOTS the cap G on the partial sums each event keeps
 *                            between the pair kernels and the finalize
 *                            kernels.  The pair blocks of a set with nb
 *                            blocks are dealt out in nb | 1 rounds that touch
 *                            every block once; the first G rounds store slots
 *                            0 .. G-1, and each further G rounds ("phase")
 *                            run as another launch that stores G scratch
 *                            slots, which a fold kernel adds into the first
 *                            G: a fixed order, so results stay
 *                            deterministic.  0 (default): every round its
 *                            own slot while all slots fit 1 GiB, else as many
 *                            slots and scratch slots as fit (at least enough
 *                            for 16 pair blocks per SM in each phase).  A
 *                            different G changes the order of the sums
 *                            (results within rounding)
 *   HAWKES_OPT_BMDS_FUSED    1: a mixed-precision BMDS-Hawkes HMC
 *                            trajectory evaluates the BMDS gradient inside
 *                            the Hawkes gradient pass (one pair loop for both
 *                            terms, from a time-ordered FP32 copy of Y that
 *                            the call makes: 4 npad^2 bytes of device
 *                            memory) and runs the BMDS kernels only for
 *                            ell_B at the trajectory's two ends; 0 (default,
 *                            as fast or faster on GB300 at D = 6 from 4,733
 *                            to 20,000 events): the BMDS kernels (the
 *                            gradient alone between the ends) run beside
 *                            every Hawkes evaluation on a second stream  */
enum {
    HAWKES_OPT_BLOCK_WARPS = 1,
    HAWKES_OPT_CTAS_PER_SM = 2,
    HAWKES_OPT_PROFILE = 3,
    HAWKES_OPT_TIMES_SORTED = 4,
    HAWKES_OPT_MIXED_FIXUP_EXP = 5,
    HAWKES_OPT_SKIP_FAR_BLOCKS = 6,
    HAWKES_OPT_FP64_ORDERED = 7,
    HAWKES_OPT_COL_GROUPS = 8,
    HAWKES_OPT_ONE_LAUNCH = 9,
    HAWKES_OPT_PARTIAL_SLOTS = 10,
    HAWKES_OPT_BMDS_FUSED = 11
};
hawkes_status hawkes_ctx_set_option(hawkes_ctx *ctx, int32_t option, int64_t value);

/* Kernel timing collected while HAWKES_OPT_PROFILE is on (waits for the
 * recorded events).  kernel: 0 = rate pass (lambda row sums), 1 = gradient
 * pass, 2 = validation + time sort + packing, 3 = rate finalization (ell,
 * with the FP64 recompute of rows whose mixed-precision rate underflows),
 * 4 = gradient finalization.  Returns the summed device time in ms, the
 * number of launches and the number of unordered event pairs those launches
 * processed (0 for stages 2-4). */
hawkes_status hawkes_ctx_kernel_stats(hawkes_ctx *ctx, int32_t kernel, double *total_ms,
                                      int64_t *launches, double *pairs);
hawkes_status hawkes_ctx_reset_stats(hawkes_ctx *ctx);

/* Number of kernel launches this context has enqueued since creation (or
 * the last reset_stats): `own` counts the library's hand-written kernels,
 * `library` the launches of the CUB radix sort used for the time order
 * (counted as one per sort call). */
hawkes_status hawkes_ctx_launch_count(const hawkes_ctx *ctx, int64_t *own, int64_t *library);

/* ----------------------------------------------------------- autotuner -- */

/* Tile shape of the mixed pair kernels for one dimension d and one size
 * bucket (bucket = ceil(log2 n)): row groups of warps per CTA (1, 2, 4 or 8;
 * the pair block is 32 x rows-per-lane x row groups events square), column
 * groups (1, 2 or 4, splitting the block's columns over more warps; 0 =
 * chosen per pass as for HAWKES_OPT_COL_GROUPS; row groups x column groups
 * <= 8) and the cap on persistent CTAs
 * per SM (0 = as many as fit).  Entries set here or found by hawkes_autotune
 * are used whenever HAWKES_OPT_BLOCK_WARPS / HAWKES_OPT_CTAS_PER_SM are 0
 * and the entry still leaves three pair blocks per SM at the call's size. */
hawkes_status hawkes_ctx_set_tuning(hawkes_ctx *ctx, int32_t d, int32_t bucket, int32_t warps, int32_t col_groups,
                                    int32_t ctas_per_sm);
hawkes_status hawkes_ctx_get_tuning(const hawkes_ctx *ctx, int32_t d, int32_t bucket, int32_t *warps,
                                    int32_t *col_groups, int32_t *ctas_per_sm);

/* Time every tile shape (row groups, column groups, CTA cap) for the
 * caller's data (t, X as in hawkes_loglik_grad_locations; mixed precision)
 * with CUDA events on `stream`, store the fastest for (d, bucket of n) in
 * the context, and return it.  The options it sets while timing are put
 * back.  Allocates (and frees) one output buffer and synchronizes the
 * stream; out_ms (nullable) receives the fastest evaluation time. */
hawkes_status hawkes_autotune(hawkes_ctx *ctx, const double *t, const double *X, int64_t n, int32_t d,
                              const hawkes_params *params, hawkes_stream stream, int32_t *best_warps,
                              int32_t *best_col_groups, int32_t *best_ctas_per_sm, double *out_ms);

/* ------------------------------------------------------- log-likelihood -- */

/* ell(X, t | Theta) of Eq. (1).
 *   t: device [n] event times (>= 0, finite), any order.
 *   X: device [n*d] locations, row-major.
 *   n >= 1, 1 <= d <= 8.
 *   out_loglik: device [1].  A zero rate (e.g. n = 1, or an event tied in
 *   time with every other) gives -inf and status OK. */
hawkes_status hawkes_loglik(hawkes_ctx *ctx, const double *t, const double *X, int64_t n, int32_t d,
                            const hawkes_params *params, hawkes_precision prec, hawkes_stream stream,
                            double *out_loglik);

/* ell of Eq. (1) and its gradient with respect to every location
 * (Appendix A), optionally with respect to Theta.
 *   out_grad_X: device [n*d], row-major, in the caller's event order.
 *   out_grad_params: device [6] in Theta order, or NULL to skip.
 * A zero rate records HAWKES_ERR_ZERO_RATE in the device status, writes
 * ell = -inf and fills the gradients with NaN. */
hawkes_status hawkes_loglik_grad_locations(hawkes_ctx *ctx, const double *t, const double *X, int64_t n,
                                           int32_t d, const hawkes_params *params, hawkes_precision prec,
                                           hawkes_stream stream, double *out_loglik, double *out_grad_X,
                                           double *out_grad_params);

/* Probability that each event arises from self-excitation under the given
 * state, xi(x_n, t_n) / (xi(x_n, t_n) + mu(x_n, t_n)) = Xi_n / lambda_n
 * (Section 4.3; its posterior mean over MCMC states is the caller's
 * average).  out_prob: device [n] in the caller's event order; NaN for an
 * event whose rate is zero. */
hawkes_status hawkes_self_excitation_prob(hawkes_ctx *ctx, const double *t, const double *X, int64_t n, int32_t d,
                                          const hawkes_params *params, hawkes_precision prec, hawkes_stream stream,
                                          double *out_prob);

/* ----------------------------------------------------------------- BMDS -- */

/* Bayesian multidimensional scaling likelihood of Section 2.2.3, Eq. (4):
 * observed distances y_nn' are truncated-normal around the latent distances
 * delta_nn' = |x_n - x_n'| with variance sigma2, truncated to y > 0,
 *   ell_B = N (1 - N) / 4 log(sigma2)
 *           - sum_{n > n'} [ (y_nn' - delta_nn')^2 / (2 sigma2) + log Phi(delta_nn' / sigma) ],
 * and its gradients with respect to every location and to sigma2.  With
 * ell of Eq. (1) it forms the BMDS-Hawkes log-posterior whose HMC over the
 * locations (Section 3) needs both gradients.
 *   Y:  device [n*n] row-major, of type y_type (HAWKES_F64: double,
 *       HAWKES_F32: float); only the entries below the diagonal
 *       (Y[n*N + n'], n > n') are read, the rest may hold anything.  Each
 *       must be finite and >= 0 (else the device status records
 *       HAWKES_ERR_INVALID_DATA and every output is NaN).  The mixed
 *       precision rounds FP64 distances to FP32 as it reads them, so a float
 *       copy of Y (made once by the caller, Y being data) gives the same
 *       results from half the memory traffic; HAWKES_PREC_FP64 widens float
 *       distances exactly.
 *   X:  device [n*d] locations, row-major; 1 <= d <= 8, 1 <= n <= 2^30.
 *   sigma2 > 0, finite.
 *   out_loglik: device [1];  out_grad_X: device [n*d] row-major or NULL;
 *   out_grad_sigma2: device [1] or NULL.
 * Coincident locations (delta = 0) contribute their value terms and no
 * gradient term (|x_n - x_n'| has no derivative there; 0 is the symmetric
 * subgradient).  HAWKES_PREC_MIXED evaluates each pair in FP32 (locations
 * split into FP32 hi/lo parts) and adds the partial sums in FP64;
 * HAWKES_PREC_FP64 does every operation in FP64.  Results are
 * deterministic.  The call uses a workspace of
 * hawkes_bmds_workspace_bytes(n, d, prec) bytes (about n^2 (d + 1) / 32
 * bytes in the mixed precision for n >= 8192), which the context allocates
 * on first use and keeps at the largest size seen. */
hawkes_status hawkes_bmds_loglik_grad(hawkes_ctx *ctx, const void *Y, hawkes_dtype y_type, const double *X, int64_t n,
                                      int32_t d, double sigma2, hawkes_precision prec, hawkes_stream stream,
                                      double *out_loglik, double *out_grad_X, double *out_grad_sigma2);

/* Device workspace (bytes) that hawkes_bmds_loglik_grad needs for (n, d,
 * prec): one partial-sum slot per tile pair and a few per-CTA sums.
 * Returns 0 for arguments outside the ranges above. */
size_t hawkes_bmds_workspace_bytes(int64_t n, int32_t d, hawkes_precision prec);

/* ------------------------------------------------ Metropolis-within-Gibbs -- */

/* Incremental log-likelihood changes for the block-wise Metropolis-Hastings
 * updates of the event locations (Section 3).  A state holds copies of t and
 * X and the rates lambda_n of Eq. (1) in FP64.  Moving a block B of events to
 * new locations changes only the pair terms that involve B, so
 *   Delta ell = ell(X with x_b -> x*_b, b in B) - ell(X)
 *             = sum_n [log lambda*_n - log lambda_n]
 * costs O(|B| N) pair evaluations instead of the O(N^2) of a full evaluation
 * (the integrated rate does not depend on X).  Rates, logs and decisions
 * are FP64, and so are the pair terms unless hawkes_mwg_set_precision
 * selects FP32 for them; calls enqueue on `stream`, allocate nothing after hawkes_mwg_create and read
 * nothing back to the host (the accept decision and the commit happen on the
 * device), so a sequence of steps may be captured in a CUDA graph.  Use one
 * stream per state.  Device-side data errors (an index out of range or
 * repeated within a block, a non-finite proposal, invalid t or X at
 * creation) make Delta ell NaN, reject every step, and are reported and
 * cleared by hawkes_mwg_sync_status. */
typedef struct hawkes_mwg hawkes_mwg;

/* Create a state on `device` from device arrays t [n] (>= 0, finite) and X
 * [n*d] (row-major, finite), copying both; computes every lambda_n in FP64
 * (O(n^2), enqueued on `stream`).  max_block (1..256) bounds the block size of
 * later proposals.  Returns HAWKES_ERR_INVALID_ARG for bad sizes or
 * parameters, HAWKES_ERR_OOM if device memory runs out. */
hawkes_status hawkes_mwg_create(int32_t device, const double *t, const double *X, int64_t n, int32_t d,
                                const hawkes_params *params, int32_t max_block, hawkes_stream stream,
                                hawkes_mwg **out);
void hawkes_mwg_destroy(hawkes_mwg *s);
const char *hawkes_mwg_last_error(const hawkes_mwg *s);

/* Delta ell of moving events idx[0..nb) (device int64, distinct, in [0, n))
 * to X_new (device [nb*d]); the state is not changed.  out_delta: device [1].
 * Delta ell is +inf when the move makes a zero rate positive, and a rate that
 * stays zero contributes 0.  0 <= nb <= max_block. */
hawkes_status hawkes_mwg_delta(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *X_new,
                               hawkes_stream stream, double *out_delta);

/* One Metropolis-Hastings step with the same proposal: accept iff
 * log_u < Delta ell + log_q_ratio (device scalars; log_q_ratio =
 * log q(x|x*) - log q(x*|x) of the caller's proposal, NULL for a symmetric
 * one; a NaN on either side rejects).  On accept the moved locations, the
 * rates and the running ell are updated.  out_delta (device [1]) and
 * out_accepted (device int32 [1]) may be NULL. */
hawkes_status hawkes_mwg_step(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *X_new,
                              const double *log_q_ratio, const double *log_u, hawkes_stream stream,
                              double *out_delta, int32_t *out_accepted);

/* Proposals for the block idx[0..nb) from the state's current locations,
 * written to X_new (device [nb*d]) with the block's log q-ratio
 * log q(x|x*) - log q(x*|x) in *log_q_ratio (device [1]), ready for
 * hawkes_mwg_step.  Random numbers are the caller's uniforms in (0, 1).
 *
 * Circle priors (Eq. (3), D = 2 only): event m has prior centre
 * centers[2m..2m+1] and radius radii[m] (device arrays over all n events).
 * The proposal of Eq. (6) is uniform on the lens between the prior circle and
 * the disc of radius radii[m]*eps around the current point, drawn by
 * rejection: try k takes radius r eps sqrt(u[(b*tries+k)*2]) and angle
 * 2 pi u[(b*tries+k)*2+1] (u: device [nb*tries*2]); the first draw inside the
 * circle is the proposal, and if every try misses the event stays.  With
 * A(x) the lens area (closed form) and P(x) = 1 - (1 - A/(pi (r eps)^2))^tries
 * the chance that some try lands, the ratio sums
 * log(P(x*)/A(x*)) - log(P(x)/A(x)) over the events that move, which keeps
 * the chain exact for any number of tries. */
hawkes_status hawkes_mwg_propose_circle(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *centers,
                                        const double *radii, double eps, int32_t tries, const double *u,
                                        hawkes_stream stream, double *X_new, double *log_q_ratio);

/* Box priors (Eq. (2)): coordinate k of event m lies in [lo[m*d+k],
 * hi[m*d+k]] (device arrays over all n events); the proposal is N(x_k, sd^2)
 * truncated to the box, drawn by inverse CDF from u[b*d+k] (device
 * [nb*d]); the ratio is sum log Z(x) - log Z(x*) with
 * Z(y) = Phi((hi - y)/sd) - Phi((lo - y)/sd). */
hawkes_status hawkes_mwg_propose_box(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *lo,
                                     const double *hi, double sd, const double *u, hawkes_stream stream,
                                     double *X_new, double *log_q_ratio);

/* Recompute every rate and ell from the current locations (O(n^2)); the
 * incremental updates accumulate rounding over many accepted steps. */
hawkes_status hawkes_mwg_refresh(hawkes_mwg *s, hawkes_stream stream);

/* Precision of the pair terms in later delta and step calls (a state starts
 * in HAWKES_PREC_FP64).  HAWKES_PREC_MIXED evaluates them in FP32: FP32
 * (hi, lo) copies of X and t (made on `stream` by this call and kept up to
 * date by accepted steps), differences (hi - hi) + (lo - lo), the MUFU
 * exponential with the prefactor as an FP32 factor, compensated FP32 sums,
 * exact time comparisons; the rates, logs, Delta ell and the decision stay
 * FP64.  An unmoved event takes the FP64 path where its rate is below
 * max(prefactors) 2^-60 (FP32 terms could underflow) or where the move takes
 * away all but 1/1024 of it (the FP32 error would be magnified); a moved
 * event whose new rate is below that bound is recomputed in FP64.  The
 * relative error of each new rate is then a few 2^-24 times (1 + the
 * exponent of its dominant terms); refresh more often than in FP64.  When
 * some |x| or t is 2^100 or more the state keeps evaluating in FP64, and a
 * proposal coordinate of that size counts as a bad proposal.  Returns
 * HAWKES_ERR_INVALID_ARG when a kernel prefactor or scale (times log2 e)
 * lies outside [2^-100, 2^100]. */
hawkes_status hawkes_mwg_set_precision(hawkes_mwg *s, hawkes_precision prec, hawkes_stream stream);

/* Copy the current locations (device [n*d]), rates (device [n]) and running
 * ell (device [1]) out; any pointer may be NULL. */
hawkes_status hawkes_mwg_read(hawkes_mwg *s, hawkes_stream stream, double *X_out, double *lam_out,
                              double *out_loglik);

/* Synchronize `stream`, then report and clear the state's device status. */
hawkes_status hawkes_mwg_sync_status(hawkes_mwg *s, hawkes_stream stream);

/* ------------------------------------------------------------------ HMC -- */

/* One Hamiltonian Monte Carlo proposal over all locations (Section 3: HMC
 * over X, after Neal 2011) with potential U = -ell, identity mass matrix,
 * and n_steps leapfrog steps of size eps:
 *   p += eps/2 grad ell(X);  X += eps p;  reflect at box walls;  p += eps/2 grad ell(X)
 * (the gradient at the end of one step is reused at the start of the next).
 * Reflection mirrors a coordinate that left [lo, hi] back across the wall it
 * crossed and flips its momentum, repeatedly (at most 1000 times, else the
 * proposal is rejected).  Box walls carry the uniform location priors of
 * Eq. (2); pass box_lo = box_hi = NULL for unconstrained locations.
 *   X_inout: device [n*d]; replaced by the proposal when accepted.
 *   p0:      device [n*d] initial momenta (drawn by the caller).
 *   log_u:   device [1] log of the caller's uniform draw; the proposal is
 *            accepted iff log_u < H0 - H1 with H = -ell + |p|^2/2 (FP64) and
 *            H1 finite.
 *   out_H0, out_H1: device [1];  out_accepted: device int32 [1].
 * The L-step trajectory runs as one CUDA graph cached in the context (keyed
 * by n, d, n_steps, precision, the presence of boxes, the workspace, the
 * options that shape its launches and the plan's pair launches); the first
 * call with a new key captures it. */
hawkes_status hmc_leapfrog_trajectory(hawkes_ctx *ctx, const double *t, double *X_inout, const double *p0,
                                      const double *box_lo, const double *box_hi, int64_t n, int32_t d,
                                      const hawkes_params *params, double eps, int32_t n_steps,
                                      const double *log_u, hawkes_precision prec, hawkes_stream stream,
                                      double *out_H0, double *out_H1, int32_t *out_accepted);

/* One HMC proposal over the latent locations of the BMDS-Hawkes model
 * (Section 2.2.3 and Section 3, the influenza application): potential
 * U = -ell (Eq. (1)) - ell_B (Eq. (4), distances Y of type y_type, variance
 * sigma2; see hawkes_bmds_loglik_grad), unconstrained locations, otherwise
 * as hmc_leapfrog_trajectory (same arguments, H = U + |p|^2/2, one CUDA
 * graph per shape cached in the context; the cache key includes Y's address
 * and sigma2).  Each leapfrog step evaluates both gradients: the BMDS
 * kernels run on the locations in the caller's order and their gradient is
 * added to the Hawkes gradient before the kicks.  Both terms use `prec`. */
hawkes_status hawkes_bmds_hmc_trajectory(hawkes_ctx *ctx, const double *t, double *X_inout, const double *p0,
                                         int64_t n, int32_t d, const hawkes_params *params, const void *Y,
                                         hawkes_dtype y_type, double sigma2, double eps, int32_t n_steps,
                                         const double *log_u, hawkes_precision prec, hawkes_stream stream,
                                         double *out_H0, double *out_H1, int32_t *out_accepted);

/* One HMC proposal for each of n_sets independent sets (laid out as in
 * hawkes_batch_loglik_grad), all advanced by one CUDA graph per shape: the
 * leapfrog of hmc_leapfrog_trajectory with each set's own step size, box
 * walls, Hamiltonian and accept decision.
 *   eps: HOST [n_sets] step sizes;  log_u: device [n_sets];
 *   X_inout, p0, box_lo, box_hi: device, laid out like X;
 *   out_H0, out_H1: device [n_sets];  out_accepted: device int32 [n_sets].
 * Each set's rows are replaced by its proposal when that set accepts. */
hawkes_status hawkes_batch_hmc_trajectory(hawkes_ctx *ctx, int32_t n_sets, const int64_t *offsets,
                                          const int32_t *dims, const double *t, double *X_inout, const double *p0,
                                          const double *box_lo, const double *box_hi, const hawkes_params *params,
                                          const double *eps, int32_t n_steps, const double *log_u,
                                          hawkes_precision prec, hawkes_stream stream, double *out_H0,
                                          double *out_H1, int32_t *out_accepted);

/* ------------------------------------------------------------- batched -- */

/* Log-likelihoods and location gradients of n_sets independent data sets
 * in one pass: set b has n_b = offsets[b+1]-offsets[b] events of dimension
 * dims[b] and parameters params[b].  offsets (n_sets+1 entries, offsets[0]
 * = 0), dims and params are HOST arrays.
 *   t: device, the sets' times back to back (offsets index it).
 *   X: device, the sets' locations back to back, each set row-major with its
 *      own width: set b starts at element sum_{b'<b} n_b' * dims[b'].
 *   out_loglik: device [n_sets];  out_grad_X: device, laid out like X.
 * Every set's rows are pair-evaluated by one persistent launch per distinct
 * dimension, with work items from all sets of that dimension balanced over
 * the SMs. */
hawkes_status hawkes_batch_loglik_grad(hawkes_ctx *ctx, int32_t n_sets, const int64_t *offsets,
                                       const int32_t *dims, const double *t, const double *X,
                                       const hawkes_params *params, hawkes_precision prec,
                                       hawkes_stream stream, double *out_loglik, double *out_grad_X);

/* ------------------------------------------------------ no allocation -- */

/* The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory.  Code hosted by a framework or plugin
 * system that owns every device allocation (a pool that a raw cudaMalloc
 * would bypass), and real-time or embedded callers that forbid allocation
 * after start-up, cannot create a hawkes_ctx, whose workspace is allocated.
 *
 * hawkes_loglik_noalloc computes the same log-likelihood as hawkes_loglik
 * in HAWKES_PREC_FP64 (every operation in double, here over ordered pairs)
 * for up to HAWKES_NOALLOC_MAX_N events, and calls no cudaMalloc, cudaFree or
 * allocating library routine.  Its scratch is a fixed array of
 * HAWKES_NOALLOC_MAX_N * 16 + 32 doubles (about 1 MiB) in the library's
 * static device memory, which every GPU that loads the library holds until
 * the process exits.
 *   t, X: device [n], [n*d] (row-major), on the calling thread's current
 *         CUDA device; any time order.  1 <= n <= HAWKES_NOALLOC_MAX_N,
 *         1 <= d <= 8; larger n returns HAWKES_ERR_INVALID_ARG.
 *   out_loglik: device [1]; -inf for a zero rate; NaN when some t_n is
 *         negative or not finite or some coordinate is not finite.
 * Work is enqueued on `stream`.  The first call in each CUDA context (the
 * device's primary context, or a context the caller made current) looks up
 * the device address of the scratch array in that context
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Every call in a context shares the one scratch array and leaves its
 * contents behind; the status word is cleared by each call.  Calls whose work
 * overlaps on the GPU (different streams, no ordering between them) race and
 * give wrong results. */
#define HAWKES_NOALLOC_MAX_N 8192
hawkes_status hawkes_loglik_noalloc(const double *t, const double *X, int64_t n, int32_t d,
                                    const hawkes_params *params, hawkes_stream stream, double *out_loglik);

/* ------------------------------------------------------------ probing -- */

/* Measure, on `device`, how many FP32 fused multiply-adds and how many MUFU
 * ex2 (ex2.approx.ftz.f32) results one SM completes per clock, and the SM
 * clock during the measurement (MHz).  The pair kernels are bound by these
 * two pipes; the benchmark derives their roofline from this measurement.
 * Runs two short kernels and synchronizes the device. */
hawkes_status hawkes_probe_pipe_rates(int32_t device, double *fma_per_sm_clk, double *ex2_per_sm_clk,
                                      double *sm_clock_mhz);

/* FP64 FMA results per SM per clock on `device` (independent chains): the
 * whole kernel is timed with events and divided by the SM clock, read from
 * the clock counter against the global timer.  On this GPU DADD and DMUL
 * run at the same rate, so this is the rate that bounds the FP64 precision
 * path.  Synchronizes the device. */
hawkes_status hawkes_probe_dfma_rate(int32_t device, double *dfma_per_sm_clk);

/* Evaluate the base-2 exponential of the FP64 pair terms (Tang's
 * table-driven method: a 2048-entry table of 2^(j/2048) and a degree-3 Taylor
 * polynomial of 2^f - 1 for |f| <= 2^-12) at n arguments, so that it can be
 * checked against the host's exp2:  out[i] = 2^y[i] for y[i] <= 0, rounded
 * once also where the result is subnormal; y[i] < -1100 (-inf included)
 * gives 0 and y[i] > 0 gives 1.  y, out: device arrays of n doubles on the
 * current device; work is enqueued on `stream`.  n = 0 does nothing; n < 0
 * or a null array returns HAWKES_ERR_INVALID_ARG. */
hawkes_status hawkes_probe_exp2_fp64(const double *y, double *out, int64_t n, hawkes_stream stream);

/* Library version, e.g. "hawkes 0.1.0 sm_103a". */
const char *hawkes_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HAWKES_H */
