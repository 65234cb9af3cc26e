/*
 * speedup.h -- C ABI of the GB300 (sm_103a) path-integral Monte Carlo
 * estimator of the discretized transition amplitude A_N^(p)(a,b;T) with
 * level-p short-time effective actions (Balaz, Vidanovic, Stojiljkovic,
 * Vudragovic, Belic, Bogojevic, "SPEEDUP Code for Calculation of Transition
 * Amplitudes via the Effective Action Approach").
 *
 * Units: hbar = m = 1, imaginary time (Sec. 2).  A path has N = 2^s slices of
 * width eps = T/N; q_0 = a, q_N = b.  The estimand (Sec. 4, Eq. SNp) is
 *
 *   A_N^(p)(a,b;T) = int dq_1..dq_{N-1} (2 pi eps)^(-N/2) exp(-S_N^(p)),
 *   S_N^(p) = sum_k [ (q_{k+1}-q_k)^2/(2 eps) + eps W_p(x_k, xb_k; eps) ],
 *
 * x_k = (q_k+q_{k+1})/2, xb_k = (q_{k+1}-q_k)/2, and W_p the level-p
 * effective potential (Sec. 2.1, Eq. ansatz truncated at m <= p-1, with the
 * coefficients of Eq. 1Drec and Eq. diagonal).  Paths are drawn by bisection
 * (Sec. 4.1) from a Philox4x32-10 stream, and the amplitudes of every level
 * n = 0..s of the bisection hierarchy (N = 2^n, Sec. 4.1) come from the same
 * paths.
 *
 * Conventions for every entry point:
 *  - Returns SU_OK (0) or a negative SU_E* code; su_last_error() then gives a
 *    one-line message (thread-local, valid until the next call on the thread).
 *  - Host pointers are caller-owned and only read or written during the call.
 *  - "Device" pointers are CUDA global-memory addresses on the current device,
 *    caller-owned, written asynchronously on the given stream (NULL = the
 *    legacy default stream); the caller synchronizes that stream before
 *    reading them.
 *  - Nothing here falls back to the CPU: without a usable CUDA device every
 *    compute entry point returns SU_ECUDA.
 */
#ifndef SPEEDUP_H
#define SPEEDUP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define SU_OK          0
#define SU_EINVAL     -1   /* an argument is out of range or not finite      */
#define SU_ENOMEM     -2   /* a host or device allocation failed              */
#define SU_ECUDA      -3   /* a CUDA call failed or no device is usable       */
#define SU_ETIMEOUT   -4   /* a bounded device-side wait ran out              */
#define SU_ENONFINITE -5   /* a coefficient or a per-sample weight is NaN/Inf */
#define SU_ENOTSUP    -6   /* valid, but larger than this build supports      */

/* ---- potentials V(q) (Sec. 3.3) ------------------------------------------ */
#define SU_HO    0   /* omega^2 q^2 / 2                        params: omega      */
#define SU_AHO   1   /* A q^2/2 + g q^4/24                     params: A, g       */
#define SU_DW    2   /* h (q^2 - 1)^2                          params: h          */
#define SU_MPT   3   /* -lambda / cosh^2(alpha q)  (Eq. 1D-MPT) params: lambda, alpha */
#define SU_POLY  4   /* sum_i v_i q^i, degree <= 8             params: v_0..v_d   */
/* A general potential (Eq. 1Drec in the derivatives V^(j)(x), j = 0..2p-2,
 * Sec. 3.1): V = sum_{i<=8} a_i q^i + sum_{g<4} A_g e^{-beta_g (q - c_g)^2}
 *              + sum_{t<4} B_t sech^2(alpha_t (q - d_t))
 *              [+ sum_{e<4} E_e e^{-kappa_e (q - x0_e)}].
 * params (33): a_0..a_8, (A, beta, c) x 4, (B, alpha, d) x 4; or 45: the same
 * and (E, kappa, x0) x 4 (Morse potentials are sums of exponentials); a term
 * with a zero amplitude is absent, beta > 0 and alpha != 0 otherwise
 * (SU_EINVAL).
 * W_p is evaluated per slice from V's derivatives at the slice midpoint and
 * the monomials of W_p in them (1629 monomial-power entries at p = 12, 24 196
 * at p = 18), so it needs no collapsed table: p <= 18, SU_FP64 only (the
 * derivatives carry factors up to (2p-1)!, beyond the single-precision range),
 * su_plan_* / speedup_amplitude / speedup_logweights / su_autotune, the batched
 * launch (speedup_amplitude_batch / su_batch_plan_* / su_batch_autotune, one
 * program per level p of the batch) and the evolution operator
 * (speedup_evolution_matrix / _band / _spectrum) only; everything else
 * answers SU_ENOTSUP. */
#define SU_GENERAL 5

/* ---- arithmetic of the per-slice W_p evaluation --------------------------- */
#define SU_FP64  0   /* everything in double                                   */
#define SU_FP32  1   /* path and W_p in float, log-sum-exp reductions in double */

#define SU_MAX_P 144 /* highest effective-action level (Sec. 3.3: AHO to 144)   */
#define SU_MAX_S 10  /* deepest bisection level, N <= 1024                     */

typedef struct {
    int precision;        /* SU_FP64 (default) or SU_FP32                           */
    int n_blocks;         /* contiguous sample blocks for the error estimate; 64    */
    int hierarchy;        /* 1 (default): levels n = 0..s; 0: only n = 0 and n = s  */
    uint32_t instance;    /* Philox counter word 1 (stream id of this instance); 0  */
    double width_factor;  /* bisection width multiplier; 1 (default) = exact bridge,
                             sqrt(2) = the literal sigma_n = sqrt(T/2^n) of Sec. 4.1;
                             the Gaussian density ratio is added to every weight    */
    void *stream;         /* cudaStream_t for all device work; NULL (default)      */
    int64_t sample0;      /* first sample index: samples sample0 .. sample0+n_mc-1,
                             so disjoint ranges on several devices form one run; 0  */
    int seg_log2;         /* launch shape: bisection levels kept in registers, the
                             path processed in segments of 2^seg_log2 slices, 1..5
                             (capped at s); 0 (default) = automatic               */
    int rounds;           /* launch shape: paths per thread per work item, 1..8;
                             0 (default) = automatic.  Automatic = the shape
                             su_autotune stored for this precision, model, p and s
                             in this process, else the built-in rule (seg_log2 =
                             4 for SU_FP64, 5 for SU_FP32, capped at s; rounds =
                             1, doubled while the per-item tuples would exceed
                             512 MB and as many CTAs stay resident).  The shape
                             changes the order of the floating-point sums only. */
    int kernel;           /* 0 (default): a single-precision plan with 32-slice
                             segments whose level tables have a shape compiled
                             into the library (the even-ring shapes of the
                             harmonic oscillator and of the quartic potentials
                             at p <= 18, see su_fixed_shape) runs the sampler
                             specialised for that shape; 1: always the generic
                             sampler.  Both give the same results bit for bit. */
} su_options;

/* per bisection level n = 0..s (N = 2^n slices) */
typedef struct {
    double amp;        /* estimate of A_N^(p)(a,b;T)                              */
    double log_amp;    /* its logarithm (finite where amp underflows)             */
    double err;        /* std. dev. of the n_blocks block means / sqrt(n_blocks)  */
    double rel_err;    /* err / amp                                               */
    double err_naive;  /* sqrt((<f^2> - <f>^2) / (n - 1)), the Sec. 4.1 estimate  */
    double ess;        /* effective sample size (sum f)^2 / sum f^2               */
    double max_share;  /* largest single weight / sum of weights                  */
    int64_t n;         /* samples used                                            */
} su_level_result;

/* Fill *opt with the defaults listed above. */
void su_options_default(su_options *opt);

/* One-line message for the last error on this thread ("" if none). */
const char *su_last_error(void);

/* Library and device description: writes at most cap bytes (NUL-terminated). */
int su_version(char *buf, int cap);

/*
 * speedup_amplitude -- A_N^(p)(a,b;T) for every bisection level n = 0..s
 * (N = 2^n), from n_mc bisection paths (Sec. 4 and 4.1).
 *
 *   model, params, n_params : potential (SU_* above) and its parameters.
 *   a, b, T                 : endpoints and propagation time, T > 0.
 *   p                       : effective-action level, 1..SU_MAX_P.
 *   s                       : bisection depth, 0..SU_MAX_S.
 *   n_mc                    : samples, >= 1.  Sample i (i = opt->sample0 ..
 *                             opt->sample0 + n_mc - 1) uses the Philox counter
 *                             (call t, opt->instance, i lo32, i hi32) under the
 *                             key (seed lo32, seed hi32).
 *   opt                     : NULL for defaults.
 *   out                     : host, s+1 entries, out[n] for level n.  Level 0 is
 *                             the analytic single-slice value with err = 0.
 *                             Without the hierarchy only out[0] and out[s] are
 *                             written.
 *
 * Host arguments in, host results out; the device work runs on opt->stream and
 * the call returns after it.  Device scratch is allocated and freed inside.
 */
int speedup_amplitude(int model, const double *params, int n_params,
                      double a, double b, double T, int p, int s,
                      int64_t n_mc, uint64_t seed, const su_options *opt,
                      su_level_result *out);

/*
 * speedup_generate_coeffs -- the level-p effective potential collapsed at a
 * fixed eps (Eq. ansatz with the coefficients of Eq. 1Drec / Eq. diagonal,
 * computed in double-double arithmetic and rounded):
 *
 *   W_p(x, xb; eps) = sum_{j=0}^{J} xb^(2j) sum_{i=0}^{D_j} P_{ij} z^i,
 *   z = x^2 (SU_HO, SU_AHO, SU_DW and even SU_POLY), z = x (other SU_POLY),
 *   z = tanh^2(alpha x) (SU_MPT).
 *
 *   table    : host, capacity doubles; receives P, column j after column j-1,
 *              i ascending within a column.
 *   shape    : host, SU_MAX_P + 2 ints; shape[0] = J + 1 columns, shape[1] =
 *              the ring (0: z = x^2, 1: z = x, 2: z = tanh^2(alpha x)),
 *              shape[2 + j] = D_j + 1 entries of column j.
 *   n_terms  : host, receives the number of entries written.
 * Returns SU_ENOTSUP if capacity is too small (n_terms still says how many).
 */
int speedup_generate_coeffs(int model, const double *params, int n_params, int p,
                            double eps, double *table, int capacity, int *shape,
                            int *n_terms);

/*
 * su_fit_continuum -- the continuum estimate of Sec. 4 (Eq. fit) from one
 * run's levels (host only): weighted least squares of
 *   A_N = A + B / N^p  [+ C / N^(p+1) when n_terms = 3],   N = 2^n,
 * over the levels n = n_min..s of levels[] (speedup_amplitude's output,
 * s + 1 entries), weights 1 / err_n^2.  *A = the constant, *A_err its
 * least-squares standard error (levels of one run share samples, so this
 * treats them as independent), *chi2 = the weighted residual sum (either may
 * be NULL).  n_min >= 1 (level 0 has no statistical error); SU_EINVAL when a
 * used level has no finite positive error or there are fewer levels than
 * terms.
 */
int su_fit_continuum(const su_level_result *levels, int s, int p, int n_min, int n_terms,
                     double *A, double *A_err, double *chi2);

/* ---- many instances in one persistent launch ------------------------------ */

/* One amplitude A_N^(p)(a,b;T), N = 2^s, of a batch.  A zero-initialised
 * tail (p = 0, n_mc = 0, hierarchy = 0) takes the batch's p and n_mc and the
 * top level only. */
typedef struct {
    double a, b, T;
    int s;               /* 0..SU_MAX_S                                           */
    int p;               /* effective-action level 1..SU_MAX_P; 0 = the batch's p  */
    int64_t n_mc;        /* samples, >= 1; 0 = the batch's n_mc                    */
    int hierarchy;       /* 0: the top level n = s only (one result);
                            1: every level n = 0..s from the same paths (s + 1
                            results, level 0 analytic)                           */
    int reserved;        /* 0                                                     */
} su_instance;

/*
 * speedup_amplitude_batch -- the amplitudes A_N^(p_i)(a_i,b_i;T_i), N = 2^(s_i),
 * of every instance of one model (Sec. 4; e.g. a matrix of short-time
 * amplitudes on an endpoint grid, or a convergence sweep over p), from n_mc_i
 * bisection paths each, in one persistent launch of the batched kernel,
 * replayed from a CUDA graph.  Work items are (instance, error block, chunk)
 * triples ordered by their cost (samples x slices x table entries), taken
 * from an atomic queue; each instance's tables (one per level p_i and
 * slice width) are staged per item (the general potential: its program per
 * level p_i, read from device memory; double precision only).
 *
 *   p, n_mc      : the defaults for instances whose p or n_mc is 0.
 *   inst, n_inst : host, 1..2^24 instances.  Instance i draws from Philox
 *                  stream opt->instance + i (counter word 1), samples
 *                  0..n_mc_i - 1.
 *   opt          : precision, n_blocks (per instance, capped at its n_mc),
 *                  stream; width_factor must be 1, sample0 0; hierarchy,
 *                  seg_log2 and rounds are not used (per-instance hierarchy;
 *                  the shape of each (p, s, hierarchy) class is the one
 *                  su_batch_autotune stored, else the rule: 2^4-slice
 *                  register segments in double, 2^5 in single precision
 *                  and for the general potential, capped at s).
 *   out          : host, one entry per instance with hierarchy 0 and s_i + 1
 *                  (levels n = 0..s_i) per instance with hierarchy 1, in
 *                  instance order (su_batch_plan_sizes gives the count).  An
 *                  instance with s_i = 0 gets the analytic level-0 value with
 *                  err 0.
 */
int speedup_amplitude_batch(int model, const double *params, int n_params, int p,
                            const su_instance *inst, int64_t n_inst, int64_t n_mc,
                            uint64_t seed, const su_options *opt, su_level_result *out);

typedef struct su_batch_plan su_batch_plan;

/* the same, split: create (host tables, per-instance data and the sorted work
 * list uploaded to plan-owned device memory), sizes, execute, finalize */
int su_batch_plan_create(int model, const double *params, int n_params, int p,
                         const su_instance *inst, int64_t n_inst, int64_t n_mc,
                         uint64_t seed, const su_options *opt, su_batch_plan **plan);
int su_batch_plan_destroy(su_batch_plan *plan);
/* *tuple_bytes: d_tuples size (per instance and work item, one tuple (M, S,
 * Q, n) of 4 doubles per sampled level); *scratch_bytes: d_scratch size;
 * *slice_actions per execute (hierarchy slices counted); *n_results (may be
 * NULL): the entries of out. */
int su_batch_plan_sizes(const su_batch_plan *plan, int64_t *tuple_bytes, int64_t *scratch_bytes,
                        int64_t *slice_actions, int64_t *n_results);
/* The launch shape the plan chose for instance i: *seg_log2 = its register
 * segment (2^seg_log2 slices), *chunks = work items per error block, *from
 * = 0 (rule) or 1 (stored by su_batch_autotune). */
int su_batch_plan_shape(const su_batch_plan *plan, int64_t i, int *seg_log2, int *chunks, int *from);

/* The batched kernels a plan launches.  In single precision every level p of
 * the batch whose table shape is compiled into the library (su_fixed_shape)
 * runs a batched kernel with that shape compiled in (its instances with
 * 32-slice segments take the specialised path code), the other levels the
 * generic kernel, one persistent launch per kernel in the plan's graph.
 * *fixed_shape = the compiled shape's index when the plan launches that one
 * kernel only, -1 when it launches only the generic kernel, -2 when several.
 * opt->kernel = 1 forces -1; every choice gives the same results bit for
 * bit (the work items do not depend on it). */
int su_batch_plan_kernel(const su_batch_plan *plan, int *fixed_shape);

/* asynchronous on stream; the first call builds the plan's CUDA graph (a
 * memset of the queue head and the persistent kernel), later calls replay it
 * (and rebuild it if the buffers change); *launches = graph launches made */
int su_batch_plan_execute(su_batch_plan *plan, void *d_tuples, void *d_scratch, void *stream,
                          int *launches);
/* host tuples in, out as speedup_amplitude_batch; d_scratch (may be NULL) is
 * read for the non-finite flag.  SU_ECUDA if an instance's samples were not
 * all reduced. */
int su_batch_plan_finalize(const su_batch_plan *plan, const double *h_tuples,
                           const void *d_scratch, su_level_result *out);

/* One timed shape of su_batch_autotune: class (p, s, hierarchy), shape, and
 * the device time per slice-action of the probe batch. */
typedef struct {
    int p, s, hierarchy;
    int seg_log2;
    double ns_per_slice;
} su_batch_tuning;

/*
 * su_batch_autotune -- for every (p, s, hierarchy) class of the batch with
 * s >= 1, times the batched kernel on a probe of that class (its first
 * max_probe instances with their own samples, one execute after a warm-up,
 * best of two) for every register segment seg_log2 = 1..min(s, 5) whose
 * shared memory fits, and stores the fastest in a process-wide table under
 * (precision, model, p, s, hierarchy); later batch plans use it.  No
 * counterpart in the paper.  Arguments as su_batch_plan_create;
 *   best, cap, n_best : host, optional: the chosen shape of up to cap
 *                       classes, *n_best = the number of classes.
 * Synchronous.  su_autotune_clear forgets these shapes too.
 */
int su_batch_autotune(int model, const double *params, int n_params, int p, const su_instance *inst,
                      int64_t n_inst, int64_t n_mc, uint64_t seed, const su_options *opt, int max_probe,
                      su_batch_tuning *best, int cap, int *n_best);

/* ---- learned bisection proposal -------------------------------------------- */

/*
 * A small network proposes every bisection midpoint (Sec. 4.1) from the
 * instance and the midpoint's parents: x = (a, b, T, n/s, q_L, q_R) ->
 * Linear(6,128) -> GELU -> Linear(128,128) -> GELU -> Linear(128,128) -> GELU
 * -> Linear(128,2) = (shift, ls), GELU(v) = v (1 + erf(v/sqrt 2))/2, and the
 * midpoint is q = (q_L + q_R)/2 + sigma_n (shift + e^ls z) with the plain
 * sampler's normal z.  Each midpoint adds the exact log density ratio
 * z^2/2 - (shift + e^ls z)^2/2 + ls (bridge over proposal) to the weight of
 * every level >= n, so the estimate of A_N^(p) stays unbiased for any
 * network.  Bfloat16 weights and activations, float accumulation (tensor
 * cores), single-precision path and W_p, double reductions.
 *
 * theta: SU_MLP_PARAMS floats, W1[128][6], b1[128], W2[128][128], b2[128],
 * W3[128][128], b3[128], W4[2][128], b4[2] (matrices [out][in]).
 */
#define SU_MLP_PARAMS 34178

typedef struct su_proposal su_proposal;

/* upload a network (host theta, copied); SU_ENONFINITE on a NaN/Inf weight */
int su_proposal_create(const float *theta, int n_params, su_proposal **prop);
int su_proposal_destroy(su_proposal *prop);

/* the network on n rows of features: d_X (device, n x 6 floats) ->
 * d_Y (device, n x 2 floats: shift, ls).  Asynchronous on stream. */
int su_mlp_forward(const su_proposal *prop, const float *d_X, int64_t n, float *d_Y, void *stream);

/*
 * speedup_amplitude_proposal -- speedup_amplitude with the midpoints drawn
 * from the network (opt->precision must be SU_FP32, s <= 6, width_factor 1).
 */
int speedup_amplitude_proposal(int model, const double *params, int n_params,
                               double a, double b, double T, int p, int s,
                               int64_t n_mc, uint64_t seed, const su_options *opt,
                               const su_proposal *prop, su_level_result *out);

/*
 * speedup_amplitude_judged -- the learned proposal judged against, and
 * falling back to, the plain sampler.  Two pilot runs of n_pilot samples
 * each (the samples after the run's own range: opt->sample0 + n_mc ..),
 * one per sampler (single precision, top level), give each sampler's device
 * time per sample and per-sample relative variance n / ESS - 1; from them
 * the estimated time to the relative statistical error target_rel_err,
 *   t = (seconds per sample) (n / ESS - 1) / target_rel_err^2.
 * The main run (n_mc samples, the same as speedup_amplitude or
 * speedup_amplitude_proposal would draw) uses the proposal only when both
 * pilots are usable (finite positive estimate, ESS >= 10), they agree
 * (|z| <= 5 with z = (A_proposal - A_plain) / sqrt(err_proposal^2 +
 * err_plain^2)), and the proposal's estimated time is the shorter; otherwise
 * the plain sampler, with the reason in judge->reason.  An unbiased but
 * unconfirmed proposal estimate (where the plain pilot diverges) is therefore
 * never returned silently: it stays in judge->pilot_amp[1].  No counterpart
 * in the paper.  Arguments as speedup_amplitude_proposal (s >= 1), and:
 *   n_pilot         : samples per pilot, >= 2 (enough to fill the GPU, e.g. 2e5).
 *   target_rel_err  : the relative error the times are estimated for, > 0.
 *   out             : host, s + 1 entries, as speedup_amplitude.
 *   judge           : host, the figures the choice was made on.
 * Synchronous.
 */
#define SU_JUDGE_PLAIN_FASTER       0  /* both usable and agreeing; plain is faster    */
#define SU_JUDGE_PROPOSAL_FASTER    1  /* both usable and agreeing; proposal is faster */
#define SU_JUDGE_PROPOSAL_UNUSABLE  2  /* the proposal's pilot is not usable: plain    */
#define SU_JUDGE_PLAIN_UNUSABLE     3  /* the plain pilot is not usable, so the proposal
                                          cannot be confirmed: plain                    */
#define SU_JUDGE_DISAGREE           4  /* the pilots disagree (|z| > 5): plain          */

typedef struct {
    int chosen;              /* 0 = plain sampler, 1 = learned proposal          */
    int reason;              /* SU_JUDGE_*                                       */
    double target_rel_err;
    double pilot_amp[2];     /* [0] plain, [1] proposal: top-level estimates     */
    double pilot_err[2];
    double pilot_ess[2];
    double pilot_relvar[2];  /* n / ESS - 1 (infinite when unusable)             */
    double pilot_s[2];       /* device seconds of each pilot                     */
    double t_target[2];      /* estimated seconds to target_rel_err (inf: unusable) */
    double z;                /* pilot agreement (NaN unless both usable)         */
    double run_s;            /* device seconds of the main run                   */
} su_judge;

int speedup_amplitude_judged(int model, const double *params, int n_params,
                             double a, double b, double T, int p, int s,
                             int64_t n_mc, uint64_t seed, const su_options *opt,
                             const su_proposal *prop, int64_t n_pilot, double target_rel_err,
                             su_level_result *out, su_judge *judge);

/*
 * speedup_proposal_logweights -- per-sample log-weights of the proposal path
 * (W_p sum plus the proposal's log density ratio), laid out as
 * speedup_logweights; d_outs (device, may be NULL) receives the network's
 * (shift, ls) per sample and heap index j: d_outs[((i - sample0) * (N-1) + j) * 2].
 */
int speedup_proposal_logweights(int model, const double *params, int n_params,
                                double a, double b, double T, int p, int s,
                                int64_t sample0, int64_t n_samples, uint64_t seed,
                                const su_options *opt, const su_proposal *prop,
                                double *d_w, float *d_outs);

/*
 * Training of the proposal (weighted maximum likelihood of midpoints of plain
 * paths).  Loss over rows r (one row per midpoint: its features x_r, its
 * standardized offset u_r = (q - (q_L + q_R)/2) / sigma_n, weight rw_r):
 *   L = sum_r rw_r [ls_r + (u_r - shift_r)^2 e^(-2 ls_r) / 2] / sum_r rw_r.
 * Bfloat16 tensor-core forward and backward, float accumulation and float
 * master weights.
 */
typedef struct {
    int64_t n_train;       /* plain paths to learn from; 1e6                        */
    int steps;             /* Adam steps; 2000                                      */
    int batch_paths;       /* paths per step (rows = batch_paths * (N-1)); 512      */
    double lr;             /* Adam learning rate; 1e-3                              */
    double clip_quantile;  /* top-level log-weights above this quantile are clipped
                              for the training weights (rare huge weights would
                              otherwise fit one path); 0.999                         */
    uint64_t seed;         /* minibatch draws (Philox key, drawn on the device); 1  */
} su_train_options;

void su_train_options_default(su_train_options *t);

/* loss and gradient (host, SU_MLP_PARAMS floats in theta's order) of n rows
 * given on the device: d_X (n x 6), d_u (n), d_rw (n) floats.  Synchronous. */
int su_mlp_loss_grad(const float *theta, const float *d_X, const float *d_u, const float *d_rw,
                     int64_t n, double *loss, float *grad);

/*
 * speedup_train_proposal -- draw topt->n_train plain single-precision paths of
 * the instance (seed), weigh them by their top-level weight (clipped at
 * clip_quantile), and run topt->steps Adam steps on minibatches drawn in
 * proportion to those weights.  theta: host, SU_MLP_PARAMS floats, initial
 * network in, trained network out.  loss_out (host, steps doubles, may be
 * NULL) receives the minibatch losses.  2 <= s <= 6.  Synchronous.  The
 * minibatches are drawn on the device and one step is replayed as a CUDA
 * graph on a stream of the call's own.
 */
int speedup_train_proposal(int model, const double *params, int n_params,
                           double a, double b, double T, int p, int s, uint64_t seed,
                           const su_train_options *topt, float *theta, double *loss_out);

/* ---- device-resident interface (inputs and outputs stay in HBM) ----------- */

typedef struct su_plan su_plan;

/*
 * su_plan_create -- validate, generate the coefficient tables of every level
 * (host), and upload them to device memory owned by the plan.  Arguments as
 * for speedup_amplitude.
 */
int su_plan_create(int model, const double *params, int n_params,
                   double a, double b, double T, int p, int s,
                   int64_t n_mc, uint64_t seed, const su_options *opt, su_plan **plan);

/* Release a plan and its device memory (NULL is a no-op). */
int su_plan_destroy(su_plan *plan);

/* ---- systems of several coordinates (Sec. 2.2) ----------------------------- */

#define SU_MAX_D 4   /* d = D x M coordinates (D dimensions, M particles)      */

/*
 * A polynomial potential V(x_1..x_d) of total degree <= 6 and at most 256
 * terms: term t is coefs[t] * prod_i x_i^exps[t d + i] (exps: host, n_terms x
 * d ints in 0..6; coefs: host, n_terms doubles, finite).  The level-p
 * effective potential W(x, xb; eps) = sum_{m<p} sum_{k<=m} eps^(m-k) W_{m,k}
 * follows from the contracted recursion Eq. MBrec with the diagonal Eq. DIA
 * (double-double on the host); every coordinate has unit mass, no quantum
 * statistics (amplitudes are not symmetrised).  p <= 12; SU_FP64, or SU_FP32
 * (path and W in float, the stream's float layout, log-sum-exp in double);
 * the exact bridge only (width_factor 1), one launch shape (seg_log2 = 0,
 * rounds <= 1); SU_ENOTSUP otherwise.
 *
 * su_plan_create_nd -- a plan for A_N^(p)(a, b; T), N = 2^s, with a and b
 * (host, d doubles each) the endpoint vectors; it is executed, finalized and
 * destroyed by the su_plan_* calls above.  A_free is the product of the d
 * one-dimensional free amplitudes.  Coordinate c of bisection midpoint j
 * takes normal j d + c of the sample's stream (speedup_normals layout).  The
 * scratch (su_plan_sizes) also holds every resident thread's path segment
 * endpoints: grid x 128 x (2^max(s-5, 0) + 1) x d doubles.
 */
int su_plan_create_nd(int d, const int *exps, const double *coefs, int n_terms,
                      const double *a, const double *b, double T, int p, int s,
                      int64_t n_mc, uint64_t seed, const su_options *opt, su_plan **plan);

/* speedup_amplitude for a system of d coordinates (host in, host out). */
int speedup_amplitude_nd(int d, const int *exps, const double *coefs, int n_terms,
                         const double *a, const double *b, double T, int p, int s,
                         int64_t n_mc, uint64_t seed, const su_options *opt,
                         su_level_result *out);

/* speedup_logweights for a system of d coordinates: d_w (device) receives
 * n_samples x s doubles, w_n of sample sample0 + i at d_w[i s + n - 1]. */
int speedup_logweights_nd(int d, const int *exps, const double *coefs, int n_terms,
                          const double *a, const double *b, double T, int p, int s,
                          int64_t sample0, int64_t n_samples, uint64_t seed,
                          const su_options *opt, double *d_w);

/*
 * speedup_generate_nd -- W(x, xb; eps) of a system of d coordinates at one
 * eps, as monomials (host only, no device): term t is
 * out_w[t] * prod_i x_i^out_exps[2 d t + i] xb_i^out_exps[2 d t + d + i]
 * (out_exps: capacity x 2d ints; out_w: capacity doubles).  *n_out = the
 * number of terms; SU_ENOTSUP if it exceeds capacity.
 */
int speedup_generate_nd(int d, const int *exps, const double *coefs, int n_terms, int p,
                        double eps, int *out_exps, double *out_w, int capacity, int *n_out);

/*
 * speedup_wp -- the level-p effective potential W_p(x, xb; eps) of a
 * one-dimensional model (Eq. ansatz, coefficients of Eq. 1Drec and Eq.
 * diagonal) at n_points points, on the host (no device), as plans evaluate
 * their level-0 weight: the collapsed table of speedup_generate_coeffs in
 * double-double for the model potentials, the general mode's program in the
 * derivative symbols V^(j)(x) for SU_GENERAL.  x, xb, w: host arrays of
 * n_points doubles; w[i] = W_p(x[i], xb[i]; eps).  Errors: SU_EINVAL (unknown
 * model, wrong parameters, p outside 1..SU_MAX_P, eps not finite and > 0,
 * n_points < 0, a missing array), SU_ENOTSUP (SU_GENERAL above p = 18).
 */
int speedup_wp(int model, const double *params, int n_params, int p, double eps,
               const double *x, const double *xb, int64_t n_points, double *w);

/*
 * speedup_wp_nd -- W(x, xb; eps) of a system of d coordinates (potential
 * arguments as su_plan_create_nd; Sec. 2.2, Eq. MBrec, Eq. DIA) at n_points
 * points, on the host, through the evaluation program of the
 * several-coordinates kernel (prefix nodes, Horner in one variable, the
 * level's rounded table).  x, xb: host arrays laid out [point][d]; w: host,
 * n_points doubles.  Errors as speedup_generate_nd, and SU_EINVAL for eps not
 * finite and > 0, n_points < 0 or a missing array.
 */
int speedup_wp_nd(int d, const int *exps, const double *coefs, int n_terms, int p, double eps,
                  const double *x, const double *xb, int64_t n_points, double *w);

/*
 * su_plan_sizes -- sizes of the caller-provided device buffers of
 * su_plan_execute, in bytes: *tuple_bytes for d_tuples, *scratch_bytes for
 * d_scratch; *levels = the number of levels sampled (s, or 1 without the
 * hierarchy); *slice_actions = W_p evaluations per execute.
 */
int su_plan_sizes(const su_plan *plan, int64_t *tuple_bytes, int64_t *scratch_bytes,
                  int *levels, int64_t *slice_actions);

/*
 * su_plan_execute -- sample the plan's n_mc paths on the device (Sec. 4.1) and
 * reduce their weights per block and level (log-sum-exp in double).
 *
 *   d_tuples  : device, tuple_bytes; receives, for block b and sampled level
 *               d (d = 0 is level s, d = 1 level s-1, ...), the four doubles
 *               (M, S, Q, n): M = max w, S = sum exp(w - M),
 *               Q = sum exp(2(w - M)), n = samples, at
 *               d_tuples[4 * (b * levels + d)].
 *   d_scratch : device, scratch_bytes, library-owned for the duration.
 *   stream    : cudaStream_t or NULL.
 * Asynchronous; the tuples are ready when the stream reaches this point.
 * *launches (may be NULL) receives the number of kernel launches made.
 */
int su_plan_execute(su_plan *plan, void *d_tuples, void *d_scratch, void *stream,
                    int *launches);

/*
 * su_plan_finalize -- turn host copies of the block tuples into per-level
 * results exactly as speedup_amplitude does (out: s+1 entries).
 * Also returns SU_ENONFINITE if the device flagged a non-finite weight
 * (read from d_scratch, which must be the buffer execute used).
 */
int su_plan_finalize(const su_plan *plan, const double *h_tuples, const void *d_scratch,
                     su_level_result *out);

/* ---- evolution operator on a grid ----------------------------------------- */

/*
 * speedup_evolution_matrix -- the space-discretized short-time evolution
 * operator whose diagonalisation gives energy eigenvalues and eigenfunctions
 * (Sec. 5, Fig. 3): on the grid x_i = -L + i Delta, i = 0..n-1,
 * Delta = 2L/(n-1) (each point rounded as (i Delta) + (-L), x_{n-1} = L),
 *   U_ij = Delta (2 pi t)^(-1/2) exp(-(x_j - x_i)^2/(2t) - t W_p(x, xb; t)),
 *   x = (x_i + x_j)/2, xb = (x_j - x_i)/2,
 * the single-slice amplitude with the level-p effective potential, and
 * U_ij = 0 where (x_j - x_i)^2/(2t) > 40 (the free factor is below e^-40 and
 * the short-time expansion in xb^2 = O(t) does not apply).  U is symmetric;
 * its eigenvalues approach e^(-t E_k) (E_k = -ln(lambda_k)/t) and its
 * eigenvectors / sqrt(Delta) the eigenfunctions.
 *   model, params, n_params, p : as for speedup_amplitude.
 *   t     : propagation time of one slice, > 0.
 *   L     : grid half-width, > 0.   n : grid points, 2..65536.
 *   precision : SU_FP64 or SU_FP32 (W_p in float; the free factor and the
 *           output in double); SU_GENERAL in SU_FP64 only.
 *   d_U   : device, n*n doubles, row-major.
 * Work on stream; returns after the matrix is written (the stream is
 * synchronised).  Errors: SU_EINVAL, SU_ENONFINITE (a coefficient is not
 * representable in the chosen precision), SU_ECUDA, SU_ENOMEM.
 */
int speedup_evolution_matrix(int model, const double *params, int n_params, int p, double t, double L, int n,
                             int precision, double *d_U, void *stream);

/*
 * su_evolution_band_size -- the geometry of the band storage below: the
 * half width w (U_ij = 0 for |i - j| > w: the band of reading "free factor
 * below e^-40") and the row pitch (n rounded up to 32).  Host only.
 */
int su_evolution_band_size(double t, double L, int n, int *half_width, int64_t *pitch);

/*
 * speedup_evolution_band -- the upper band of the evolution operator of
 * speedup_evolution_matrix (Sec. 5, Fig. 3), diagonal-major:
 *   d_band[k * pitch + i] = U_{i,i+k},  k = 0..w,  i = 0..n-1
 * (zero where i + k >= n and outside the band; U is symmetric, so this is
 * all of it).  About (w + 1) n doubles instead of n^2: 170 MB instead of
 * 2.1 GB on the 16 385-point grid of Fig. 3.
 *   d_band   : device, capacity bytes >= (w + 1) * pitch * 8.
 * Arguments otherwise as speedup_evolution_matrix; returns after the band is
 * written.
 */
int speedup_evolution_band(int model, const double *params, int n_params, int p, double t, double L, int n,
                           int precision, double *d_band, int64_t capacity, void *stream);

/* What speedup_evolution_spectrum did. */
typedef struct {
    int half_width;       /* w of the band                                      */
    int block;            /* columns of the subspace block (8, 16 or 32)        */
    int iterations;       /* filter and Rayleigh-Ritz rounds after the first    */
    int converged;        /* 1: every residual within 1e-11 theta_0             */
    int64_t band_bytes;   /* device bytes of the band                           */
    int64_t matvecs;      /* products of U with one vector (a block counts B)   */
    double lower, upper;  /* spectrum bounds of U from 40 Lanczos steps         */
    double band_ms;       /* device time: the band                              */
    double solve_ms;      /* device and host time of the eigensolver            */
    int block_matvecs;    /* band matrix-block products U X                     */
    double block_matvec_ms; /* their device time (CUDA events)                  */
} su_spectrum_info;

/*
 * speedup_evolution_spectrum -- the lowest nev energies E_k = -ln(lambda_k)/t
 * (ascending) of the evolution operator (Sec. 5, Fig. 3) from the nev largest
 * eigenvalues lambda_k of the band matrix: Chebyshev-filtered block subspace
 * iteration with Rayleigh-Ritz in double precision on the device (band
 * matrix-block products, Gram products and rotations in this library's
 * kernels; B x B Cholesky and Jacobi on the host), no dense matrix and no
 * library eigensolver.
 *   nev        : 1..26 (and <= n/2).
 *   energies   : host, nev doubles.
 *   residuals  : host, nev doubles or NULL: |U x_k - lambda_k x_k| of the
 *                unit Ritz vectors (the eigenvalue error is at most about
 *                residual^2 / gap).
 *   d_vectors  : device, n * nev doubles or NULL: eigenfunction k on the grid,
 *                psi_k(x_i) = d_vectors[k * n + i] (unit L2 norm in x; sign
 *                arbitrary).
 *   info       : host or NULL.
 * Synchronous; allocates the band and the work buffers itself.  Errors as
 * speedup_evolution_band, SU_EINVAL for nev, SU_ENOTSUP if the residuals do
 * not reach 1e-11 lambda_0 within 60 rounds (energies and info still written).
 */
int speedup_evolution_spectrum(int model, const double *params, int n_params, int p, double t, double L, int n,
                               int precision, int nev, double *energies, double *residuals, double *d_vectors,
                               su_spectrum_info *info, void *stream);

/* ---- fault injection (test support) ---------------------------------------- */

/* No counterpart in the paper: host-side hooks for the failure-detection tests.
 * Every hook is off until set and fires once. */
#define SU_FAULT_CLEAR        0  /* turn every hook off                                  */
#define SU_FAULT_ALLOC        1  /* the arg-th device allocation from now fails (ENOMEM) */
#define SU_FAULT_TABLE_NAN    2  /* the next coefficient table gets a NaN (ENONFINITE)   */
#define SU_FAULT_QUEUE_STOP   3  /* the next batched execute stops after arg work items;
                                    its finalize reports the missing samples (ECUDA)    */
#define SU_FAULT_WITHHOLD_MMA 4  /* the next proposal launch withholds its first MMA
                                    commit: the bounded wait (one second) runs out and
                                    the call returns SU_ETIMEOUT                         */
int su_fault_inject(int kind, int64_t arg);

/* ---- launch-shape autotuner ----------------------------------------------- */

typedef struct {
    int seg_log2;      /* su_options.seg_log2 of this shape                       */
    int rounds;        /* su_options.rounds of this shape                         */
    double ms;         /* device time of one execute of the probe plan (best of 2) */
} su_tuning;

/*
 * su_autotune -- times every launch shape (seg_log2 = 1..min(s, 5), rounds =
 * 1, 2, 4, 8 where the shared memory allows) of the sampler on n_probe
 * samples of the given instance (opt: precision, n_blocks, hierarchy, stream;
 * its seg_log2 and rounds are ignored), stores the fastest in a process-wide
 * table under (precision, model, p, s), and returns it.  Later plans of that
 * key with automatic shape use it.  No counterpart in the paper: a host-side
 * search over this implementation's launch parameters.
 *   best          : host, the fastest shape.
 *   all, cap      : host, optional (NULL, 0): up to cap timed shapes.
 *   n_all         : host, optional: shapes timed.
 * Synchronous.  Errors: SU_EINVAL (arguments as for speedup_amplitude, s >= 1,
 * n_probe >= 1), SU_ECUDA, SU_ENOMEM.
 */
int su_autotune(int model, const double *params, int n_params, double a, double b, double T,
                int p, int s, int64_t n_probe, uint64_t seed, const su_options *opt,
                su_tuning *best, su_tuning *all, int cap, int *n_all);

/*
 * su_plan_execute_range -- checkpoint / resume: sample only the error blocks
 * [b0, b1) of the plan (block b = samples [b n_mc / n_blocks, (b+1) n_mc /
 * n_blocks) of the run) and write only their tuples in d_tuples; the other
 * blocks' tuples are left as they are.  A run interrupted after blocks
 * [0, k) is checkpointed by saving the tuple array (n_blocks * levels * 4
 * doubles) and resumed, in any later process, by loading it into d_tuples
 * and executing [k, n_blocks): the counter-based stream and the per-block
 * reduction make the result identical to the uninterrupted run, bit for bit.
 * No counterpart in the paper (its C code runs to completion).
 */
int su_plan_execute_range(su_plan *plan, int64_t b0, int64_t b1, void *d_tuples, void *d_scratch, void *stream,
                          int *launches);

/* su_plan_execute with the device time of its launches: CUDA events around
 * them on stream, *ms = elapsed milliseconds (synchronises the stop event). */
int su_plan_execute_timed(su_plan *plan, void *d_tuples, void *d_scratch, void *stream, int *launches,
                          float *ms);

/* Forget every shape su_autotune stored (automatic shapes revert to the rule). */
int su_autotune_clear(void);

/* The launch shape a plan uses. */
int su_plan_shape(const su_plan *plan, int *seg_log2, int *rounds);

/* The sampler a plan launches: *fixed_shape = the index of the table shape
 * compiled into it (see su_fixed_shape), or -1 for the generic sampler. */
int su_plan_kernel(const su_plan *plan, int *fixed_shape);

/* Host only: the index of the compiled table shape (0..19) equal to the
 * shape of the collapsed W_p tables of this model and level p (Eq. SNp in
 * powers of xb^2 and z; the shape does not depend on eps), or -1 if none
 * is.  A single-precision plan of that model and p with 32-slice segments
 * and width_factor = 1 runs the sampler specialised for that shape unless
 * opt->kernel = 1.  SU_ENOTSUP for the general potential (no table). */
int su_fixed_shape(int model, const double *params, int n_params, int p, int *index);


/*
 * speedup_logweights -- per-sample log-weights (Sec. 4.1 normalisation written
 * out): w_n = -eps_n sum_k W_p(x_k, xb_k; eps_n) on the level-n subpath, plus
 * the width-factor correction, for samples sample0 .. sample0 + n_samples - 1
 * and levels n = 1..s.
 *
 *   d_w : device, n_samples * s doubles, w[(i - sample0) * s + (n - 1)]
 *         (written in double for both precisions).
 * Asynchronous on opt->stream.  Requires s >= 1.
 */
int speedup_logweights(int model, const double *params, int n_params,
                       double a, double b, double T, int p, int s,
                       int64_t sample0, int64_t n_samples, uint64_t seed,
                       const su_options *opt, double *d_w);

/*
 * speedup_philox_words -- the raw Philox4x32-10 output blocks of samples
 * sample0 .. sample0 + n_samples - 1, calls 0 .. n_calls - 1:
 *   d_out[((i - sample0) * n_calls + t) * 4 + r], r = 0..3   (device, uint32).
 * Asynchronous on stream.
 */
int speedup_philox_words(uint64_t seed, uint32_t instance, int64_t sample0,
                         int64_t n_samples, int n_calls, uint32_t *d_out, void *stream);

/*
 * speedup_normals -- the Gaussian normals the sampler draws (Sec. 4.1
 * Box-Muller, both branches, from the Philox stream above), j in the heap
 * order of the bisection midpoints.  SU_FP64: normal j of sample i is branch
 * (j & 1) of call j >> 1, 53-bit uniforms u1 from words (w0, w1) and u2 from
 * (w2, w3).  SU_FP32: with j' = j + 1, normal j is slot j' & 3 of call
 * j' >> 2; slots 0, 1 are the two branches from the 24-bit uniforms (float
 * arithmetic) of w0 and w1, slots 2, 3 those of w2 and w3.
 *   d_out[(i - sample0) * n_normals + j]   (device, double).
 * Asynchronous on stream.
 */
int speedup_normals(uint64_t seed, uint32_t instance, int64_t sample0, int64_t n_samples,
                    int n_normals, int precision, double *d_out, void *stream);

/*
 * speedup_amplitude_noalloc -- speedup_amplitude for callers that cannot
 * allocate device memory: those running under an allocator that owns all of
 * the GPU's memory, inside a memory-capped or pre-partitioned process, or in
 * a loop where cudaMalloc/cudaFree and the synchronisation they imply are not
 * allowed.  The paper has no counterpart; the arguments, results and errors
 * are those of speedup_amplitude, and so are the tables and the launch shape
 * (opt->seg_log2, opt->rounds, a shape stored by su_autotune, or the built-in
 * rule; double-precision tables too large for shared memory are read from
 * global memory).  SU_GENERAL is not served (SU_ENOTSUP).
 *
 * Device scratch (coefficient tables, per-item and per-block log-sum-exp
 * tuples, the non-finite flag) lives in one static device array of
 * SU_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits.  The call makes no cudaMalloc,
 * cudaFree or other device allocation (its host-side work arrays use ordinary
 * host memory).
 *  - Size limit: the tables, the per-item tuples (items x levels x 32 bytes,
 *    items = n_blocks x ceil(n_mc / n_blocks / (128 rounds))) and the
 *    per-block tuples (n_blocks x levels x 32 bytes) must fit the array
 *    together.  With automatic rounds the call raises rounds (up to 8, while
 *    the sampler stays resident) until they fit; a request that still does
 *    not fit fails with SU_ENOTSUP and a message naming the sizes.
 *  - The array's device address is looked up (cudaGetSymbolAddress) on every
 *    call, with the caller's device current.
 *  - The call is synchronous: it copies the tables in and the tuples out
 *    through pageable host memory and synchronises opt->stream before it
 *    returns, so it cannot be recorded into a CUDA graph (stream capture).
 *  - Every call shares the one array and leaves its contents behind; calls
 *    whose device work overlaps (other threads, other streams of the same
 *    device) race on it and must be serialised by the caller.
 */
#define SU_NOALLOC_SCRATCH_BYTES (8u << 20)

int speedup_amplitude_noalloc(int model, const double *params, int n_params,
                              double a, double b, double T, int p, int s,
                              int64_t n_mc, uint64_t seed, const su_options *opt,
                              su_level_result *out);

/*
 * su_fma_peak -- measured multiply-add throughput of the current device in
 * SU_FP64 or SU_FP32 (independent FMA chains on every SM, CUDA-event timed,
 * best of three launches): *fma_per_s multiply-adds per second (x2 = flop/s).
 * A measurement utility for the ALU roofline of the sampler; the paper has no
 * counterpart.  Synchronous; allocates a small device buffer internally.
 */
int su_fma_peak(int precision, double *fma_per_s);

#ifdef __cplusplus
}
#endif

#endif /* SPEEDUP_H */
