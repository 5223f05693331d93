/*
 * nr.h -- C ABI of the GB300 (sm_103a) batched neutron-reflectivity library.
 *
 * The library evaluates, for a batch of layered slab models ("stacks"), the
 * specular reflectivity, the Gaussian log-likelihood of observed data, and
 * the exact gradient of that log-likelihood with respect to every slab and
 * instrument parameter -- the quantities that gradient-based optimisation,
 * Hamiltonian Monte-Carlo and variational inference evaluate at every step
 * in arXiv 2509.06924 (Secs. 2.2-2.4; the forward model of Sec. 2.1 and the
 * refjax kernel interface of Sec. 3).
 *
 * Physics (the paper names the Abeles matrix formalism, Sec. 2.1, and
 * Gaussian interfacial roughness, Sec. 3, but prints no equation; these are
 * the readings this library implements):
 *   media j = 0 (fronting) .. n+1 (backing), layers j = 1..n;
 *   k_0 = q/2,  k_j = sqrt(k_0^2 - 4 pi (rho_j - rho_0) + 4 pi i iota_j),
 *     principal root (Im k_j >= 0);
 *   r_j = (k_j - k_{j+1}) / (k_j + k_{j+1}) * exp(-2 k_j k_{j+1} sigma_j^2)
 *     (Nevot-Croce), j = 0..n;
 *   amplitude r = M_10 / M_00 of M = C_0 C_1 ... C_n with
 *     C_j = [[e^{-i b_j}, r_j e^{-i b_j}], [r_j e^{i b_j}, e^{i b_j}]],
 *     b_0 = 0, b_j = k_j d_j (equivalently the Parratt recursion);
 *   R(q) = |r|^2;
 *   smearing with a pointwise FWHM dQ (Sec. 3 smearing kernels; Sec. 4.1
 *     pointwise FWHM): S(Q) = sum_k w_k R(Q + dQ x_k / (2 sqrt(ln 2))),
 *     (x_k, sqrt(pi) w_k) the K-point Gauss-Hermite rule;
 *   model m = scale * S + bkg (instrument parameters, Sec. 2.1);
 *   loglik = -1/2 sum_i [((m_i - R_i)/e_i)^2 + ln(2 pi e_i^2)] (Gaussian
 *     likelihood with count-derived deviations, Sec. 2.1; chi^2 of Eq. 25).
 *
 * Packed parameters of one stack with n layers: 4n+6 doubles
 *     d[n] | rho[n+2] | iota[n+1] | sigma[n+1] | scale | bkg
 *   d: thicknesses (A) of layers 1..n; rho: SLD (absolute A^-2, e.g.
 *   2.07e-6 for Si) of fronting, layers, backing; iota: absorption
 *   (imaginary SLD, >= 0) of layers and backing (the fronting medium is
 *   non-absorbing); sigma: roughness (A) of interfaces 0..n, top to bottom.
 *   Stacks are packed back to back in stack order.
 *
 * Conventions of every call:
 *   - All calls return nr_status; on failure nr_last_error() gives a
 *     message (thread-local, valid until the next call on that thread).
 *   - Metadata arrays (n_layers, dataset, q_off) are HOST memory; bulk
 *     arrays (params, q, dq, r_obs, r_err) and outputs are DEVICE memory
 *     when batch->memory == NR_MEM_DEVICE, HOST memory (preferably pinned)
 *     when batch->memory == NR_MEM_HOST.  The library never frees or
 *     retains caller memory; host metadata is copied into the plan.
 *   - Device-memory calls are asynchronous on `stream` (a cudaStream_t,
 *     NULL = legacy default stream).  Host-memory calls copy in, compute
 *     and copy out on `stream` and return after the stream is synchronised.
 *   - Metadata is validated on the host (NR_EINVAL).  Problems that are only
 *     visible in device data (non-finite parameters, a quadrature node at
 *     q <= 0, e <= 0) never trap the GPU: the affected outputs become NaN
 *     and a sticky device flag is raised, read by nr_device_status().
 *   - A context is bound to the device that was current at nr_create and
 *     is not thread-safe; use one context per host thread.
 */
#ifndef NR_H_
#define NR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NR_MAX_LAYERS 64 /* n_layers in [0, NR_MAX_LAYERS]                  */
#define NR_MAX_QUAD 32   /* quadrature nodes K in [1, NR_MAX_QUAD]          */

typedef enum {
    NR_OK = 0,
    NR_EINVAL = 1,     /* bad argument or metadata                            */
    NR_ENOMEM = 2,     /* device or pinned-host allocation failed             */
    NR_ECUDA = 3,      /* a CUDA runtime call failed (message has the name)   */
    NR_ETIMEOUT = 4,   /* reserved: a bounded device wait gave up             */
    NR_ENONFINITE = 5  /* device data produced a non-finite or invalid value  */
} nr_status;

typedef enum {
    NR_MIXED = 0,      /* FP32 bulk with double-float guards (the fast path)  */
    NR_FP64_PLAIN = 1  /* plain FP64 forward; gradient by central differences */
} nr_precision;

typedef enum { NR_MEM_DEVICE = 0, NR_MEM_HOST = 1 } nr_memory;

/* Device status flags returned by nr_device_status (bitwise OR). */
#define NR_FLAG_NONFINITE_PARAM 1 /* a parameter was NaN/Inf                 */
#define NR_FLAG_BAD_Q 2           /* a quadrature node fell at q <= 0        */
#define NR_FLAG_BAD_ERR 4         /* an uncertainty e_i was <= 0 or NaN      */
#define NR_FLAG_DEBUG_BOUNDS 8    /* NR_DEBUG builds only: a kernel met a work
                                     item or queue slot outside its buffers
                                     and skipped it (its outputs are invalid) */

typedef struct nr_options {
    int32_t n_quad;        /* K quadrature nodes (default 17 when 0)          */
    int32_t precision;     /* nr_precision                                    */
    int32_t deterministic; /* 1: bitwise-reproducible reductions (default 1)  */
    int32_t autotune;      /* 1: nr_plan times launch shapes and caches them  */
    int32_t tile_q;        /* override: Q points per CTA tile (0 = auto)      */
    int32_t chunk_q;       /* override: Q points per work item (0 = auto)     */
    int32_t grid_ctas;     /* override: persistent CTAs (0 = auto)            */
    int32_t serial;        /* 1: launch the register buckets of a batch one
                              after another on the call's stream; 0 (default):
                              concurrently on forked streams joined back into
                              it (each bucket is one persistent launch)      */
} nr_options;

typedef struct nr_batch {
    int32_t n_stacks;         /* S >= 0                                       */
    int32_t n_datasets;       /* D >= 1 when S > 0                            */
    const int32_t *n_layers;  /* HOST [S]: layers of each stack               */
    const int32_t *dataset;   /* HOST [S]: dataset (Q grid + data) of a stack */
    const int64_t *q_off;     /* HOST [D+1]: dataset d owns points
                                 [q_off[d], q_off[d+1]); q_off[0] = 0         */
    int32_t memory;           /* nr_memory of the bulk arrays and outputs     */
    int32_t reserved;
    const double *params;     /* [sum_s (4 n_s + 6)] packed parameters        */
    const float *q;           /* [q_off[D]] momentum transfer Q > 0 (1/A)     */
    const float *dq;          /* [q_off[D]] resolution FWHM dQ >= 0 (1/A)     */
    const float *r_obs;       /* [q_off[D]] observed reflectivity (loglik*)   */
    const float *r_err;       /* [q_off[D]] its standard deviation e > 0      */
} nr_batch;

typedef struct nr_ctx nr_ctx;

/* Create a context on the current CUDA device.  opt may be NULL (defaults).
 * Allocates the context's device status word and computes the quadrature
 * rule.  Errors: NR_EINVAL (bad options), NR_ECUDA, NR_ENOMEM. */
nr_status nr_create(nr_ctx **out, const nr_options *opt);

/* Release the context, its plans and workspaces (synchronises the device). */
void nr_destroy(nr_ctx *ctx);

/* Message of the last non-OK status returned on this thread. */
const char *nr_last_error(void);

/* Validate the batch metadata, build its work list on the device and, when
 * the context was created with autotune = 1 (NR_MIXED, device-memory
 * batches), time candidate launch shapes on the batch's own data: per
 * register bucket the two-evaluations-per-thread and the one-evaluation
 * kernel at the widest tile and at half of it; the fastest is kept for the
 * plan.  Optional: the compute calls plan on first use (without tuning).
 * Must precede CUDA-graph capture of a compute call, which then allocates
 * nothing and copies no metadata.  Errors: NR_EINVAL, NR_ENOMEM, NR_ECUDA. */
nr_status nr_plan(nr_ctx *ctx, const nr_batch *batch);

/* Smeared model m = scale * S(Q_i) + bkg for every stack and Q point of its
 * dataset.  r_out: [sum_s len(dataset(s))] floats, stack-major, in stack
 * order (stack s starts at the sum of the dataset lengths of stacks < s).
 * Forward model of Sec. 2.1 with the smearing of Sec. 3. */
nr_status nr_reflectivity(nr_ctx *ctx, const nr_batch *batch, float *r_out, void *stream);

/* Gaussian log-likelihood of each stack against its dataset (Sec. 2.1;
 * chi^2 term of Eq. 25).  loglik: [S] doubles.  r_obs and r_err required. */
nr_status nr_loglik(nr_ctx *ctx, const nr_batch *batch, double *loglik, void *stream);

/* Log-likelihood and its gradient w.r.t. all packed parameters (the exact
 * gradient of Secs. 2.2-3; hand-written adjoint under NR_MIXED, central
 * differences of the FP64 forward under NR_FP64_PLAIN).  grad: packed
 * exactly like params.  Either output pointer may be NULL. */
nr_status nr_loglik_grad(nr_ctx *ctx, const nr_batch *batch, double *loglik, double *grad,
                         void *stream);

/* nr_loglik_grad plus the derivative of each stack's log-likelihood in a
 * shared resolution scale: every dQ_i of the stack's dataset is taken as
 * f * dQ_i and grad_res[s] = d loglik_s / d ln f at f = 1.  A fit that
 * infers a common smearing percentage (the LED co-fit's resolution
 * parameter, Sec. 4.2) needs it: with dQ_i = f Q_i, d loglik / d f =
 * grad_res / f.  The adjoint carries it through the quadrature nodes,
 * dq_k / d ln f = dQ_i x_k / (2 sqrt(ln 2)) (Gaussian smearing of Sec. 3).
 *   grad_res: [S] doubles, same memory kind as the batch; loglik and grad as
 *             for nr_loglik_grad (either may be NULL).
 * NR_MIXED only: a context created with NR_FP64_PLAIN returns NR_EINVAL.
 * Other errors as for nr_loglik_grad. */
nr_status nr_loglik_grad_res(nr_ctx *ctx, const nr_batch *batch, double *loglik, double *grad,
                             double *grad_res, void *stream);

/* SLD and absorption depth profiles of every stack, the curves the paper's
 * figures draw with posterior bands (Sec. 4.1 quartz film, Sec. 4.2 LED):
 *   rho(z) = rho_0 + sum_{j=0..n} (rho_{j+1} - rho_j) (1 + erf((z - z_j) / (sqrt(2) sigma_j))) / 2
 * with z_j = d_1 + ... + d_j the depth of interface j below the fronting
 * (z_0 = 0), and iota(z) alike (iota_0 = 0); sigma_j = 0 is a sharp step
 * that takes the deeper medium's value at z = z_j.
 *   batch:    only n_stacks, n_layers (HOST), params and memory are read;
 *             datasets may be absent.
 *   z, nz:    depths in A (same memory kind as the batch), shared by all stacks.
 *   rho_out, iota_out: [n_stacks * nz] floats, stack-major (either may be
 *             NULL, not both).
 * Device batches run asynchronously on `stream`; host batches are staged
 * and synchronised.  The call uploads the stacks' parameter offsets into a
 * context buffer: calls of one context must not overlap on different
 * streams.  Non-finite parameters (or sigma < 0) raise
 * NR_FLAG_NONFINITE_PARAM.  Errors: NR_EINVAL, NR_ECUDA. */
nr_status nr_sld_profile(nr_ctx *ctx, const nr_batch *batch, const float *z, int32_t nz, float *rho_out,
                         float *iota_out, void *stream);

/* Synchronise `stream`, return the sticky device flags raised since the
 * last call (NR_FLAG_*) in *flags and clear them.  Returns NR_ENONFINITE
 * when any flag was set, NR_OK otherwise. */
nr_status nr_device_status(nr_ctx *ctx, void *stream, int32_t *flags);

/* The library's own K-point Gauss-Hermite rule for exp(-x^2) (host
 * computation; x and w are HOST arrays of K doubles). */
nr_status nr_quadrature(int32_t K, double *x, double *w);

/* Evaluations (stack x Q point x quadrature node) one compute call performs
 * on this batch, and the launch shape last chosen for it (for reporting).
 * Any output pointer may be NULL. */
nr_status nr_plan_info(nr_ctx *ctx, const nr_batch *batch, int64_t *evals, int32_t *tile_q,
                       int32_t *chunk_q, int32_t *grid_ctas, int32_t *launches);

/* The launches one compute call makes on this batch after planning (and
 * tuning), one per register bucket: grad = 1 the gradient calls, 0 the
 * forward ones (model, log-likelihood).  *count receives the number of
 * buckets; for i < min(*count, max_groups): nmax[i] the bucket's layer
 * capacity (1: exactly one layer; 0: any, forward), paired[i] 1 when the
 * two-evaluations-per-thread kernel runs it, tile_q[i] Q points per CTA
 * tile, grid[i] persistent CTAs, items[i] work items.  Arrays may be NULL. */
nr_status nr_plan_groups(nr_ctx *ctx, const nr_batch *batch, int32_t grad, int32_t max_groups, int32_t *count,
                         int32_t *nmax, int32_t *paired, int32_t *tile_q, int32_t *grid, int32_t *items);

/* ------------------------------------------------------------------------
 * Autotune cache.  nr_plan on a context created with autotune = 1 times the
 * candidate launch shapes of every register bucket (paired or one-evaluation
 * kernel x tile of TQ or TQ/2 Q points x CTAs per SM at the occupancy limit,
 * one fewer, or half) on the batch's own data and keeps the fastest.  When
 * the environment variable NR_TUNE_CACHE names a file, the choices are read
 * from it first and the new ones written back (a JSON object
 * {"version": 1, "entries": {key: {"paired", "tile_q", "ctas_per_sm",
 * "ms"}}}), so later processes skip the timing.  Key of an entry:
 *   "<GPU name>|<SMs>|<mode>|<K>|<bucket nmax>|<log2 of the work items>|t<tuner version>"
 * with mode 0 for the forward and 2 for the gradient launches.  The two
 * calls below read and write one entry of such a file; they are host-only
 * (no device needed).  _get returns NR_EINVAL when the file or the key is
 * absent or unreadable; _put rewrites the file (keys may not contain '"'
 * or '\'), NR_EINVAL on an I/O error.
 * ---------------------------------------------------------------------- */
typedef struct nr_tune_entry {
    int32_t paired;      /* 1: the two-evaluations-per-thread kernel          */
    int32_t tile_q;      /* Q points per CTA tile                              */
    int32_t ctas_per_sm; /* persistent CTAs per SM                             */
    int32_t reserved;
    double ms;           /* time of the chosen shape's launch when tuned (ms) */
} nr_tune_entry;

nr_status nr_tune_cache_get(const char *path, const char *key, nr_tune_entry *entry);
nr_status nr_tune_cache_put(const char *path, const char *key, const nr_tune_entry *entry);

/* ------------------------------------------------------------------------
 * nr_loglik_grad_noalloc -- log-likelihood and gradient without allocating.
 * The paper has no counterpart: this entry point exists for callers that are
 * not allowed to allocate device memory (a plug-in whose host application
 * owns every allocation through its own pool, a real-time loop that must not
 * enter the driver's allocator, a process that has reserved the GPU's memory
 * up front).  It needs no context and no plan and calls no cudaMalloc or
 * cudaFree: its work list, queue tickets and status word live in one fixed
 * device array of the library (about 1 MiB, held by every GPU that loads the
 * library until the process exits).
 *
 *   batch:        as for nr_loglik_grad, DEVICE memory only
 *                 (batch->memory == NR_MEM_DEVICE), at most
 *                 NR_NOALLOC_MAX_STACKS stacks; r_obs and r_err required.
 *   n_quad:       quadrature nodes K in [1, NR_MAX_QUAD].
 *   loglik, grad: device outputs as for nr_loglik_grad (either may be NULL).
 *   device_flags: optional device int32; cleared, then given the NR_FLAG_*
 *                 bits this call raised (NULL: flags are not reported).
 *   stream:       cudaStream_t.  The work list is copied from pageable
 *                 host memory of the library, so the call waits for the
 *                 stream's earlier work before that copy and returns once
 *                 it is staged; the kernels then run asynchronously.
 * Returns NR_EINVAL (with a message in nr_last_error) for more than
 * NR_NOALLOC_MAX_STACKS stacks, host-memory batches, bad metadata or a
 * stream that is capturing a CUDA graph (this entry point cannot be
 * captured: a replay would copy whatever work list the latest call left in
 * the library's host arrays), NR_ECUDA if a runtime call fails.
 * The first call on a device looks up the array's device address with that
 * device current.  Every call shares the
 * one array and leaves its contents behind (the call clears what must start
 * at zero), so calls that overlap on the GPU (e.g. on two streams) race:
 * issue them on one stream.  Results equal nr_loglik_grad's up to rounding
 * (bitwise when nr_loglik_grad keeps whole stacks in one work item).
 * ---------------------------------------------------------------------- */
#define NR_NOALLOC_MAX_STACKS 16384

nr_status nr_loglik_grad_noalloc(const nr_batch *batch, int32_t n_quad, double *loglik, double *grad,
                                 int32_t *device_flags, void *stream);

/* ------------------------------------------------------------------------
 * On-device Hamiltonian Monte Carlo over many chains of a co-fitted model
 * (Sec. 2.3: leapfrog integration, Eq. 7, of L steps of size dt with a
 * diagonal mass matrix, then the Metropolis-Hastings acceptance of Eq. 8).
 *
 * Model of one chain: P free parameters theta_k with uniform priors on
 * [lo_k, hi_k] (the priors of Tables 1-4), sampled in unconstrained
 * coordinates u (Sec. 2.3.1's advice for bounded parameters):
 *   theta_k = lo_k + (hi_k - lo_k) / (1 + exp(-u_k)),
 *   log pi(u) = sum_c loglik_c(theta(u)) + sum_k [log s_k + log(1 - s_k)],
 * s_k the sigmoid of u_k (prior density times Jacobian).  Each of the
 * chain's n_contrasts contrasts is one stack whose packed slots (layout as
 * nr_batch.params) either copy a free parameter (slot_src = k, tied across
 * contrasts, e.g. a co-fitted substrate SLD or shared layers) or hold the
 * fixed value slot_val.  Contrast c is fitted to dataset[c].
 * ---------------------------------------------------------------------- */
typedef struct nr_cofit_model {
    int32_t n_chains;         /* C >= 1                                         */
    int32_t n_contrasts;      /* stacks per chain, >= 1                         */
    int32_t n_free;           /* P >= 1 free parameters per chain               */
    const int32_t *n_layers;  /* [n_contrasts] HOST                             */
    const int32_t *dataset;   /* [n_contrasts] HOST, into the datasets below    */
    int32_t n_datasets;
    const int64_t *q_off;     /* [n_datasets + 1] HOST, as nr_batch             */
    const float *q, *dq;      /* DEVICE, as nr_batch                            */
    const float *r_obs, *r_err;
    const int32_t *slot_src;  /* [sum_c (4 n_c + 6)] HOST: k in [0, P) or -1    */
    const double *slot_val;   /* [same] HOST: value of the fixed slots          */
    const double *lo, *hi;    /* [P] HOST: prior bounds, finite, lo < hi        */
    int32_t res_param;        /* free parameter k that scales every dQ of every
                                 contrast (dQ_i -> theta_k dQ_i: a shared
                                 resolution / smearing percentage, Sec. 4.2;
                                 its gradient comes from the resolution
                                 derivative of nr_loglik_grad_res); -1: none  */
} nr_cofit_model;

typedef struct nr_sampler nr_sampler;

/* Build a sampler for the model on the context's device: copies the slot
 * tables and bounds, allocates the per-chain workspaces and plans the
 * likelihood batch of C x n_contrasts stacks (chain-major).  The data
 * arrays are referenced, not copied: they must outlive the sampler.
 * Errors: NR_EINVAL (bad model), NR_ENOMEM, NR_ECUDA. */
nr_status nr_sampler_create(nr_ctx *ctx, const nr_cofit_model *model, nr_sampler **out);

/* Release the sampler (synchronises the device).  A sampler computes in its
 * context: destroy samplers before the context. */
void nr_sampler_destroy(nr_sampler *sampler);

/* log pi(u) [C] and its gradient d log pi / du [C x P] (either may be NULL)
 * at u [C x P]; all DEVICE, asynchronous on `stream`. */
nr_status nr_sampler_logp_grad(nr_sampler *sampler, const double *u, double *logp, double *grad,
                               void *stream);

/* One HMC transition of every chain.
 *   u:        [C x P] DEVICE, the chains' states; replaced by the accepted
 *             end points (rejected chains keep theirs).
 *   z:        [C x P] DEVICE standard-normal draws; the momentum is
 *             p = z / sqrt(inv_mass).
 *   log_unif: [C] DEVICE logs of uniform draws; a chain accepts iff
 *             log_unif < H(start) - H(end) (Eq. 8; NaN rejects).
 *   inv_mass: [P] DEVICE diagonal of M^-1.  eps: step dt; n_leapfrog: L >= 1.
 *   logp:     [C] DEVICE log pi of the resulting states (may be NULL).
 *   accepted: [C] DEVICE 1 / 0 (may be NULL).
 * L + 1 likelihood-gradient evaluations of the C x n_contrasts batch; no
 * allocation and no host synchronisation once the sampler exists, so a
 * step can be captured in a CUDA graph.  Errors: NR_EINVAL, NR_ECUDA. */
nr_status nr_hmc_step(nr_sampler *sampler, double *u, const double *z, const double *log_unif,
                      const double *inv_mass, double eps, int32_t n_leapfrog, double *logp, int32_t *accepted,
                      void *stream);

/* ------------------------------------------------------------------------
 * Variational inference with many independent restarts (Sec. 2.4; the LED
 * co-fit of Sec. 4.2 runs restarts of a multivariate normal q in an
 * unconstrained space, optimised by Adam).  The sampler's chains are the
 * restarts: R = n_chains.  q(u; phi) = N(mu, L L^T) over the sampler's
 * unconstrained coordinates.
 *   phi:      [R x (P + P (P + 1) / 2)] DEVICE, per restart mu [P] then the
 *             lower triangle of L row by row ((i, j <= i) at
 *             i (i + 1) / 2 + j) with log L_ii on the diagonal; updated.
 *   adam_m, adam_v: Adam's first and second moments, same shape (start at 0).
 *   t:        DEVICE int32 counter of the iterations done (start at 0); the
 *             call increments it on the device, so a captured call advances
 *             it on every graph replay.
 *   eps:      [R x P] DEVICE standard-normal draws, u = mu + L eps.
 *   opt:      HOST Adam settings (lr > 0, 0 <= beta1, beta2 < 1, eps > 0).
 *   elbo:     [R] DEVICE single-sample ELBO estimates at the incoming phi
 *             (log pi(u) + eps^T eps / 2 + sum log L_ii + P/2 log 2 pi; may
 *             be NULL).
 * One iteration: u = mu + L eps, log pi and its gradient at u (one
 * likelihood-gradient evaluation of R x n_contrasts stacks), the gradient of
 * the single-sample negative ELBO (Eqs. 22-24) with eps held fixed, and one
 * Adam step of every entry of phi.  No allocation or synchronisation: a
 * step can be captured in a CUDA graph.  Errors: NR_EINVAL, NR_ECUDA. */
typedef struct nr_adam {
    double lr, beta1, beta2, eps;
} nr_adam;

nr_status nr_vi_step(nr_sampler *sampler, double *phi, double *adam_m, double *adam_v, int32_t *t,
                     const double *eps, const nr_adam *opt, double *elbo, void *stream);

/* ------------------------------------------------------------------------
 * Testing hook (the paper has no counterpart): the next `count` device
 * allocations the library attempts (context status word, plans, work lists,
 * staging buffers, sampler workspaces) fail as if the device were out of
 * memory, without calling cudaMalloc; the call that needed one returns
 * NR_ENOMEM and leaves the context usable.  0 disarms.  Process-wide.
 * ---------------------------------------------------------------------- */
nr_status nr_debug_fail_allocs(int32_t count);

/* Testing hook of NR_DEBUG builds (release builds return NR_EINVAL): with
 * on = 1, the first work item of the batch's gradient plan (planned by this
 * call if needed) is given a stack index one past the batch, as a corrupted
 * plan would hold; the next gradient call's kernels must report
 * NR_FLAG_DEBUG_BOUNDS and skip that item (its stack's outputs are then
 * invalid) instead of reading outside the stack array.  on = 0 restores the
 * item and clears the plan's per-stack arrival counters, after which the plan
 * computes correctly again.  Synchronous. */
nr_status nr_debug_poison_plan(nr_ctx *ctx, const nr_batch *batch, int32_t on);

#ifdef __cplusplus
}
#endif

#endif /* NR_H_ */
