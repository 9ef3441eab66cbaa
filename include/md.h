/*
 * md.h -- C ABI of libmd, a GB300 (sm_103a) implementation of the force
 * evaluation inside the fourth-order symplectic integrator of arXiv 1212.0262
 * (Rocha Filho, "Molecular dynamics for long-range interacting systems on
 * Graphic Processing Units") for three models:
 *
 *   MD_HMF     Hamiltonian Mean Field, Sec. 2 Eq. 2; mean-field force Eqs. 5-7
 *   MD_RING    Ring model, Sec. 2 Eq. 1; pair force Eqs. 8-9 (sign: minus the
 *              gradient of Eq. 1)
 *   MD_GRAV2D  2D self-gravitating particles, Sec. 2 Eq. 3 (natural log)
 *
 * Conventions shared by every call:
 *  - Return value: MD_OK (0) or a positive MD_E* code.  No C++ exception crosses
 *    the ABI.  The message of the last failure is md_last_error(ctx) (or
 *    md_last_error(NULL) when no context exists yet, e.g. md_init failing).
 *  - Layout: positions q and momenta p are structure-of-arrays of dim*N doubles,
 *    dim = 1 for HMF and Ring (q = theta) and dim = 2 for 2D
 *    (q = [x_0..x_{N-1}, y_0..y_{N-1}], p = [px..., py...]).
 *  - "host" pointers are ordinary (pageable or pinned) CPU memory owned by the
 *    caller and only read or written during the call.  "device" pointers are
 *    CUDA global memory on the context's device, owned by the caller.
 *  - Work is queued on the context's stream (md_set_stream; default: a stream the
 *    context creates).  Calls that return host values synchronise that stream.
 *  - A context is used by one host thread at a time.  Contexts are independent.
 *  - Floating point: the state (q, p), kicks, drifts and every reduction are FP64.
 *    MD_FP64 evaluates pair and mean-field forces in FP64; MD_MIXED evaluates
 *    the pair arithmetic (Ring, 2D) and the sines and cosines (HMF) in FP32 and
 *    accumulates per-particle sums in FP64 per tile (Sec. 3.2, last paragraph;
 *    Sec. 5).
 */
#ifndef MD_H
#define MD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* models */
#define MD_HMF 0
#define MD_RING 1
#define MD_GRAV2D 2
#define MD_GRAV3D 3 /* 3D self-gravitating particles: not one of the paper's three models
                     * (its introduction lists self-gravitating systems; its conclusion
                     * calls other N-particle systems a direct extension).  Unit masses,
                     * Kac 1/N coupling and additive softening as in Eqs. 1-3:
                     * V = -(1/N) sum_{i<j} (|r_ij|^2 + eps)^(-1/2),
                     * f_i = -(1/N) sum_j r_ij (|r_ij|^2 + eps)^(-3/2).
                     * md_grad / md_tangent_step with the kinetic observable. */
#define MD_SHEET1D 4 /* 1D self-gravitating sheets (named in the paper's introduction among
                      * long-range models, not studied there): unit masses, Kac 1/N coupling,
                      * V = (1/N) sum_{i<j} |x_i - x_j| for eps = 0 (f_i = -(1/N) sum_j
                      * sign(x_i - x_j), sign(0) = 0: exact integer counts), or
                      * sqrt((x_i - x_j)^2 + eps) for eps > 0.  eps >= 0.  In MD_MIXED the
                      * eps = 0 signs are decided on the FP32 positions.  md_grad and
                      * md_tangent_step need eps > 0 (the eps = 0 force is piecewise constant). */

/* precisions */
#define MD_FP64 0
#define MD_MIXED 1

/* status codes */
#define MD_OK 0
#define MD_EINVAL 1     /* bad argument (size, model, NULL, value out of range) */
#define MD_ENOMEM 2     /* device or host allocation failed */
#define MD_ECUDA 3      /* a CUDA call failed (message has the CUDA error string) */
#define MD_ETIMEOUT 4   /* a bounded device-side wait gave up */
#define MD_ENONFINITE 5 /* the state or an observable is NaN or infinite */
#define MD_ESTATE 6     /* call not valid in the context's current state */

/* initial-condition kinds for md_set_ic (all seeded, counter-based SplitMix64) */
#define MD_IC_WATERBAG 0     /* params[4] = {th_lo, th_hi, p_lo, p_hi}: theta (or the sheets' x)
                              * ~U[th_lo,th_hi), p~U[p_lo,p_hi) */
#define MD_IC_RING 1         /* params[1] = {sigma}: theta~U[-pi,pi), p~N(0,sigma^2) */
#define MD_IC_DISK 2         /* params[1] = {sigma}: uniform unit disk, p~N(0,sigma^2) per component */
#define MD_IC_ANNULUS 3      /* params[2] = {r1, r2}: uniform annulus r1<=r<r2, at rest */
#define MD_IC_UNIFORM_REST 4 /* params unused: theta~U[-pi,pi), at rest */
#define MD_IC_BALL 5         /* params[1] = {sigma}: uniform unit ball (r = u^(1/3), cos(polar) =
                              * 1 - 2u', azimuth 2 pi u''), p~N(0,sigma^2) per component */

/* observables for md_grad */
#define MD_OBS_KINETIC 0       /* O = (1/2) sum p^2 at the final time */
#define MD_OBS_MAGNETIZATION 1 /* O = |M| of Eq. 7 at the final time (HMF, Ring) */

typedef struct md_ctx md_ctx;
typedef struct md_batch md_batch;

/* Create a system of N particles of `model` with softening eps (Ring, 2D, 3D: must
 * be >= 1e-30; sheets: 0 or >= 1e-30; ignored for HMF but must be 0 or >= 1e-30; the
 * floor keeps every softened square distance a normal FP32 number, the precision of
 * the kernels' divisions and reciprocal seeds) and time step dt (Sec. 3, Eq. 4),
 * on the current CUDA device.  The state is drawn from `seed` with the model's
 * default recipe: water-bag theta~U[-1,1), p~U[-1.2,1.2) (HMF); theta~U[-pi,pi),
 * p~N(0,0.5^2) (Ring); uniform unit disk, p~N(0,0.3^2) per component (2D);
 * uniform unit ball, p~N(0,0.3^2) per component (3D; state layout x, y, z blocks);
 * water-bag x~U[-1,1), p~U[-0.5,0.5) (sheets).
 * Precision defaults to MD_FP64.  Returns NULL on failure (see md_last_error(NULL)).
 * The context owns its device memory until md_free. */
md_ctx *md_init(int model, int64_t N, double eps, double dt, uint64_t seed);

/* Release a context and its device memory.  NULL is ignored. */
void md_free(md_ctx *ctx);

/* Message of the last failure on ctx, or of the last failure of a call without a
 * context when ctx is NULL.  Never NULL; owned by the library. */
const char *md_last_error(const md_ctx *ctx);

/* Status code (MD_*) of the last failing call made by the calling thread (MD_OK if
 * none has failed): for calls that return no status, such as md_init returning NULL. */
int md_last_status(void);

/* MD_FP64 or MD_MIXED.  Takes effect for the next md_step / md_force / md_grad. */
int md_set_precision(md_ctx *ctx, int precision);

/* Queue all later work of ctx on `stream` (a cudaStream_t; NULL = legacy default
 * stream).  The caller keeps ownership of the stream. */
int md_set_stream(md_ctx *ctx, void *stream);

/* Change the time step (Sec. 3, Eq. 4).  dt may be negative (backward flow). */
int md_set_dt(md_ctx *ctx, double dt);

/* Change the softening eps of Eqs. 1 and 3 (the values md_init accepts). */
int md_set_eps(md_ctx *ctx, double eps);

/* Tuning knobs of the kernels (defaults: r_mixed 8, r_fp64 2, ring_tc 1, symmetric 1,
 * step_graphs 1, the rest 0):
 *   "r_mixed"          i-particles per thread of the FP32 pair kernels (4 or 8)
 *   "r_fp64"           i-particles per thread of the FP64 pair kernels (2 or 4)
 *   "pair_ctas_per_sm" CTAs per SM of the pair kernels (0 = occupancy limit)
 *   "pair_vcta"        stream-K ranges per resident CTA of the pair kernels, which the
 *                      CTAs take in turn from a counter (1 to 32; 0 = the kernel's
 *                      measured default: 8 for the symmetric FP32 Ring kernel, 3 for the
 *                      symmetric FP64 3D kernel, 4 otherwise)
 *   "hmf_ctas_per_sm"  CTAs per SM of the HMF stage kernels (0 = default: 4 for the FP32
 *                      sine/cosine stages, the occupancy limit otherwise)
 *   "ring_tc"          Ring FP32: sin(d) and sin(d/2) of Eq. 9 from split-TF32
 *                      tensor-core products (0 off; 1 or 2: 4 or 2 16-row blocks per warp)
 *   "symmetric"        forward stages of Ring (FP32: with ring_tc 1) and 2D, FP32 and
 *                      FP64 (r_fp64 2): every unordered pair evaluated once and added to
 *                      both particles (Newton's third law; the paper evaluates both
 *                      orders, Sec. 3.2).  Needs column-partial storage of about
 *                      N^2 / 128 bytes (Ring, FP32 or FP64), N^2 / 256 (FP32 2D),
 *                      N^2 / 64 (FP64 2D), 3 N^2 / 256 (FP32 3D) or N^2 / 512 (FP32
 *                      sheets); above 16 GiB of it (N beyond about 1.48e6 for Ring,
 *                      2.1e6 for FP32 2D) the one-sided kernel runs.
 *   "step_graphs"      md_step replays its steps after the first from captured CUDA
 *                      graphs of 8 steps (1, default) or launches every stage (0).
 * MD_EINVAL for an unknown key or value. */
int md_set_tuning(md_ctx *ctx, const char *key, int64_t value);

/* Which force kernel the context's next Ring / 2D stage runs (MD_KERNEL_*), from
 * its model, precision and tuning; -1 for a NULL context. */
#define MD_KERNEL_HMF 0          /* HMF mean-field stage (Sec. 3.1) */
#define MD_KERNEL_PAIRS_FP64 1   /* FP64 all-pairs, every ordered pair */
#define MD_KERNEL_PAIRS 2        /* FP32 all-pairs on the CUDA cores, every ordered pair */
#define MD_KERNEL_PAIRS_TC 3     /* FP32 with tensor-core products (Ring), every ordered pair */
#define MD_KERNEL_PAIRS_SYM 4    /* FP32 on the CUDA cores, every unordered pair once */
#define MD_KERNEL_PAIRS_TC_SYM 5 /* FP32 with tensor-core products (Ring), every unordered pair once */
#define MD_KERNEL_PAIRS_FP64_SYM 6 /* FP64 all-pairs, every unordered pair once */
int md_force_kernel(const md_ctx *ctx);

/* Redraw the state with recipe `kind` (MD_IC_*) and `params` from `seed`.
 * Draw order: positions (counters 0..dim*N-1; the disk and annulus use two
 * counters per particle), then momenta; Gaussians by Box-Muller from two
 * consecutive counters. */
int md_set_ic(md_ctx *ctx, int kind, const double *params, uint64_t seed);

/* Copy dim*N positions and momenta from host (set) or to host (get). */
int md_set_state(md_ctx *ctx, const double *q, const double *p);
int md_get_state(md_ctx *ctx, double *q, double *p);

/* Same with device pointers on the context's device (stream-ordered, async). */
int md_set_state_device(md_ctx *ctx, const double *q, const double *p);
int md_get_state_device(md_ctx *ctx, double *q, double *p);

/* Advance nsteps >= 0 integration steps of Sec. 3 (items 1-12 with Eq. 4's
 * splitting; three force evaluations per step, the force at the end of a step
 * reused by the next one).  Queued on the stream; returns without waiting.
 * After the call p and q sit on the step boundary. */
int md_step(md_ctx *ctx, int64_t nsteps);

/* One fused integrator stage (Sec. 3 step list): evaluate the force at the
 * current positions, kick p += b*dt*f, then drift q += d*dt*p (d == 0: kick only,
 * and for Ring/2D the force is kept for the next md_step).  md_step(n) is the
 * sequence (B0,D0) (B1,D1) (B1,D0), then n-1 times (2*B0,D0) (B1,D1) (B1,D0),
 * then (B0,0), with the Eq. 4 constants B0 = w1/2, B1 = (w0+w1)/2, D0 = w1,
 * D1 = w0 (w1 = 1/(2-2^(1/3)), w0 = -2^(1/3)/(2-2^(1/3))).  Asynchronous. */
int md_stage(md_ctx *ctx, double b, double d);

/* The four constants B0, B1, D0, D1 of Eq. 4 used by md_step (host array of 4). */
void md_yoshida(double *c4);

/* Forces at the current positions (Eq. 6 for HMF, minus the gradient of Eqs. 1/3
 * for Ring/2D) into host f[dim*N], at the context's precision.  Synchronous. */
int md_force(md_ctx *ctx, double *f);

/* Same into device f[dim*N] (stream-ordered). */
int md_force_device(md_ctx *ctx, double *f);

/* Total kinetic energy K = (1/2) sum p^2 and potential V (Eq. 5 for HMF; the
 * i<j pair sums of Eqs. 1 and 3 for Ring and 2D, and of the 3D potential of
 * MD_GRAV3D), both in FP64.  Synchronous.
 * MD_ENONFINITE if either is not finite.  Either pointer may be NULL. */
int md_energy(md_ctx *ctx, double *K, double *V);

/* Magnetization (Mx, My) of Eq. 7 in FP64 (HMF and Ring; MD_EINVAL otherwise). */
int md_magnetization(md_ctx *ctx, double *mx, double *my);

/* Gradient of an observable of the state reached after nsteps from the current
 * state, with respect to that current state and eps: a pure function of the
 * context (its state is unchanged afterwards).  Discrete adjoint of md_step's
 * map: reversed integration rebuilds the kick positions, restarting from an FP64
 * checkpoint stored every `checkpoint_every` steps (>= 1).
 * grad_q, grad_p: host arrays of dim*N (required); grad_eps, value: host scalars
 * (may be NULL; grad_eps is 0 for HMF).  Synchronous.  Uses the context's
 * precision for the force and Jacobian-vector products.  MD_EINVAL for
 * MD_OBS_MAGNETIZATION outside HMF and Ring, and for MD_SHEET1D at eps = 0. */
int md_grad(md_ctx *ctx, int observable, int64_t nsteps, int checkpoint_every,
            double *grad_q, double *grad_p, double *grad_eps, double *value);

/* Advance the state nsteps steps exactly as md_step, together with a tangent
 * vector (dq, dp) carried by the linearisation of the same discrete map
 * (forward-mode derivative: dp += b dt J(q) dq at each kick, dq += d dt dp at
 * each drift, J = df/dq).  The building block of largest-Lyapunov-exponent
 * estimates (repeat, renormalising the tangent).  dq, dp: host arrays of dim*N,
 * read and overwritten.  Uses the context's precision.  Synchronous.  MD_EINVAL for
 * MD_SHEET1D at eps = 0. */
int md_tangent_step(md_ctx *ctx, int64_t nsteps, double *dq, double *dp);

/* Largest-Lyapunov-exponent run on the device: the tangent (dq, dp) is normalised
 * to unit FP64 length, then carried with the state through nsteps steps of
 * md_tangent_step's linearised map, renormalised to unit length after every
 * renorm_every steps (and after the last, shorter block); *sum_log receives the sum
 * of the logarithms of the norms found at those renormalisations, so the estimate
 * is *sum_log / (nsteps dt).  dq, dp: host arrays of dim*N, read (any non-zero
 * vector) and overwritten with the final unit tangent.  The state advances nsteps
 * steps.  The tangent stays in device memory between renormalisations (no host
 * copies inside the run).  Uses the context's precision.  Synchronous.  MD_EINVAL
 * for MD_SHEET1D at eps = 0. */
int md_lyapunov(md_ctx *ctx, int64_t nsteps, int64_t renorm_every, double *dq, double *dp, double *sum_log);

/* Route the library's device allocations through alloc(bytes, user) and
 * free(ptr, user) (for example a caching allocator of the host framework).
 * alloc returns NULL on failure, which the library reports as MD_ENOMEM; it must
 * return device memory aligned to 256 bytes (a block that is not is handed back to
 * free and the allocation fails with MD_ENOMEM).  The library synchronises the
 * device before it passes a block to free (cudaFree would), so the allocator may
 * reuse it at once.
 * Passing NULL for both restores cudaMalloc / cudaFree.  Applies to allocations
 * made after the call; memory is freed by the allocator that made it. */
int md_set_allocator(void *(*alloc)(size_t bytes, void *user), void (*free_fn)(void *ptr, void *user),
                     void *user);

/* Potential energy V of a state held in caller-owned device memory, for callers
 * that cannot allocate device memory (a host framework's caching allocator that
 * owns the GPU's memory, or a latency-critical loop where cudaMalloc / cudaFree
 * and the device synchronisation they can cause are not acceptable).  The paper
 * has no counterpart; the value is md_energy's V (Eq. 5 for HMF, the i<j sums
 * of Eqs. 1 and 3 for Ring and 2D, and of the 3D and sheet potentials), computed
 * by the same kernels in FP64.
 *   model: MD_HMF, MD_RING, MD_GRAV2D, MD_GRAV3D or MD_SHEET1D; eps as for md_init
 *   N:     1 <= N <= 65536 (the size the static scratch holds); larger N is
 *          rejected with MD_EINVAL and a message in md_last_error(NULL)
 *   q:     device, dim*N doubles (layout as md_set_state), read only
 *   V:     device, one double, written (NaN or infinite if a position is)
 *   stream: cudaStream_t the work is queued on (asynchronous; no host sync); it must
 *          belong to the current device (MD_EINVAL otherwise)
 * Allocates nothing: its scratch is one file-scope device array of about 1.6 MB
 * that every GPU loading libmd holds until the process exits.  The first call
 * on a device looks up that array's device address and creates an event (make this
 * first call before any stream capture).  All calls share the array; each call waits
 * on its stream for the previous call on the device (that event) and records it, so
 * calls on different streams or from different host threads run one after another
 * on the GPU.  Inside a stream capture the wait is left out: calls captured into
 * graphs that may run concurrently must be ordered by the caller. */
int md_potential_noalloc(int model, int64_t N, double eps, const double *q, double *V, void *stream);

/* ----- row shards: one system split by rows among several ranks ----- */
/* The paper's two-GPU schemes generalised to P ranks.  HMF (Sec. 3.1, last
 * paragraph): every rank advances its own particles and the partial magnetizations
 * (sum cos, sum sin) of all ranks are added, in rank order, before every stage.
 * Ring and 2D (Sec. 3.2, Fig. 2 and its two-GPU stage list): every rank evaluates
 * the forces on its own rows against all N positions (every ordered pair, the
 * one-sided kernels) and, after every drift, the new positions of each rank are
 * copied to all others.
 *
 * Protocol.  Each rank has one context from md_shard_init.  md_shard_begin writes
 * the rank's own segment of its exchange buffer from its state; then, and after
 * every md_shard_stage, every rank's segment must be copied into the same byte
 * range of every other rank's exchange buffer (md_shard_buffer gives the buffer and
 * the segment) before the next md_shard_stage or md_shard_force: md_shard_exchange
 * does this for ranks held by one process; a multi-process transport copies the
 * same byte ranges.  md_shard_step runs whole steps of Eq. 4 with the exchange after
 * every stage.  md_step, md_stage, md_force, md_energy, md_magnetization, md_grad
 * and md_tangent_step answer MD_ESTATE on a shard context; md_get_state /
 * md_set_state (and the _device forms) read and write the rank's own rows
 * (dim * n_rows doubles, layout as for a whole system); after md_set_state,
 * md_set_ic or md_set_precision call md_shard_begin (and exchange) again. */

/* Rows [*lo, *hi) of rank `rank` of `nranks` for a system of N particles of
 * `model` (MD_HMF, MD_RING, MD_GRAV2D): lo = floor(N rank / nranks) rounded down to
 * a multiple of 1024 rows for Ring and 2D (whole mirror groups and i-tiles), of 1 for
 * HMF.  MD_EINVAL if a rank would get no rows or nranks is outside [1, 64]. */
int md_shard_range(int model, int64_t N, int rank, int nranks, int64_t *lo, int64_t *hi);

/* Context for rank `rank`'s rows of the system md_init(model, N, eps, dt, seed)
 * would make: its state is those rows of the same initial state (same counters).
 * Ring / 2D hold the whole N-particle position mirror besides their rows' state.
 * Returns NULL on failure (md_last_error(NULL)).  Free with md_free. */
md_ctx *md_shard_init(int model, int64_t N, double eps, double dt, uint64_t seed, int rank, int nranks);

/* Write this rank's segment of its exchange buffer from its current state
 * (asynchronous, on the context's stream). */
int md_shard_begin(md_ctx *ctx);

/* One fused stage over the rank's rows: force from the exchanged buffer, kick
 * p += b dt f, drift q += d dt p (d = 0: kick only), then this rank's segment of the
 * exchange buffer for the next stage.  Asynchronous.  MD_ESTATE before
 * md_shard_begin. */
int md_shard_stage(md_ctx *ctx, double b, double d);

/* The device exchange buffer of ctx for the stage that comes next (it alternates
 * between two buffers) and this rank's segment in it: bytes [*seg_offset,
 * *seg_offset + *seg_bytes).  HMF: 16 bytes (sum cos, sum sin) per rank; Ring / 2D:
 * the position records of the rank's rows (the last rank's also the padding). */
int md_shard_buffer(md_ctx *ctx, void **buf, size_t *seg_offset, size_t *seg_bytes);

/* Exchange between the nranks contexts ctx[0..nranks-1] (ctx[r] must be rank r of
 * the same system) held by this process, on the same or different devices: every
 * rank's stream waits for every other rank's last stage (an event) and copies the
 * other ranks' segments into its own buffer (cudaMemcpyAsync).  Asynchronous. */
int md_shard_exchange(md_ctx *const *ctx, int nranks);

/* nsteps >= 0 integration steps of Sec. 3 (Eq. 4 constants, merged kicks as md_step)
 * on all nranks shards of one system held by this process, with md_shard_exchange
 * after every stage; calls md_shard_begin and exchanges first when needed.
 * Asynchronous. */
int md_shard_step(md_ctx *const *ctx, int nranks, int64_t nsteps);

/* Forces on the rank's rows at the current (exchanged) positions into host
 * f[dim * n_rows], at the context's precision.  Synchronous. */
int md_shard_force(md_ctx *ctx, double *f);

/* Wait for all work queued on the context's stream. */
int md_synchronize(md_ctx *ctx);

/* Number of kernel launches the context has queued since it was created. */
int64_t md_launch_count(const md_ctx *ctx);

/* ----- batched ensembles: many independent systems advanced together ----- */

/* nsys independent Ring / 2D systems (model[s] in {MD_RING, MD_GRAV2D}) with
 * N[s] >= 1 particles, softening eps[s] > 0, step dt[s] and default initial
 * states drawn from seed[s].  All systems share one persistent force launch per
 * integrator stage and one captured CUDA graph per block of steps.  Precision is
 * MD_MIXED (FP32 pair arithmetic, FP64 state) unless md_batch_set_precision.
 * Returns NULL on failure (md_last_error(NULL)). */
md_batch *md_batch_init(int nsys, const int *model, const int64_t *N, const double *eps,
                        const double *dt, const uint64_t *seed);
void md_batch_free(md_batch *b);
int md_batch_set_precision(md_batch *b, int precision);
int md_batch_set_stream(md_batch *b, void *stream);
/* Advance every system by nsteps steps of Sec. 3 (asynchronous).  Three fused
 * force + kick + drift stages per step cover all systems (one launch per stage,
 * two in the Newton's-third-law form: pair phase and finish phase); blocks of
 * steps are replayed from a captured CUDA graph. */
int md_batch_step(md_batch *b, int64_t nsteps);
/* Kernel shape of the batched launches: r = 0 (default) runs the mixed-precision
 * Newton's-third-law kernels (every unordered pair of a system once; tensor-core
 * Ring products), r = 4 or 8 the one-sided kernels with r i-particles per thread
 * (FP64 ensembles always run the one-sided FP64 kernel); fraction `split` (0, 1)
 * of the CTAs given to the Ring systems; CTAs per SM (0 = occupancy limit). */
int md_batch_set_tuning(md_batch *b, int r, double split, int ctas_per_sm);
/* The current shape (after md_batch_autotune: the one it picked); NULL outputs
 * are skipped. */
int md_batch_get_tuning(const md_batch *b, int *r, double *split, int *ctas_per_sm);
/* Time candidate shapes (r, split, CTAs per SM) on force-only launches, which
 * leave every state unchanged, and keep the fastest.  *best_ms (may be NULL)
 * receives the fastest launch time.  Synchronous. */
int md_batch_autotune(md_batch *b, double *best_ms);
/* Forces of every system at its current positions, from one force-only launch of
 * the kernels md_batch_step runs (same form, precision and tuning): f[s] is a host
 * array of dim*N[s] doubles for system s, or NULL to skip that system (f itself
 * must not be NULL).  Minus the gradient of Eq. 1 (Ring) or Eq. 3 (2D).  States are
 * unchanged.  Synchronous. */
int md_batch_force(md_batch *b, double *const *f);
/* K[s], V[s] for every system (host arrays of nsys).  Synchronous. */
int md_batch_energy(md_batch *b, double *K, double *V);
/* Host state of system s (dim*N[s] doubles each). */
int md_batch_get_state(md_batch *b, int s, double *q, double *p);
int md_batch_set_state(md_batch *b, int s, const double *q, const double *p);
const char *md_batch_last_error(const md_batch *b);
int64_t md_batch_launch_count(const md_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* MD_H */
