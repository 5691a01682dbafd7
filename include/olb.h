/*
 * olb.h -- C ABI of the GB300 (sm_103a) off-lattice Boltzmann library.
 *
 * The library advances the two-dimensional thermal lattice Boltzmann model
 * for van der Waals fluids of Busuioc, Ambrus, Biciusca and Sofonea
 * (arXiv:1702.01690) by whole TVD RK-3 steps on one GPU.  Each stage
 * evaluates, at every node, for the 25 populations f_kappa on the
 * Gauss-Hermite Q = 5 velocity set (Sec. 2.2, Table trots)
 *
 *   L[f] = -p . grad f  (WENO-5 fluxes, Sec. 3.2)
 *          -F . (grad_p f)  (Eq. derf; force F of Eq. F_def from the 49-point
 *                            stencils of Sec. 3.3)
 *          -(f - f^eq)/tau  (Eqs. evolution, feq)
 *
 * and combines the stages as in Eq. rk3.  Sides normal to x are periodic,
 * diffuse-reflection walls (Sec. 3.4.2) or specular-reflection planes
 * (Sec. 3.4.1); sides normal to y are periodic or specular.
 *
 * Conventions
 *  - Every call returns an int status: OLB_OK (0) or a negative OLB_ERR_*.
 *    No call throws or aborts; olb_status_string() names a status.
 *  - Host arrays are caller-owned and only read or written during the call.
 *    Device arrays are caller-owned device pointers on the context's device;
 *    the library reads or writes them in stream order on the context's
 *    stream and keeps no reference after the call returns.
 *  - Fields are FP64 arrays of nx*ny values in row-major [ny][nx] order: the
 *    value of node (i, j), 0-based, at x = (i + 1/2) ds, y = (j + 1/2) ds
 *    (Sec. 3.4), is element j*nx + i.
 *  - Populations are exchanged as FP64 arrays [25][ny][nx]; population
 *    kappa = 5*k1 + k2 has velocity (R[k1], R[k2]) with R the roots of He_5
 *    in ascending order (Table trots).
 *  - A context owns all device memory it uses and runs all its work on one
 *    CUDA stream (the one given to olb_create, or the legacy default stream
 *    for NULL).  A context is not thread-safe; distinct contexts are
 *    independent.
 */
#ifndef OLB_H
#define OLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    OLB_OK = 0,
    OLB_ERR_ARG = -1,      /* invalid argument (NULL pointer, bad size or enum) */
    OLB_ERR_CFL = -2,      /* p_max dt / ds >= 1 (Sec. 4.1) or dt > 2.5 tau */
    OLB_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    OLB_ERR_DIVERGED = -4, /* a moment became non-finite, n <= 0, b n >= 1 or T <= 0 */
    OLB_ERR_TIMEOUT = -5,  /* reserved: a bounded device wait ran out */
    OLB_ERR_STATE = -6,    /* call out of order (e.g. olb_step before init) */
    OLB_ERR_NOMEM = -7     /* device allocation failed */
};

/* Boundary kinds of the sides normal to x (side_x) and y (side_y).  A
 * specular side (Sec. 3.4.1) is a mirror plane: its three ghost layers hold
 * the populations of the first three nodes inside with the normal velocity
 * component reversed; n and Delta p are reflected evenly at walls and
 * specular sides alike, with a double reflection at corners (Sec. 3.4.3). */
enum {
    OLB_SIDE_PERIODIC = 0,         /* wrap modulo the grid size */
    OLB_SIDE_DIFFUSE = 1,          /* diffuse-reflection walls at x = 0 and
                                      x = nx ds (Sec. 3.4.2); side_x only */
    OLB_SIDE_SPECULAR = 2,         /* specular reflection on both sides */
    OLB_SIDE_SPECULAR_DIFFUSE = 3  /* specular at x = 0, diffuse wall at
                                      x = nx ds (the half channel of Sec. 4,
                                      the reduced Laplace domain of Sec. 5);
                                      side_x only */
};

/* Arithmetic of the populations. */
enum {
    OLB_FP64 = 0,       /* everything in FP64 */
    OLB_FP32_KAHAN = 1  /* FP32 arithmetic with compensated storage: every
                           population held as a pair hi + lo of floats (the
                           same 8 bytes as FP64), fluxes and stencils in FP32
                           on first differences of the pairs, the 25-velocity
                           moment sums compensated (double-float), T and
                           Delta p recovered in double-float arithmetic, the
                           RK-3 combination in double-float arithmetic */
};

/* Non-linear WENO weights. */
enum {
    OLB_WENO_JS = 0,     /* Jiang-Shu weights of Eq. weno5_omega, Table tab:weno */
    OLB_WENO_LEARNED = 1 /* weights from a trained network (olb_set_weno_mlp) where the
                            stencil is not smooth (min sigma_q < 0.9 max sigma_q, no
                            vanishing indicator); Jiang-Shu weights and Table tab:weno
                            elsewhere; single contexts only */
};

/* Problem statement (Sec. 2, Sec. 3).  Walls: index 0 is the wall at x = 0,
 * index 1 the wall at x = nx ds. */
typedef struct olb_params {
    int nx, ny;         /* nodes along x and y, >= 1 (>= 3 along an axis
                           whose sides are walls or specular) */
    double ds;          /* lattice spacing delta s > 0 (Sec. 2.1) */
    double dt;          /* time step delta t > 0 (Sec. 3.1) */
    double tau;         /* relaxation time tau > 0, constant (Eq. evolution) */
    double a, b;        /* van der Waals p^w = n T / (1 - b n) - a n^2;
                           a = 9/8, b = 1/3 is Eq. vdw; a = b = 0 is the ideal gas */
    double sigma;       /* surface-tension parameter of Eq. F_def, >= 0 */
    double Tw[2];       /* wall temperatures T_w > 0 at x = 0 and x = nx ds
                           (used at diffuse walls) */
    double uw[2];       /* tangential (y) wall velocities u_w */
    int side_x;         /* OLB_SIDE_PERIODIC, _DIFFUSE, _SPECULAR or
                           _SPECULAR_DIFFUSE */
    int side_y;         /* OLB_SIDE_PERIODIC or OLB_SIDE_SPECULAR */
    int precision;      /* OLB_FP64 or OLB_FP32_KAHAN */
    int weno_mode;      /* OLB_WENO_JS or OLB_WENO_LEARNED */
} olb_params;

typedef struct olb_ctx olb_ctx;

/* Allocator hook.  alloc(bytes, stream, user) returns device memory on the
 * current device or NULL; release(ptr, bytes, stream, user) frees it.  The
 * hook is process-wide and applies to contexts created after the call;
 * passing NULL for both restores cudaMalloc / cudaFree.  Returns OLB_ERR_ARG
 * if exactly one of the two is NULL.  Not part of the paper: it lets a host
 * framework (e.g. a caching allocator) own the device memory. */
typedef void *(*olb_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*olb_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
int olb_set_allocator(olb_alloc_fn alloc, olb_free_fn release, void *user);

/* Validate *p and create a context on the current CUDA device, using
 * `stream` (a cudaStream_t, or NULL for the legacy default stream) for all
 * its work.  Device memory (3 population buffers of 25 nx ny values and the
 * stage fields) is allocated here and nothing is launched.  Rejects
 * nx, ny < 1, nx < 3 with walls, ds, dt, tau <= 0, sigma < 0, b < 0,
 * Tw <= 0 with walls, unknown enums (OLB_ERR_ARG) and
 * p_max dt / ds >= 1 or dt > 2.5 tau (OLB_ERR_CFL; CFL rule of Sec. 4.1,
 * p_max = sqrt(5 + sqrt 10)).  On success *out receives the context. */
int olb_create(const olb_params *p, void *stream, olb_ctx **out);

/* Release the context and its device memory (synchronises its stream).
 * NULL is accepted. */
void olb_destroy(olb_ctx *ctx);

/* Set f = f^eq(n, u, T) at every node (Eq. feq) from host fields [ny][nx]
 * and reset the status word.  Rejects non-finite values, n <= 0,
 * b n >= 1 and T <= 0 with OLB_ERR_ARG before touching the device.
 * Page-locked (pinned) host arrays are read by the kernel directly, other
 * host memory through a staging copy; either way the call returns after the
 * device work is complete and the caller keeps ownership of the arrays. */
int olb_init_fields(olb_ctx *ctx, const double *n, const double *ux,
                    const double *uy, const double *T);

/* As olb_init_fields with device pointers (FP64, [ny][nx]), enqueued on the
 * context's stream without synchronisation; the values are not validated
 * on the host (olb_step's status check sees invalid ones). */
int olb_init_fields_device(olb_ctx *ctx, const double *n, const double *ux,
                           const double *uy, const double *T);

/* Advance nsteps >= 0 full RK-3 steps (Eq. rk3), then synchronise and
 * return OLB_ERR_DIVERGED if any stage met a non-finite moment, n <= 0,
 * b n >= 1 or T <= 0 (the populations then hold the diverged state),
 * else OLB_OK. */
int olb_step(olb_ctx *ctx, int nsteps);

/* As olb_step but only enqueues the work on the context's stream; the
 * status is read by olb_get_status. */
int olb_step_async(olb_ctx *ctx, int nsteps);

/* Synchronise the context's stream and return the status word accumulated
 * since the last init (OLB_OK or OLB_ERR_DIVERGED). */
int olb_get_status(olb_ctx *ctx);

/* Moments n, u_x, u_y, T of the current populations (Sec. 2.2; T from the
 * trace of Eq. sigmaq_def) into host arrays [ny][nx].  Any argument may be
 * NULL to skip it.  Page-locked (pinned) host arrays are written by the
 * kernel directly, others through a staging copy.  Returns after the values
 * are in the host arrays. */
int olb_moments(olb_ctx *ctx, double *n, double *ux, double *uy, double *T);

/* As olb_moments into device arrays (FP64, [ny][nx]), enqueued on the
 * context's stream without synchronisation. */
int olb_moments_device(olb_ctx *ctx, double *n, double *ux, double *uy,
                       double *T);

/* Global sums over the grid of the current populations, computed on the
 * GPU in FP64 (FP32 contexts sum their hi + lo pairs in FP64) in a fixed
 * order, so that repeated calls on the same state agree bit for bit:
 *   out[0] = sum_nodes n ds^2                       (mass, Sec. 2.2)
 *   out[1] = sum_nodes n u_x ds^2, out[2] = ... n u_y ds^2   (momentum)
 *   out[3] = sum_nodes sum_kappa |p|^2/2 f ds^2 = sum n (T + |u|^2/2) ds^2
 *            (kinetic energy of the particles, Eq. sigmaq_def with m = 1)
 * out: host array of 4 doubles.  Mass is conserved between periodic sides
 * and diffuse walls alike (zero net wall flux, Eq. nw); energy is exchanged
 * with the walls and with the van der Waals force.  Returns after the values
 * are in out. */
int olb_totals(olb_ctx *ctx, double *out);

/* Advance nsteps >= 0 RK-3 steps as olb_step does and record the four sums
 * of olb_totals after every `every` >= 1 steps: out (host) receives
 * floor(nsteps / every) records of 4 doubles, record r after (r + 1) every
 * steps.  At most nx * ny records (OLB_ERR_ARG otherwise).  Returns the
 * status of olb_step. */
int olb_step_totals(olb_ctx *ctx, int nsteps, int every, double *out);

/* Copy the populations to / from a host array [25][ny][nx] in FP64 (FP32
 * contexts round on set).  Used for checkpoint / resume and parity checks.
 * Both return after the copy is complete. */
int olb_get_populations(olb_ctx *ctx, double *f);
int olb_set_populations(olb_ctx *ctx, const double *f);

/* Per-kernel timing (not part of the paper; the tracing hook of the
 * library).  Runs nsteps >= 1 RK-3 steps on the context's stream as
 * individual launches of the stage kernel, each bracketed by CUDA events,
 * synchronises, and writes the mean device time in milliseconds of one
 * launch to ms[0] and the number of launches to launches[0] (either may be
 * NULL).  The populations advance exactly as with olb_step. */
int olb_profile(olb_ctx *ctx, int nsteps, double *ms, int *launches);

/* Shape of the stage kernel: tx x ty nodes per CTA, kp velocities advanced
 * at once (kp lanes of tx*ty threads, each rounded up to whole warps).
 * Compiled shapes (tx, ty, kp): (8,8,4), (16,8,2), (16,8,1), (32,8,1),
 * (32,16,1), (8,8,8), (7,8,8), (8,8,5); olb_create picks one from the
 * grid size (FP64: (8,8,4), or (7,8,8) when that lowers the most nodes one
 * SM advances; FP32: (8,8,5), or (8,8,4) with learned weights).  With
 * OLB_WENO_LEARNED only (8,8,4), (16,8,2), (32,16,1).  olb_set_tile returns
 * OLB_ERR_ARG for any other shape; results do not depend on the shape.
 * Not part of the paper (a tuning knob). */
int olb_set_tile(olb_ctx *ctx, int tx, int ty, int kp);
int olb_get_tile(olb_ctx *ctx, int *tx, int *ty, int *kp);

/* ------------------------------------------------------------------------
 * Batches: many independent runs (uneven grid sizes, each with its own
 * olb_params) advanced together, one launch per RK-3 stage with one CTA per
 * (run, tile) work item, replayed from CUDA graphs.  Not
 * part of the paper: it serves parameter sweeps (ds, T_w, drop radius) whose
 * single grids are too small to fill the GPU.  All runs must share the
 * precision.  Conventions as for single contexts; `run` indexes the array
 * given to olb_batch_create.  Device memory is allocated with cudaMalloc.
 * ------------------------------------------------------------------------ */
typedef struct olb_batch olb_batch;

/* Validate every run as olb_create does (first failing code returned) and
 * create the batch on the current device, working on `stream`. */
int olb_batch_create(const olb_params *runs, int count, void *stream, olb_batch **out);
void olb_batch_destroy(olb_batch *b);

/* f = f^eq of host fields [ny][nx] for one run (as olb_init_fields). */
int olb_batch_init_fields(olb_batch *b, int run, const double *n, const double *ux,
                          const double *uy, const double *T);

/* Advance every run by nsteps RK-3 steps (each with its own dt).  olb_batch_step
 * synchronises and returns OLB_ERR_DIVERGED if any run diverged;
 * olb_batch_step_async only enqueues.  All runs must be initialised. */
int olb_batch_step(olb_batch *b, int nsteps);
int olb_batch_step_async(olb_batch *b, int nsteps);

/* Synchronise; per_run[r] (if not NULL) receives OLB_OK or OLB_ERR_DIVERGED
 * per run; returns OLB_ERR_DIVERGED if any run diverged. */
int olb_batch_get_status(olb_batch *b, int *per_run);

/* Moments / populations of one run into host arrays (as olb_moments,
 * olb_get_populations). */
int olb_batch_moments(olb_batch *b, int run, double *n, double *ux, double *uy, double *T);
int olb_batch_get_populations(olb_batch *b, int run, double *f);

/* Stage-kernel shape of the batch (same compiled shapes as olb_set_tile). */
int olb_batch_set_tile(olb_batch *b, int tx, int ty, int kp);
int olb_batch_get_tile(olb_batch *b, int *tx, int *ty, int *kp);

/* Autotuner: times nsteps steps with every compiled shape (on a copy of the
 * state, which is restored), keeps the fastest and reports it; the choice is
 * cached per process for the batch's precision, device and grid list. */
int olb_batch_autotune(olb_batch *b, int nsteps, int *tx, int *ty, int *kp);

/* Mean device time (ms) of one stage launch over nsteps individually
 * launched steps (the runs advance). */
int olb_batch_profile(olb_batch *b, int nsteps, double *ms);

/* ------------------------------------------------------------------------
 * Learned WENO-5 weights.  Not part of the paper: a 5-32-32-3 network (tanh,
 * tanh, softmax) maps the normalised stencil x = (v - mean v)/(max v - min v)
 * of an interface to three convex weights that replace the Jiang-Shu weights
 * of Eq. weno5_omega.  Parameters: OLB_MLP_PARAMS floats, W1 [32][5], b1 [32],
 * W2 [32][32], b2 [32], W3 [3][32], b3 [3] (row-major, concatenated).
 * Training objective: the mean over samples of (sum_q w_q gn_q - tn)^2, where
 * gn_q are the three candidate values of Eq. weno5_flux minus the centre
 * value and tn the target interface value minus the centre value, both
 * divided by max v - min v.  All arrays of these calls are device pointers
 * (FP32, sample-major: x [n][5], gn [n][3], tn [n], w [n][3]); each call
 * runs on `stream` and returns after its work is complete.
 * ------------------------------------------------------------------------ */
#define OLB_MLP_PARAMS 1347

/* Weights w of n normalised stencils x. */
int olb_mlp_forward(const float *theta, const float *x, int n, float *w, void *stream);

/* Mean loss over the n samples into *loss (device float) and its gradient
 * with respect to theta into grad (device, OLB_MLP_PARAMS floats). */
int olb_mlp_grad(const float *theta, const float *x, const float *gn, const float *tn, int n,
                 float *grad, float *loss, void *stream);

/* Train theta in place with Adam (beta 0.9 / 0.999, eps 1e-8, learning rate
 * lr) over `epochs` passes of consecutive minibatches of `batch` samples;
 * loss_history (host, `epochs` floats, or NULL) receives each epoch's mean
 * minibatch loss.  Allocates its optimiser state with cudaMalloc. */
int olb_mlp_train(float *theta, const float *x, const float *gn, const float *tn, int n, int epochs,
                  int batch, float lr, void *stream, float *loss_history);

/* Load the network (host, OLB_MLP_PARAMS floats) into a context created with
 * weno_mode OLB_WENO_LEARNED; olb_step returns OLB_ERR_STATE until this is
 * done.  OLB_ERR_STATE for other contexts, OLB_ERR_ARG for non-finite values. */
int olb_set_weno_mlp(olb_ctx *ctx, const float *theta);

/* Largest grid (nx * ny nodes) olb_step_static accepts. */
#define OLB_STATIC_MAX_NODES 16384

/* Whole FP64 RK-3 steps without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not call
 * cudaMalloc / cudaFree when they step a small grid -- those calls
 * synchronise the whole device and stall every other stream, and some host
 * applications give all device memory to their own pool up front or load
 * the library as a plug-in that may not touch the allocator.
 *
 * f: caller-owned device array of the populations, FP64 [25][ny][nx] in the
 * exchange layout of olb_get_populations, read and overwritten in place with
 * the state after nsteps >= 0 steps.  *p as for olb_create, restricted to:
 * precision OLB_FP64, weno_mode OLB_WENO_JS, side_y OLB_SIDE_PERIODIC,
 * side_x OLB_SIDE_PERIODIC or OLB_SIDE_DIFFUSE, and at most
 * OLB_STATIC_MAX_NODES nodes.  Anything else (larger grids, FP32, learned
 * weights, specular sides) returns OLB_ERR_ARG before any device work;
 * invalid physics returns OLB_ERR_CFL like olb_create.  The work runs on `stream` (a
 * cudaStream_t or NULL) and the call returns after it has completed, with
 * OLB_ERR_DIVERGED if an invalid moment was met, else OLB_OK.
 *
 * The two intermediate RK-3 buffers and the status word live in one
 * file-scope device array of 2 * 25 * OLB_STATIC_MAX_NODES doubles (6.6 MB)
 * that every GPU which loads the library keeps until the process exits.  The
 * first call on a device looks up that array's device address (with the
 * device current).  All calls share the array and it keeps the last call's contents (the status
 * word is cleared by each call): calls that overlap on the GPU -- on two
 * streams, or from two threads -- race and give wrong results. */
int olb_step_static(const olb_params *p, void *stream, double *f, int nsteps);

/* Human-readable name of a status code (static string). */
const char *olb_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* OLB_H */
