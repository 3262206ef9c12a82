/*
 * evlbm.h -- C ABI of the GB300 Enskog-Vlasov lattice Boltzmann library.
 *
 * The library advances the explicit lattice Boltzmann model of Karlin &
 * Hosseini, "Practical Kinetic Models for Dense Fluids" (arXiv 2508.00577):
 * one time step is
 *   pull streaming -> raw moments (rho, j, Gamma) -> non-local force F in the
 *   Enskog gauge P0 = P_E -> shifted velocity u and energy E -> EOS (P0,
 *   gamma0) -> gradient corrections (Phi, Phi', q') -> equilibria f^eq, f*,
 *   g^eq, g* -> BGK-type collision,
 * following Eqs. (pre_LBM), (beta), (u_shift), (T_shift), (EVforce1), (Ework),
 * (P0E), (phi), (feq), (f_star), (correction_u), (correction_gamma), (gamma),
 * (geq), (gstar), (g_corr), (correction_q) of the paper.
 *
 * Conventions shared by every entry point
 *   - Lattice units: dt = 1, lattice spacing 1, periodic boundaries.
 *   - Lattice LBM_D2Q9 is the c_z-marginal of the paper's D3Q27 (3-D
 *     thermodynamics, rho E = 3/2 rho RT + 1/2 rho u^2).  A D2Q9 lattice with
 *     nz > 1 is a stack of nz independent 2-D layers.
 *   - Fields are structure-of-arrays with x fastest: node n = x + nx*(y + ny*z),
 *     N = nx*ny*nz.  Vector fields are [D][N] (D = 2 for D2Q9, 3 for D3Q27).
 *     Populations are [Q][N] with i = (cx+1) + 3(cy+1) + 9(cz+1).
 *   - Every function returns LBM_OK (0) or a negative LBM_E* code.  Errors on
 *     a context are described by lbm_last_error(ctx).  Invalid arguments never
 *     reach the GPU.
 *   - The context owns every device buffer it allocates; the caller owns every
 *     pointer it passes in and may free it as soon as the call returns.
 *   - Work is enqueued on the context's stream (the cudaStream_t handle passed
 *     to lbm_init as void*; NULL = the legacy default stream).  Calls that
 *     return host data synchronise that stream.
 */
#ifndef EVLBM_H
#define EVLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)      /* invalid argument */
#define LBM_ECUDA (-2)       /* a CUDA runtime call failed */
#define LBM_ENOMEM (-3)      /* device or host allocation failed */
#define LBM_ENONFINITE (-4)  /* a NaN or Inf was found in the state */
#define LBM_ETIMEOUT (-5)    /* a bounded device-side wait gave up */
#define LBM_EIO (-6)         /* a checkpoint file could not be written or read */

#define LBM_D2Q9 0
#define LBM_D3Q27 1

/* tile_h of lbm_set_tile (D2Q9 FP32) selecting the balanced persistent grid: per
 * strip, as many CTAs as fit on the GPU at once divided by the strip count, each
 * taking an equal share of that strip's row pairs over all layers. */
#define LBM_TILE_BALANCED (-1)

#define LBM_EOS_VDW 0        /* P_E = rho RT / (1 - b rho)  (the paper's form) */
#define LBM_EOS_CS 1         /* Carnahan-Starling contact value, eta = b rho / 4 */

#define LBM_FP64 0           /* FP64 storage and arithmetic (bit-exact reference order) */
#define LBM_FP32 1           /* FP32 storage and arithmetic */
/* 16-bit storage: each population is stored in FP16 or BF16 as its deviation from
 * the local equilibrium (Eqs. feq, geq) of the node that wrote it, scaled by its
 * weight,
 *   (h_i - h_i^eq(R)) / (w_i rho_R)   (g: / (w_i rho_R 3/2 RT_R)),
 * with that node's reference state R = (rho, u, theta0, 3/2 RT) stored beside the
 * populations as an FP32 record of 24 bytes per node; arithmetic is FP32.  D3Q27
 * runs the fused single-pass kernel, D2Q9 the stage kernels. */
#define LBM_FP16_DEV 2       /* FP16 deviation storage */
#define LBM_BF16_DEV 3       /* BF16 deviation storage */

typedef struct lbm_ctx lbm_ctx;

/* Model and lattice parameters.  The paper fixes the lattice (D3Q27), the
 * Enskog pressure P_E = rho RT/(1 - b rho), the Vlasov pressure P_V = -a rho^2
 * with capillarity kappa (Enskog-Vlasov closure, Eqs. EVforce1, Ework), the
 * bare relaxation time tau with beta = dt/(2 tau + dt) (Eq. beta) and the
 * relaxation time lambda of the shifted equilibrium (lambda = dt in the paper). */
typedef struct {
    int lattice;        /* LBM_D2Q9 or LBM_D3Q27 */
    int nx, ny, nz;     /* lattice size, each >= 1; nz = 1 for a single 2-D layer */
    int eos;            /* LBM_EOS_VDW or LBM_EOS_CS */
    double a;           /* Vlasov attraction a >= 0 */
    double b;           /* excluded volume b >= 0 */
    double R;           /* gas constant R > 0 (T in the API, RT inside) */
    double kappa;       /* capillarity coefficient kappa >= 0 */
    double tau;         /* BARE relaxation time tau > 0 (Eq. beta) */
    double lambda;      /* lambda > 0 (1.0 = dt as in the paper) */
    int thermal;        /* 1: f and g double population (energy equation);
                           0: temperature frozen at the initial field, g absent */
    int precision;      /* LBM_FP64, LBM_FP32, LBM_FP16_DEV or LBM_BF16_DEV */
    int force_form;     /* 0: divergence (Korteweg stress) form of F (conserves momentum);
                           1: literal grad(a rho^2) + kappa rho grad(lap rho) */
} lbm_params;

/* Create a context and the initial state from HOST fields (FP64):
 *   rho[N], u[D][N], T[N] (temperature; RT = R T).
 * The populations start at f = f^eq(rho, u, P0/rho) and g = g^eq(rho, u, RT)
 * (Eqs. feq, geq), so the raw momentum is rho u and the first step sees the
 * shifted velocity u + F/(2 rho) (Eq. u_shift).
 * `stream` is a cudaStream_t (or NULL).  The fields are copied to the device as they
 * are (DMA when the host arrays are pinned) and checked and converted there; the call
 * returns after the initial state is built.  On success *out receives the context.
 * Errors: LBM_EINVAL (bad parameters or pointers), LBM_ENOMEM, LBM_ECUDA,
 * LBM_ENONFINITE (non-finite or non-positive rho, non-finite or non-positive T,
 * non-finite u; the message names the lowest such node). */
int lbm_init(const lbm_params *params, const double *rho, const double *u, const double *T,
             void *stream, lbm_ctx **out);

/* Advance the state by n_steps >= 0 time steps (Eq. pre_LBM per step).
 * Asynchronous on the context's stream.  Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_step(lbm_ctx *ctx, int n_steps);

/* Macroscopic fields of the current state, exactly as the next step computes
 * them (streaming, raw moments, force, Eq. u_shift, energy): rho[N], u[D][N],
 * T[N], F[D][N] into HOST arrays (FP64).  Any output may be NULL.  Q~ is zero
 * in the Enskog gauge (Eq. P0E) and is not returned.  Synchronises the stream.
 * Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_moments(lbm_ctx *ctx, double *rho, double *u, double *T, double *F);

/* The same fields as FP32 into DEVICE arrays the caller owns (e.g. torch
 * tensors): d_rho[N], d_u[D][N], d_T[N]; any may be NULL.  Asynchronous on the
 * context's stream.  Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_moments_device(lbm_ctx *ctx, float *d_rho, float *d_u, float *d_T);

/* Restart from macroscopic fields held in DEVICE arrays (FP32): rho[N], u[D][N],
 * T[N].  The populations become the local equilibria f^eq(rho, u, theta0) and
 * (thermal) g^eq(rho, u, theta0, RT) of Eqs. f_eq and g_eq, exactly as lbm_init
 * builds them, and the isothermal temperature field becomes R*T.  Contexts of
 * precision FP32, FP16_DEV or BF16_DEV only (LBM_EINVAL for FP64); the fields
 * are not checked for finiteness.  Asynchronous on the context's stream; the
 * step count is kept.  Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_reset_device(lbm_ctx *ctx, const float *d_rho, const float *d_u, const float *d_T);

/* Copy the current post-collision populations to HOST arrays f[Q][N] and
 * g[Q][N] (g ignored and may be NULL when thermal = 0), converted to FP64
 * (deviation storage is expanded).  Synchronises the stream. */
int lbm_populations(lbm_ctx *ctx, double *f, double *g);

/* Conserved totals of the current state in FP64, reduced on the GPU in a fixed
 * order: out[0] = sum rho, out[1..3] = sum of the raw momentum (x, y, z; z = 0
 * for D2Q9), out[4] = sum of the energy population (0 when thermal = 0).
 * Returns LBM_ENONFINITE if any population is NaN or Inf.  Synchronises. */
int lbm_conserved(lbm_ctx *ctx, double out[5]);

/* Number of time steps taken since lbm_init. */
long long lbm_step_count(const lbm_ctx *ctx);

/* Diagnostic, no counterpart in the paper: the number of out-of-range global or
 * shared-memory indices the fused kernels (D2Q9, D3Q27, batched ensemble) have met
 * since the library was loaded, in a library built with bounds checking
 * (libevlbm_bc.so, compiled with -DEVLBM_BOUNDS_CHECK; such an access is skipped and
 * counted, never performed, and nothing traps).  Returns -1 from a library built
 * without the checks and -2 if reading the device counters failed.  Stands in for a
 * memory checker on machines where none can be run. */
long long lbm_bounds_violations(void);

/* Checkpoint and resume.  The method has no state beyond the post-collision
 * populations of Eq. (pre_LBM) (plus, per storage type, the per-node reference
 * records of 16-bit deviation storage and the frozen R T field when thermal = 0),
 * so a checkpoint holds exactly those device buffers, byte for byte in the
 * context's own storage format, with the step count and every lbm_params field:
 * a resumed run is bit-identical to one that never stopped.
 *
 * lbm_save writes `path` (first to "<path>.tmp", then renamed over `path`, so an
 * interrupted save never leaves a partial file under the final name).  It waits
 * for the work queued on the context's stream.  Layout (little-endian): the
 * 8 bytes "EVLBMCKP", u32 version (2), u32 0, i32 lattice nx ny nz eos thermal
 * precision force_form, f64 a b R kappa tau lambda, i64 step count, u64 byte
 * counts of the four sections (f, g, reference states, frozen R T; 0 when
 * absent), then the sections in that order.  The host is staged through a
 * buffer of at most 64 MiB.
 *
 * lbm_load reads such a file into an existing context created with the same
 * lbm_params (every field must match; the initial fields given to lbm_init do
 * not matter) and restores its step count.  The launch shape (lbm_set_tile) is
 * not part of the state and is kept.
 *
 * Errors: LBM_EINVAL (NULL arguments, not a checkpoint of this library, another
 * version, or parameters or sizes that differ from the context's; the message
 * names the field), LBM_EIO (the file cannot be opened, written or read, or is
 * truncated), LBM_ENOMEM (host staging buffer), LBM_ECUDA.  lbm_load reads the
 * populations into the context's spare buffers and the frozen R T field into host
 * memory, and switches the context over only after every section has been read:
 * after an LBM_EINVAL, LBM_EIO or LBM_ENOMEM the state and step count are those
 * from before the call (it needs host memory for the frozen R T field, 4 or 8
 * bytes per node, when thermal = 0). */
int lbm_save(lbm_ctx *ctx, const char *path);
int lbm_load(lbm_ctx *ctx, const char *path);

/* Number of kernel launches one lbm_step time step enqueues for this context
 * (1 for the fused single-pass kernels: D2Q9 FP32 and D3Q27 FP32, FP16_DEV and
 * BF16_DEV, divergence force form; 4 for the stage-by-stage kernels, 5 with walls);
 * -1 for NULL. */
int lbm_launches_per_step(const lbm_ctx *ctx);

/* Walls, for the thermal Couette flow of the paper's validation (u and T prescribed at
 * x = 0 and x = L_x; the paper does not state its wall scheme).  With enable = 1 the
 * lattice columns x = 0 and x = nx-1 become wall nodes: they do not stream (their moments
 * are those of their own populations), carry no force and do not collide; after every
 * step their populations are the equilibria f^eq(rho_a, u_w, theta0(rho_a, R T_w)) and
 * g^eq(rho_a, u_w, R T_w) of Eqs. feq and geq, with rho_a the density of the fluid node
 * next to them in x at that step and u_w = u_lo (x = 0) or u_hi (x = nx-1).  The channel
 * width between the wall nodes is nx - 1.  The initial fields given to lbm_init should
 * hold u_w and T_w on the wall columns already.  The walls move parallel to themselves
 * (u_x = 0; u_z = 0 on D2Q9).  Requires kappa = 0 (a single-phase fluid: the capillary
 * stress of a wall node would reach through the periodic x boundary), nx >= 3 and FP64 or
 * FP32 storage.  enable = 0 restores periodic x (u_lo, u_hi may then be NULL).
 * Errors: LBM_EINVAL. */
int lbm_set_walls(lbm_ctx *ctx, int enable, const double u_lo[3], const double u_hi[3], double T_w);

/* Launch shape of the fused single-pass kernels.  D3Q27: tile_w = 0 or the kernel's
 * fixed tile width, 32 (tiles of 32 x 8 columns per CTA for FP32 storage, 32 x 16 for
 * FP16/BF16; lbm_get_tile reports the width), and tile_h = the z-chunk a CTA marches
 * through (>= 1).  Above 16 planes the last chunks are shorter: chunks of
 * tile_h while more than 2 tile_h planes remain, then the rest halved down to 8 to 16
 * planes, so that the CTAs that start last (the grid runs in chunk order) end early.
 * D2Q9: strips of
 * tile_w columns (one of 64, 96, 128, 192) marching over chunks of tile_h rows
 * (>= 1; rounded up to an even number, the kernel advances two rows at a time), or
 * tile_h = LBM_TILE_BALANCED: a grid of about one CTA per resident slot of the GPU
 * (SMs x CTAs per SM, rounded down to a multiple of the strip count), each taking an
 * equal share of one strip's row pairs.  lbm_autotune times both kinds.
 * tile_w = tile_h = 0 restores the size-based default.  Contexts without a fused
 * kernel accept and ignore the shape.  Errors: LBM_EINVAL. */
int lbm_set_tile(lbm_ctx *ctx, int tile_w, int tile_h);

/* Current launch shape (0, 0 when the default is in use or no fused kernel applies). */
int lbm_get_tile(const lbm_ctx *ctx, int *tile_w, int *tile_h);

/* Autotuner: times every candidate launch shape of the fused kernel for
 * probe_steps (>= 1) steps each with CUDA events on the context's stream, in two
 * rounds over all candidates, and keeps the shape with the fastest time.  The probes read the current state and write the spare
 * buffer, so the state is unchanged.  Synchronises the stream.  The chosen shape
 * is returned in *tile_w, *tile_h (either may be NULL); both are 0 when the
 * context has no fused kernel.  Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_autotune(lbm_ctx *ctx, int probe_steps, int *tile_w, int *tile_h);

/* Wait for all work queued on the context's stream. */
int lbm_sync(lbm_ctx *ctx);

/* Release the context and its device memory.  NULL is accepted. */
int lbm_free(lbm_ctx *ctx);

/* Message describing the last error on ctx (owned by ctx; "" if none).
 * lbm_last_error(NULL) describes the last failed lbm_init in this thread. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Liquid-vapour coexistence by the Maxwell construction (equal pressure and
 * equal chemical potential of p = P_E - a rho^2, the line of the paper's
 * Fig. 1), solved by Newton iteration in FP64 on the GPU (device 0 of the
 * current context).  eos = LBM_EOS_VDW or LBM_EOS_CS; RT below the critical
 * value.  out[0] = rho_vapour, out[1] = rho_liquid (host).
 * Errors: LBM_EINVAL (RT >= RT_c or bad constants), LBM_ECUDA, LBM_ETIMEOUT
 * (no convergence within the iteration limit). */
int lbm_coexistence(int eos, double a, double b, double RT, double out[2]);

/* Spinodal densities of p = P_E - a rho^2 at RT below the critical value: the two
 * densities where dp/drho = 0 (the limits of the van der Waals loop of the line of
 * the paper's Fig. 1), by bisection in FP64 on the host.  out[0] < out[1] (host).
 * Errors: LBM_EINVAL (NULL out, bad constants, RT <= 0 or RT >= RT_c). */
int lbm_spinodal(int eos, double a, double b, double RT, double out[2]);

/* Planar liquid-vapour interface of the model's square-gradient free energy (the
 * capillary term kappa of Eq. EVforce1): kappa/2 (d rho/dx)^2 = omega(rho), omega the
 * excess grand-potential density between the coexisting densities of lbm_coexistence
 * (solved on the GPU).  out[0] = 10-90 % width of the density profile, out[1] =
 * surface tension sigma = int kappa |d rho/dx| d rho (host FP64 quadrature).  The
 * width scales as sqrt(kappa): kappa for a target width W is kappa (W / width)^2.
 * Errors: LBM_EINVAL (NULL out, kappa <= 0, or as lbm_coexistence), LBM_ECUDA,
 * LBM_ETIMEOUT. */
int lbm_interface(int eos, double a, double b, double RT, double kappa, double out[2]);

/* One FP64 time step that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory while
 * they run -- for example code executing where cudaMalloc is not allowed, or
 * an application whose device memory is pre-planned by another allocator.  The
 * caller owns every buffer: d_f, d_g (input populations, [Q][N] FP64 on the
 * device), d_RT (the frozen R*T field [N], read only when thermal = 0; d_g and
 * d_g_out are ignored then) and d_f_out, d_g_out (output populations; must not
 * alias the inputs).  The intermediate fields live in a static array inside the
 * library sized for at most 32768 nodes (7.75 MiB, held on every GPU that loads
 * the library until the process exits); larger lattices return LBM_EINVAL.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.  The first call on
 * a device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.  The
 * address is kept for the life of the process: after cudaDeviceReset (which
 * unloads the library's device code) further calls are unsupported unless the
 * library is unloaded and loaded again.  All
 * calls share the one array, so calls whose kernels overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.  The
 * populations are bit-identical to lbm_step on an LBM_FP64 context.
 * params->precision must be LBM_FP64.  Asynchronous on `stream`.
 * Errors: LBM_EINVAL (bad parameters, NULL buffers, too many nodes), LBM_ECUDA. */
int lbm_step_noalloc(const lbm_params *params, const double *d_f, const double *d_g, const double *d_RT,
                     double *d_f_out, double *d_g_out, void *stream);

/* ------------------------------------------------------------------------
 * Batched ensembles: many independent periodic 2-D domains of uneven sizes
 * (D2Q9, FP32, divergence-form force), advanced together by one persistent
 * kernel per lbm_batch_step call, launched from a captured CUDA graph.  Each
 * domain follows exactly the same step as lbm_step (Eq. pre_LBM etc.); with the
 * same launch shape its populations are bit-identical to a single context's.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

/* Create a batch of n_domains >= 1 domains of nx[d] x ny[d] nodes sharing the
 * physics of `common` (lattice LBM_D2Q9, precision LBM_FP32, force_form 0,
 * nz 1; common->nx/ny are ignored).  HOST fields are concatenated in domain
 * order: rho[sum N_d], T[sum N_d], and u as the domains' [2][N_d] blocks one
 * after the other.  `stream` is a cudaStream_t; NULL makes the batch create and
 * own a non-blocking stream (the legacy default stream cannot be captured).
 * Errors: LBM_EINVAL, LBM_ENONFINITE, LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_init(const lbm_params *common, int n_domains, const int *nx, const int *ny, const double *rho,
                   const double *u, const double *T, void *stream, lbm_batch **out);

/* Advance every domain by n_steps >= 0 steps in one persistent launch (or, when
 * n_steps x work items per step would reach 2^31, in several, each of
 * lbm_batch_launch_steps steps but the last).  Work
 * items (step, domain, tile) are taken in step-major order; an item waits, with
 * a bounded spin, for its domain's previous step.  Synchronises the stream.
 * Errors: LBM_EINVAL, LBM_ECUDA, LBM_ETIMEOUT (a wait gave up; the state is then
 * partially advanced and should be re-initialised, the batch stays usable). */
int lbm_batch_step(lbm_batch *b, int n_steps);

/* Steps one persistent launch of lbm_batch_step takes at most, for a batch with
 * items_per_step work items per step: the largest even count whose items number
 * fewer than 2^31 (the launch's 32-bit work counter), or 1; -1 if items_per_step < 1.
 * Host computation, no device needed. */
int lbm_batch_launch_steps(int items_per_step);

/* Macroscopic fields of one domain (as lbm_moments): rho[N_d], u[2][N_d], T[N_d]
 * (host FP64; any may be NULL).  Synchronises.  Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_batch_moments(lbm_batch *b, int domain, double *rho, double *u, double *T);

/* Launch shape of the work items: strips of tile_w columns (64, 96, 128, 192) and,
 * per domain, rows split into equal chunks of at most tile_h rows (>= 1; each chunk
 * an even number of rows).  LBM_TILE_BALANCED does not apply: the persistent launch
 * already hands out items as CTAs free up.  Errors: LBM_EINVAL. */
int lbm_batch_set_tile(lbm_batch *b, int tile_w, int tile_h);
int lbm_batch_get_tile(const lbm_batch *b, int *tile_w, int *tile_h);

/* Autotuner: times every launch shape (strip widths 64, 96, 128, 192 x chunk heights
 * 32, 64, 128, 256, 512) on one persistent launch of 2 * probe_steps
 * steps from a device copy of the current state (steps overlap inside a launch as
 * in a run), restoring the state before each probe and at the end; keeps the
 * fastest.  The copy takes as much device memory as the populations of one buffer
 * set, for the duration of the call; if it cannot be allocated, each shape is timed
 * on probe_steps single-step launches into the spare buffer instead.  The state is
 * unchanged either way.  Errors: LBM_EINVAL, LBM_ECUDA, LBM_ETIMEOUT. */
int lbm_batch_autotune(lbm_batch *b, int probe_steps, int *tile_w, int *tile_h);

/* Failure detection: polls (>= 1) a step wait may spin before it gives up
 * (default 2^24, about 2 s).  probe_unset_flag = 1 makes every item also wait on
 * a device flag that nothing sets, so that the next lbm_batch_step reports
 * LBM_ETIMEOUT (used to test the error path); 0 turns it off. */
int lbm_batch_set_wait_limit(lbm_batch *b, long long polls, int probe_unset_flag);

/* Total nodes of the batch (-1 for NULL). */
long long lbm_batch_nodes(const lbm_batch *b);

/* Release the batch.  NULL is accepted. */
int lbm_batch_free(lbm_batch *b);

/* Last error message of the batch ("" if none). */
const char *lbm_batch_last_error(const lbm_batch *b);

/* Critical point (rho_c, RT_c) of p = P_E - a rho^2 (host computation). */
int lbm_critical_point(int eos, double a, double b, double out[2]);

#ifdef __cplusplus
}
#endif
#endif /* EVLBM_H */
