/*
 * shl.h -- C-ABI of libshl, periodic elastic homogenisation of
 * charge-parametrised shells on NVIDIA B300 (sm_103a).
 *
 * Method: arXiv 2511.04025, "Shellular Metamaterial Design via Compact
 * Electric Potential Parametrization".  The path is
 *   charges -> truncated periodic potential F (Sec. 3.1, Eq. charge-field)
 *   -> distance d = |F - c| / |grad F| at voxel centres and a shell of
 *      half-thickness t (Sec. 4.1, Eq. beta)
 *   -> six periodic cell problems K u^(k) = f^(k) on the voxel grid
 *      (Eq. inv-design constraints; hex8 elements, K_e = E_e Khat)
 *   -> C^H_ij = sum_e (chi^i + u^i_e)^T K_e (chi^j + u^j_e)  (Eq. inv-design)
 *   -> dE/dtheta by the chain rule through the smoothed density (Eq. chain).
 *
 * Conventions shared by every entry point
 *   - Grid: r voxels per axis on the unit cell, h = 1/r.  Element and voxel
 *     e = (iz*r + iy)*r + ix has its centre at ((ix+1/2)/r, ...); node
 *     n = (iz*r + iy)*r + ix sits at (ix/r, iy/r, iz/r).  Everything is
 *     periodic.
 *   - Node vectors (displacements, loads) are structure-of-arrays: plane
 *     p = 3*k + i holds component i of load case k, so element [p*N + n],
 *     N = r^3.  A full set is 18 planes (6 load cases x 3 components).
 *   - Voigt order 11, 22, 33, 23, 13, 12 with engineering shear strains;
 *     C_out is 6x6 row-major.
 *   - The cell problems are solved with node 0 pinned (its three DOFs
 *     removed), which fixes the rigid translations; relres reports the
 *     residual of that pinned system.
 *   - Buffers ending in _dev are device pointers (a torch tensor's
 *     data_ptr() is fine); every other pointer is host memory.  The caller
 *     owns all of them; no call keeps a caller pointer after it returns
 *     (serving requests are copied at submit).
 *   - stream: a cudaStream_t passed as void*; NULL means the context's own
 *     stream.  Calls that return results in host memory synchronise that
 *     stream before returning; calls that only write _dev buffers do not.
 *   - Every call returns an shl_status.  On failure shl_last_error() gives a
 *     one-line reason.  Invalid arguments are rejected on the host before any
 *     device work.
 */
#ifndef SHL_H
#define SHL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SHL_OK = 0,
    SHL_EINVAL = 1,    /* bad argument; nothing was launched                     */
    SHL_ENOMEM = 2,    /* device workspace or admission budget exhausted         */
    SHL_ENOCONV = 3,   /* max_iter reached; results and residuals still written  */
    SHL_ENUMERIC = 4,  /* NaN/Inf met in a reduction                             */
    SHL_ECUDA = 5,     /* a CUDA runtime call failed                             */
    SHL_EAGAIN = 6,    /* serving: request not finished yet                      */
    SHL_ENOTFOUND = 7  /* serving: unknown ticket                                */
} shl_status;

typedef enum { SHL_FP64 = 0, SHL_FP32_REFINE = 1 } shl_precision;
typedef enum { SHL_MASK = 0, SHL_SMOOTH = 1 } shl_density;
typedef enum { SHL_PRECOND_JACOBI = 0, SHL_PRECOND_MG = 1 } shl_precond;

typedef struct shl_ctx shl_ctx;

/* Context options.  device: CUDA ordinal.  max_batch: serving slots (designs
 * in flight at once, 0 = 16).  hbm_budget_bytes: cap on device memory the
 * serving scheduler may hold for in-flight designs (0 = 40 % of the device's
 * free memory at creation). */
typedef struct {
    int32_t device;
    int32_t max_batch;
    uint64_t hbm_budget_bytes;
} shl_opts;

/*
 * A charge design theta = {p_m, q_m, alpha_hkl} plus the shell (Sec. 3.1,
 * Eq. charge-field):
 *   F(p) = sum_{h,k,l=0..K} alpha_hkl w_hkl sum_j q_j
 *          cos(2 pi h (x-x_j)) cos(2 pi k (y-y_j)) cos(2 pi l (z-z_j)) / (h^2+k^2+l^2)
 * with w = 1, 1/2, 1/4 for none, one, two zero indices and B_000 = 0.
 *   n      charges; pos n x 3 (any real, used mod 1); q n magnitudes
 *   alpha  (K+1)^3 weights indexed [h][k][l], or NULL for all ones
 *   K      truncation order, 1..7 (the paper uses 3)
 *   iso    iso-level c: the shell is |F - c| <= t |grad F|
 *   t      half-thickness in cell units if > 0; otherwise t is chosen so that
 *          round(vf * r^3) voxels are solid (see shl_voxelize)
 *   vf     target solid fraction in (0, 1) when t <= 0
 */
typedef struct {
    int32_t n;
    int32_t K;
    const double *pos;
    const double *q;
    const double *alpha;
    double iso;
    double t;
    double vf;
} shl_design;

/*
 * Solver options (Eq. inv-design cell problems).
 *   E, nu, E_void  solid modulus, Poisson ratio, ersatz void modulus; the
 *                  element modulus is E_e = E_void + rho_e (E - E_void)
 *   tol            stop each load case at ||f - K u||_2 / ||f||_2 <= tol
 *                  (true FP64 residual of the pinned system)
 *   max_iter       cap on CG iterations per load case, summed over restarts
 *                  (FP64) or refinement steps (FP32_REFINE)
 *   precision      SHL_FP64: PCG entirely in FP64, restarted from the true
 *                  residual until it meets tol.
 *                  SHL_FP32_REFINE: FP32 stiffness apply and vectors with
 *                  FP64-class dot accumulation; the iterate is kept in FP64
 *                  and the FP32 residual is replaced by the true FP64
 *                  residual f - K x ("reliable update") whenever it has
 *                  fallen by inner_tol, until the FP64 residual meets tol.
 *   density        SHL_MASK: binary rho; SHL_SMOOTH: rho = 1/(1+exp(-kappa(t-d)))
 *   kappa          logistic sharpness; <= 0 selects ln(9) * r (two-voxel rise)
 *   inner_tol      FP32_REFINE: residual reduction between reliable updates
 *                  (<= 0 selects 1e-4)
 *   warm_start     use the displacements passed in (shl_solve) or kept for the
 *                  session (serving) as the initial guess
 *   precond        SHL_PRECOND_MG (default): geometric multigrid V-cycle
 *                  (Sec. 4.2: 2x2x2 coarsening, Galerkin coarse operators,
 *                  damped block-Jacobi smoothing, pinned dense solve on the
 *                  coarsest level) in FP32, used when r halves down to a
 *                  coarsest grid of at most 6^3 nodes (in SHL_FP64 mode it
 *                  preconditions FP64 CG: the residual is rounded to FP32 for
 *                  the V-cycle and the correction widened back); otherwise,
 *                  or with SHL_PRECOND_JACOBI, point Jacobi.
 *   mg_nu          smoothing sweeps before and after the coarse correction on
 *                  the fine level and the first coarse level (<= 0: 1)
 *   mg_nu_coarse   the same on the smaller levels (index >= 2, at most 1/64 of
 *                  the fine nodes), whose sweeps are cheap (<= 0: 2 for
 *                  r <= 32, else 3)
 *   mg_gamma       visits of each level >= 2 per visit of the level above: 1
 *                  V-cycle, 2 W-cycle; 0 (default) W-cycle from r = 128 up,
 *                  where those levels cost little next to the fine level
 *   mg_omega       block-Jacobi damping as omega * lambda_max(D^-1 A) per level,
 *                  lambda_max estimated by power iteration at setup (<= 0: 1.6);
 *                  if the preconditioned CG still breaks down, the solve is
 *                  repeated with point Jacobi
 *   active         0 (default): every element carries stiffness, void ones the
 *                  ersatz E_void.  1: the active set of Sec. 4.2.1 -- elements
 *                  with rho_e <= cull are culled (no stiffness, no ersatz
 *                  floor), active ones have E_e = rho_e E, nodes with no active
 *                  element drop out of the solve (u = 0 there) and C^H sums the
 *                  active elements.  The result is the E_void -> 0 limit of the
 *                  ersatz problem (first order in E_void).  Floating pieces of
 *                  solid make the system singular but consistent; CG converges
 *                  on it.  Not available in shl_grad (SHL_EINVAL).
 *   cull           density threshold of the active set (<= 0 selects 1e-3)
 */
typedef struct {
    double E, nu, E_void;
    double tol;
    int32_t max_iter;
    int32_t precision;
    int32_t density;
    int32_t warm_start;
    double kappa;
    double inner_tol;
    int32_t precond;
    int32_t mg_nu;
    double mg_omega;
    int32_t active;
    double cull;
    int32_t mg_nu_coarse;
    int32_t mg_gamma;
} shl_solve_opts;

/* Per-result record. */
typedef struct {
    int32_t iters[6];      /* CG iterations per load case (summed over restarts)    */
    double relres[6];      /* final ||f - K u|| / ||f|| per load case, FP64         */
    int32_t n_refine;      /* restarts (FP64) or reliable updates (FP32_REFINE)   */
    int32_t status;        /* shl_status of this result                            */
    double t;              /* half-thickness used                                  */
    double margin;         /* half gap around t when t was chosen from vf          */
    int64_t n_solid;       /* voxels with d <= t                                   */
    int64_t n_ambiguous;   /* voxels with |d - t| <= 1e-9 t                        */
    float ms_field, ms_rhs, ms_solve, ms_chom; /* stage times (CUDA events)        */
    int32_t precond;       /* preconditioner of the returned solve: SHL_PRECOND_MG, or
                              SHL_PRECOND_JACOBI (asked for, grid not coarsenable, or
                              after a multigrid breakdown)                          */
} shl_stats;

int shl_create(const shl_opts *opts, shl_ctx **out);
int shl_destroy(shl_ctx *ctx);
const char *shl_last_error(shl_ctx *ctx);
/* Default solver options: E=1, nu=0.3, E_void=1e-6, tol=1e-10, FP64, mask. */
void shl_default_solve_opts(shl_solve_opts *o);

/*
 * F and grad F at the r^3 voxel centres (Sec. 3.1, Eq. charge-field and its
 * analytic gradient), in FP64.  F_dev: r^3 doubles; gradF_dev: r^3 x 3
 * doubles (x,y,z per voxel) or NULL.  2 <= r <= 1024.
 */
int shl_field(shl_ctx *ctx, const shl_design *d, int32_t r, double *F_dev, double *gradF_dev, void *stream);

/*
 * Voxelise the shell (Sec. 4.1, Eq. beta).  d_e = |F(p_e) - c| / |grad F(p_e)|
 * (+inf where grad F = 0).  If d->t > 0 that t is used; otherwise t is chosen
 * from d->vf: with d_(1) <= ... <= d_(n) sorted, k0 = round(vf n) clamped to
 * [1, n-1], take the k nearest k0 (k0, k0-1, k0+1, ...; within 64 ranks) whose
 * gap d_(k+1) - d_(k) exceeds 1e-9 d_(k+1), and t = (d_(k) + d_(k+1)) / 2.
 *   mask_dev   r^3 bytes, 1 where d_e <= t (may be NULL)
 *   rho_dev    r^3 doubles, the smoothed occupancy beta_e = 1/(1+exp(-kappa(t-d_e)))
 *              (may be NULL); kappa <= 0 selects ln(9) r
 *   d_dev      r^3 doubles receiving d_e (may be NULL)
 *   t_out, margin_out, n_solid, n_ambiguous: host outputs (each may be NULL)
 * Returns SHL_EINVAL when no resolvable gap lies within 64 ranks of k0.
 */
int shl_voxelize(shl_ctx *ctx, const shl_design *d, int32_t r, double kappa, uint8_t *mask_dev, double *rho_dev,
                 double *d_dev, double *t_out, double *margin_out, int64_t *n_solid, int64_t *n_ambiguous,
                 void *stream);

/*
 * q = K p, the assembled periodic stiffness K = sum_e E_e Khat applied
 * matrix-free (Eq. inv-design; Sec. 4.2.2 computes finest-level stiffness on
 * the fly).  nvec load cases (1..6) in the SoA layout above (3*nvec planes).
 *   mask_dev   r^3 bytes: E_e = mask ? E : E_void   (used when rho_dev == NULL)
 *   rho_dev    r^3 doubles: E_e = E_void + rho (E - E_void)
 *   precision  SHL_FP64: p_dev, q_dev are double; SHL_FP32_REFINE: float
 */
int shl_apply(shl_ctx *ctx, int32_t r, const uint8_t *mask_dev, const double *rho_dev, double E, double nu,
              double E_void, int32_t precision, int32_t nvec, const void *p_dev, void *q_dev, void *stream);

/*
 * Loads of the six cell problems, f^(k) = - sum_e K_e chi^k (Eq. inv-design),
 * FP64, 18 SoA planes.  Density as in shl_apply.
 */
int shl_rhs(shl_ctx *ctx, int32_t r, const uint8_t *mask_dev, const double *rho_dev, double E, double nu,
            double E_void, double *f_dev, void *stream);

/*
 * C^H_ij = sum_e E_e (chi^i + u^i_e)^T Khat (chi^j + u^j_e), |Y| = 1
 * (Eq. inv-design), FP64 accumulation, from given displacements u_dev
 * (18 SoA planes of doubles).  C_out: 36 host doubles.
 */
int shl_chom(shl_ctx *ctx, int32_t r, const uint8_t *mask_dev, const double *rho_dev, double E, double nu,
             double E_void, const double *u_dev, double *C_out, void *stream);

/*
 * Solve the six periodic cell problems for a given density (node 0 pinned,
 * preconditioned CG on all six load cases at once -- o->precond, multigrid by
 * default -- with per-case convergence and skip) and return C^H.  u_dev (18 SoA planes of doubles, may
 * be NULL) receives the displacements; if o->warm_start it also supplies the
 * initial guess.
 */
int shl_solve(shl_ctx *ctx, int32_t r, const uint8_t *mask_dev, const double *rho_dev, const shl_solve_opts *o,
              double *u_dev, double *C_out, shl_stats *st, void *stream);

/*
 * The whole path for one design: field, voxelisation (t from d->t or d->vf),
 * the six cell problems and C^H.  C_out: 36 host doubles.  st may be NULL.
 * Returns SHL_ENOCONV if a load case did not reach o->tol (C_out and st are
 * still written).
 */
int shl_homogenize(shl_ctx *ctx, const shl_design *d, int32_t r, const shl_solve_opts *o, double *C_out,
                   shl_stats *st, void *stream);

/*
 * Hand-written adjoint (Eq. chain): for an objective E(C^H, V) with dE/dC^H =
 * dE_dC (36 host doubles, row-major) and dE/dV = dE_dV, V = (1/r^3) sum_e
 * rho_e the solid volume fraction of the smoothed density (the objectives of
 * Sec. 5.3 divide stiffness by it), the gradient with respect to the charge
 * positions (g_pos, n x 3), magnitudes (g_q, n), iso-level (g_iso), shell
 * half-thickness (g_t) and spectral weights (g_alpha, (K+1)^3 or NULL),
 * through the smoothed density rho_e = 1/(1+exp(-kappa(t - d_e))) with the
 * ersatz floor E_e = E_void + rho_e (E - E_void).  o->density must be
 * SHL_SMOOTH.  Each cell problem is self-adjoint, so no adjoint solve is
 * needed: dE/drho_e = (E - E_void) sum_ij dE_dC_ij (chi^i+u^i_e)^T Khat
 * (chi^j+u^j_e), then the logistic, the distance proxy d = |F-c|/|grad F| and
 * the field.  When t comes from d->vf it is selected first and then held
 * fixed.  C_out (36) receives C^H.  u_dev (18 SoA planes of doubles, may be
 * NULL) receives the displacements and, with o->warm_start, seeds the solve
 * (pass the forward's u_dev to make a backward pass solve-free).  V_out
 * receives V.  Any output pointer may be NULL; SHL_EINVAL for a non-finite
 * dE_dC or dE_dV.
 */
int shl_grad(shl_ctx *ctx, const shl_design *d, int32_t r, const shl_solve_opts *o, const double *dE_dC,
             double dE_dV, double *u_dev, double *C_out, double *g_pos, double *g_q, double *g_iso, double *g_t,
             double *g_alpha, double *V_out, shl_stats *st, void *stream);

/*
 * n designs, each on its own r[i]^3 grid; C_out: n x 36; st: n records or
 * NULL.  The designs run concurrently on the context's serving slots (up to
 * max_batch at once, admitted by HBM footprint as in shl_serve_submit), each
 * solved exactly as shl_homogenize would solve it alone.  Stream order: every
 * design starts after the work queued on `stream` before the call, and work
 * queued on `stream` after the call starts after every design.  Blocks until
 * all are done.  SHL_EINVAL (nothing launched) if any design or the options
 * are invalid or a footprint exceeds the budget; otherwise the first hard
 * error of any design, else SHL_ENOCONV if any load case missed o->tol.
 */
int shl_homogenize_batch(shl_ctx *ctx, int32_t n, const shl_design *d, const int32_t *r, const shl_solve_opts *o,
                         double *C_out, shl_stats *st, void *stream);

/*
 * Serving: continuous batching of homogenisation requests (the paper's
 * interactive edit -> re-evaluate loop, Sec. 5.1, and the batches of designs
 * an optimiser submits, Sec. 4.3).  Requests are copied at submit and queued
 * FIFO; a pool of max_batch worker slots (each with its own stream and
 * workspace) takes the head request as soon as a slot is free and its HBM
 * footprint fits the budget, so requests that arrive while others run are
 * admitted immediately and their kernels overlap on the GPU.  Each slot runs
 * the same path as shl_homogenize, so a result is identical alone and in a
 * mix.  With opts.warm_start and session >= 0, the session's last
 * displacements (kept on the device, same r) seed the solve.
 */
typedef struct {
    shl_design design;    /* copied at submit */
    int32_t r;
    shl_solve_opts opts;
    int64_t session;      /* warm-start key, < 0 for none */
} shl_request;

typedef struct {
    double C[36];
    shl_stats stats;
    double t_submit, t_admit, t_done;  /* seconds since the context was created */
    int32_t warm;                      /* 1 if the solve started from a session's displacements */
    int32_t slot;                      /* worker slot that ran it */
} shl_result;

typedef struct {
    int32_t slots, queued, running;
    uint64_t completed;
    uint64_t held_bytes;    /* slot workspaces + warm-start cache */
    uint64_t budget_bytes;
} shl_serve_info;

/* Non-blocking.  SHL_EINVAL (nothing queued) for an invalid request or one
 * whose footprint can never fit the budget. */
int shl_serve_submit(shl_ctx *ctx, const shl_request *req, uint64_t *ticket);
/* SHL_EAGAIN while queued or running; on completion fills out (out->stats.status
 * is the request's own status) and forgets the ticket; SHL_ENOTFOUND otherwise. */
int shl_serve_poll(shl_ctx *ctx, uint64_t ticket, shl_result *out);
/* Blocks until the request completes, then as shl_serve_poll. */
int shl_serve_wait(shl_ctx *ctx, uint64_t ticket, shl_result *out);
/* Removes a queued request (SHL_OK); SHL_EAGAIN if it is already running
 * (it completes normally); SHL_ENOTFOUND for an unknown ticket. */
int shl_serve_cancel(shl_ctx *ctx, uint64_t ticket);
/* Blocks until nothing is queued or running. */
int shl_serve_drain(shl_ctx *ctx);
int shl_serve_info_get(shl_ctx *ctx, shl_serve_info *out);

/* Telemetry of a context since creation: kernels launched by the library and
 * device workspace bytes currently held.  No device work. */
typedef struct {
    uint64_t kernel_launches;
    uint64_t workspace_bytes;
} shl_counters;
int shl_get_counters(shl_ctx *ctx, shl_counters *out);

/* Arithmetic peaks of the context's device, measured by short FMA-throughput
 * kernels (independent FMA chains in every thread of 4 CTAs per SM): scalar
 * FP32, packed FP32 pairs and FP64, in GFLOP/s (an FMA counts 2 flop, a packed
 * FMA 4).  The ceilings beside the copy rate for kernels bound by CUDA-core
 * arithmetic (the FP64 field evaluation of Sec. 3.1, the FP32 stiffness
 * apply).  Synchronises the context's stream; takes a few milliseconds. */
typedef struct {
    double fp32_fma_gflops;
    double fp32x2_fma_gflops;
    double fp64_fma_gflops;
} shl_peaks;
int shl_probe_peaks(shl_ctx *ctx, shl_peaks *out);

/* Failure-detection probe of the bounded device waits (no paper
 * counterpart): one CTA waits on an mbarrier that nothing completes, for at
 * most `polls` polls of the same bounded wait the stiffness apply uses on its
 * copies, then records the timeout in an error word exactly as the apply does.
 * *timed_out = 1 when the wait ended by its bound (expected), 0 otherwise.
 * The kernel returns normally, so the context stays usable.  polls in
 * [1, 2^20]; synchronises the context's stream.  SHL_EINVAL on bad arguments. */
int shl_probe_wait_timeout(shl_ctx *ctx, uint32_t polls, int32_t *timed_out);

/*
 * Allocation-free variant of shl_chom (the paper has no counterpart; this is
 * an interface for callers that cannot allocate device memory, e.g. code
 * running inside another framework's memory pool or a latency-critical loop
 * where cudaMalloc may stall or is not permitted).  Computes the same C^H as
 * shl_chom, but writes the 36 doubles to the device buffer C_dev (row-major)
 * and needs no context: the reduction's scratch is a fixed 256 KiB array
 * inside the library that every GPU loading the library holds until exit.
 * It calls no cudaMalloc/cudaFree.
 *   - runs on the calling thread's current device, on stream (NULL = legacy
 *     default stream); returns without synchronising; u_dev, C_dev and the
 *     density must be device memory of that device (SHL_EINVAL otherwise);
 *   - 1 <= r <= 512; larger grids are rejected with SHL_EINVAL;
 *   - the first call on each device looks up the scratch address
 *     (cudaGetSymbolAddress); make that first call before any stream capture;
 *   - the scratch array belongs to the device's primary context (the one the
 *     CUDA runtime uses); the looked-up address is kept for the life of the
 *     process, so do not call this entry point after cudaDeviceReset or from
 *     a context created with the driver API;
 *   - all calls share the one scratch array (it keeps the last call's
 *     contents; the call clears what must start at zero), so calls whose
 *     work overlaps on the GPU (different streams, no ordering) race;
 *   - errors are reported by the return code and shl_last_error(NULL).
 * Density arguments as in shl_apply; u_dev as in shl_chom.
 */
int shl_chom_noalloc(int32_t r, const uint8_t *mask_dev, const double *rho_dev, double E, double nu, double E_void,
                     const double *u_dev, double *C_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SHL_H */
