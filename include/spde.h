/*
 * spde.h -- C ABI of the GB300 SPDE sampler (sm_103a).
 *
 * The sampler draws Gaussian random fields with Matern covariance
 * (nu = 1/2 in 3-D, i.e. exponential covariance sigma^2 exp(-kappa r)) by
 * solving the reaction-diffusion SPDE (kappa^2 - Laplace) theta = g W
 * (Sec. 4, Eq. SPDE) in mixed RT0 x P0 form (Eq. reac_diff_weak, Eq. linsys)
 * on a uniform hex grid of an embedding box, then L2-projects each sample
 * onto a non-matching tet mesh (Sec. 5.1, Eq. proj_op) and applies the
 * lognormal map exp (workflow figure of Sec. 6).
 *
 * Conventions shared by every entry point
 *   - All functions return an spde_status; no C++ exception crosses the ABI.
 *     On failure spde_last_error() returns a message for the calling thread.
 *   - "device" pointers are CUDA global-memory pointers on the context's
 *     device; "host" pointers are ordinary CPU memory.  The caller keeps
 *     ownership of every buffer it passes.  Memory the library allocates
 *     itself (grids, coupling matrices, solver workspace) is owned by the
 *     context and released by spde_destroy().
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Kernels are enqueued on it.  The sampling calls are
 *     asynchronous on it (they return once the work is enqueued; the
 *     solver's convergence is decided on the device) unless stated
 *     otherwise; their outcome is collected by spde_wait.
 *   - A context serialises calls on itself with an internal mutex; calls that
 *     use the same level's workspace from different streams are ordered on
 *     the device (the later one waits for the earlier one's completion event).
 *
 * Discrete system (scaled form).  Grid: N = nx ny nz cubes of edge h (a cube
 * n^3 from spde_level_add, a box from spde_level_add_box; "n^3" below means N
 * and "i + n (j + n k)" means i + nx (j + ny k) on a box).  The mixed
 * unknowns of one sample are stored as four contiguous N-entry arrays
 * [ux | uy | uz | theta], each indexed c = i + nx (j + ny k) (x fastest).
 * ux[c] is the normal flux through the +x face of cell c (the face between
 * cells i and i+1); the entry with i = nx-1 lies on the box wall and is held
 * at 0 (essential condition u.n = 0, Sec. 4.2); likewise uy (j = ny-1) and
 * uz (k = nz-1).  With D = diag(h^{-3/2} on fluxes, h^{-1/2} on cells) the
 * library solves the symmetrically scaled system  (D A D) (D^{-1} U) = D F,
 * where A = [[M, B^T], [B, -kappa^2 W]] (Eq. linsys_blocks):
 *     y_u   = T u + D1^T theta,   T = tridiag(1/6, 2/3, 1/6) along each
 *             flux line, (D1^T theta)_f = theta_left - theta_right,
 *     y_th  = D1 u - (kappa h)^2 theta,  (D1 u)_c = sum_axes (u_+ - u_-).
 * Physical cell values are theta = h^{-1/2} (scaled theta).
 */
#ifndef SPDE_H
#define SPDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPDE_OK = 0,
    SPDE_EINVAL = 1,   /* invalid argument (sizes, NaN/inf, bad level, ...) */
    SPDE_ENOMEM = 2,   /* device allocation failed or footprint over budget */
    SPDE_EMESH = 3,    /* mesh rejected (inverted/degenerate tet, tet outside the box,
                          coupling row sum != tet volume); spde_last_error names the tet */
    SPDE_ENOCONV = 4,  /* iteration cap reached before the tolerance; outputs hold
                          the last iterate, spde_get_stats gives the residual */
    SPDE_ETIMEOUT = 5, /* a bounded device wait gave up (a multigrid sweep waited about
                          one second for a plane copy); that solve's outputs are invalid */
    SPDE_ECUDA = 6,    /* a CUDA runtime call failed */
    SPDE_EBUSY = 7,    /* request table full, or grids / meshes changed while requests are in flight */
    SPDE_ECANCELED = 8 /* (spde_poll result) the request was cancelled */
} spde_status;

/* precision of the field solve */
enum {
    SPDE_PREC_MIXED = 0, /* FP32 MINRES + V-cycle inside FP64 iterative refinement, batched */
    SPDE_PREC_FP64 = 1   /* plain path: FP64 MINRES + FP64 V-cycle, one sample at a time */
};

/* inner solver of the refinement */
enum {
    SPDE_SOLVER_MINRES = 0,   /* MINRES on the mixed system, block-diagonal preconditioner (default) */
    SPDE_SOLVER_SCHUR_CG = 1  /* CG on the Schur complement (kappa h)^2 I + D1 T^{-1} D1^T of the cell
                                 unknowns, T^{-1} by exact line solves, same V-cycle preconditioner;
                                 same solution */
};

/* output kinds of spde_sample / spde_project (or-ed with SPDE_OUT_F64) */
enum {
    SPDE_OUT_LOGNORMAL = 0,     /* exp(theta_h) on the tets, [nsamples][ntets] */
    SPDE_OUT_GAUSSIAN = 1,      /* theta_h = W_h^{-1} G theta on the tets, [nsamples][ntets] */
    SPDE_OUT_GRID_GAUSSIAN = 2, /* theta on the embedding grid (physical), [nsamples][n^3] */
    SPDE_OUT_F64 = 16           /* element type double instead of float */
};

typedef struct {
    int precision;      /* SPDE_PREC_MIXED (default) or SPDE_PREC_FP64 */
    double tol;         /* stop when ||F - A x||_2 / ||F||_2 <= tol (scaled system, FP64); 1e-10 */
    double inner_tol;   /* FP32 inner MINRES: stop when a column's preconditioned
                           residual estimate drops by this factor, or by
                           0.1 tol / (the column's current relative residual)
                           when that is larger (a last step that needs less does
                           not over-solve); 1e-5 */
    int max_outer;      /* refinement steps (mixed path); 8 */
    int max_iter;       /* MINRES iterations per solve; 400 */
    double omega;       /* damped-Jacobi weight of the V-cycle smoother; 0.8 */
    double schur_c;     /* weight c of the 7-point Schur approximation kappa^2 h^2 I + c L; 1.0 */
    double flux_diag;   /* flux-block preconditioner, a multiple of the identity; 1.5 = diag(T)^{-1} */
    int check_every;    /* synchronous path: MINRES iterations between host convergence checks;
                           8 (at most 64 are used) */
    int device;         /* CUDA device ordinal; 0 */
    int use_graphs;     /* 1 (default): each refinement solve runs as one captured CUDA graph whose
                           conditional while-nodes run the refinement steps and the MINRES
                           iterations, with every convergence test on the device, so the sampling
                           calls return without synchronising.  0, per-kernel timing on, or the
                           Schur-CG solver: the synchronous path (host loop, convergence read back
                           every check_every iterations).  Both give the same bits. */
    int64_t serve_budget_bytes; /* device memory the serving lanes may hold; 120 GiB */
    int serve_max_batch;        /* columns per serving lane; 64 */
    int solver;                 /* SPDE_SOLVER_MINRES (default) or SPDE_SOLVER_SCHUR_CG */
    int sweep_planes;           /* fine z planes per CTA of the V-cycle sweeps: 8, 16, 32 or 64 (64:
                                   whole-row tiles only; the 32 x 16 tiles take the default) where a
                                   level's z extent allows; 0 (default) = per level, the longest march
                                   that still gives every SM a few CTAs */
    int coarse_fp16;            /* 1: the V-cycle levels held by the one-CTA coarse kernel (at most 4096
                                   cells, 16^3 on a cube) are stored in FP16, each column scaled by its
                                   largest value, arithmetic in FP32 (FP32 path only); 0 (default): FP32 */
    int sweep_rows;             /* 1 (default): the FP32 V-cycle sweeps of levels 32, 64 or 128 cells
                                   wide (constant kappa, or one kappa per column) run on whole-row
                                   tiles; every cell takes the same arithmetic in the same order as
                                   on the 32 x 16 tiles, so the V-cycle gives the same bits (only the
                                   per-CTA partial sums of b.y that MINRES reads are grouped
                                   differently).  0: the 32 x 16 tiles on every level */
} spde_opts;

typedef struct {
    int outer_iters;        /* refinement steps of the last call's solves (max) */
    int inner_iters;        /* MINRES iterations summed over refinement steps (max over solves;
                               the synchronous path counts in steps of check_every) */
    double max_rel_residual;/* max over samples of the final ||F - A x|| / ||F|| (FP64) */
    double setup_ms;        /* last spde_mesh_attach: clipping + CSR build on the device */
    int64_t nnz;            /* nonzeros of the last attached coupling matrix */
} spde_stats;

/* Schedule of a level's solver (spde_autotune / spde_level_set_tuning). */
typedef struct {
    double omega;        /* damped-Jacobi weight of the V-cycle smoother, in (0, 1) */
    double inner_tol;    /* reduction asked of the FP32 inner solve per refinement step, in (0, 1) */
    double flux_diag;    /* flux-block preconditioner (a multiple of the identity), > 0 */
    int sweep_planes;    /* z planes per CTA of the V-cycle sweeps (0, 8, 16, 32, 64; see spde_opts) */
    double ms_per_call;  /* (spde_autotune) device time of one call with this schedule */
    double default_ms;   /* (spde_autotune) the same with the context's options */
    int evaluated;       /* (spde_autotune) schedules timed */
} spde_tuning;

typedef struct spde_ctx spde_ctx;

/* Fill *opts with the defaults listed above. */
spde_status spde_opts_init(spde_opts* opts);

/* Create a context on opts->device (opts may be NULL for defaults).
 * *ctx receives the handle; release it with spde_destroy. */
spde_status spde_grid_create(spde_ctx** ctx, const spde_opts* opts);

/* Define embedding grid `level` (0 <= level < 16): n^3 cubic cells on the
 * box [lo, hi] (Sec. 4.1, domain embedding; Sec. 6.1, nested grids).
 * n must be a power of two, 4 <= n <= 512 (a grid holds at most 2^29 cells),
 * and hi - lo equal on all three axes (cubic cells).  Replaces an existing
 * level of the same index. */
spde_status spde_level_add(spde_ctx* ctx, int level, int n, const double lo[3], const double hi[3]);

/* Define embedding grid `level` as a box of n[0] x n[1] x n[2] cubic cells on
 * [lo, hi] (Sec. 4.1: the embedding domain is a box around the target mesh,
 * as the 1600 x 2420 x 240 ft box of Sec. 7.2).  Every n[a] is a power of two
 * in [4, 1024], n[0] n[1] n[2] <= 2^29, and (hi - lo)[a] / n[a] is the same spacing h on all axes
 * (relative difference <= 1e-12).  The multigrid hierarchy halves every
 * extent above 1; the first level whose extents are not multiples of
 * 32 x 16 x 8 must have at most 4096 cells (e.g. 256 x 256 x 32 is accepted,
 * 512 x 512 x 16 is not).  Cell (i, j, k) has index i + n[0] (j + n[1] k).
 * Otherwise as spde_level_add (SPDE_EINVAL for bad arguments; the Schur-CG
 * solver option needs cubic grids and returns SPDE_EINVAL on a box). */
spde_status spde_level_add_box(spde_ctx* ctx, int level, const int n[3], const double lo[3], const double hi[3]);

/* Attach the target tet mesh of `level` and build its L2-projection operator
 * on the device (Sec. 5.1-5.2): G[tau][c] = |tau cap c| by exact FP64
 * clipping, Pi = W_h^{-1} G stored as CSR (rows = tets).
 *   xyz  host, [nverts][3] double vertex coordinates
 *   tets host, [ntets][4] int32 vertex ids (either orientation; fixed on copy)
 * Both arrays are copied; the caller keeps them.  Every tet must lie inside
 * the box and have volume > 1e-9 h^3; every coupling row must sum to the
 * tet volume within 1e-10 |tau| + 1e-12 h^3 (slivers included: the pieces'
 * rounding is at the scale of the cell) -- else SPDE_EMESH naming the first
 * bad tet.  Synchronises the default stream of the context. */
spde_status spde_mesh_attach(spde_ctx* ctx, int level, int64_t nverts, const double* xyz,
                             int64_t ntets, const int32_t* tets);

/* Draw `nsamples` fields on `level` (Fig. workflow of Sec. 6; Sec. 4.2 noise,
 * Eq. linsys solve, Eq. proj_op projection, exp).  Sample i uses the Philox
 * sample index first_sample + i under key `seed`, so results depend only on
 * (seed, sample index, level grid, mesh, kappa, sigma).
 *   kappa > 0, sigma > 0 finite; nu is fixed at 1/2.
 *   out   device (or host) buffer of the layout `out_kind` states; host
 *         memory is detected and filled before the call returns: pinned host
 *         memory of this device is written by the output kernels directly (it
 *         is mapped into the device's address space), other host memory
 *         through an internal device buffer and one copy.
 * Asynchronous on `stream` (opts.use_graphs = 1 and no per-kernel timing):
 * the call enqueues noise, one graph launch per batch (refinement and MINRES
 * run on the device) and the projection, and returns; `out` is valid once
 * `stream` has synchronised.  Argument errors are returned at once; the
 * solver's outcome (SPDE_ENOCONV: tolerance not reached, `out` holds the
 * last iterate; SPDE_ETIMEOUT) is returned by spde_wait.  With a host `out`
 * the call returns once `out` holds the result, with that outcome.  The first call for a
 * (level, batch size, kappa) captures the graph (a few ms).  On the
 * synchronous path the call synchronises `stream` and returns the outcome
 * itself. */
spde_status spde_sample(spde_ctx* ctx, int level, int nsamples, double kappa, double sigma,
                        uint64_t seed, uint64_t first_sample, int out_kind, void* out, void* stream);

/* Spatially varying kappa(x) and sigma(x) on `level` (Sec. 1: the sampler,
 * unlike circulant embedding, admits correlation lengths and marginal
 * variances that vary in space).  The values are constant per cell of the
 * level's embedding grid: host arrays of n^3 doubles, x fastest
 * (i + n (j + n k)), every kappa and sigma finite and > 0 (else SPDE_EINVAL
 * naming the cell).  The reaction block becomes diag(kappa_c^2) W and the
 * noise of cell c is scaled by g_c = sigma_c sqrt(8 pi kappa_c) (the nu = 1/2,
 * d = 3 normaliser of Sec. 4 evaluated cell by cell).  The arrays are copied
 * to the device (3 n^3 words); two null pointers clear the fields; the level
 * keeps them until then or until spde_level_add redefines it.  SPDE_EBUSY
 * while serving requests are in flight. */
spde_status spde_level_set_fields(spde_ctx* ctx, int level, const double* kappa_cells,
                                  const double* sigma_cells);

/* spde_sample with the fields of spde_level_set_fields in place of one kappa
 * and sigma.  The mixed operator and the FP64 residual take kappa_c per
 * cell; the multigrid preconditioner takes per-cell diagonals on every
 * level (the children's mean of (kappa_c h)^2 on coarse levels), so the
 * field is exact to the tolerance and only the iteration count depends on
 * how strongly kappa varies.  Asynchronous as spde_sample.  MINRES solver
 * only (SPDE_EINVAL with SPDE_SOLVER_SCHUR_CG); SPDE_EINVAL when the level
 * has no fields. */
spde_status spde_sample_fields(spde_ctx* ctx, int level, int nsamples, uint64_t seed,
                               uint64_t first_sample, int out_kind, void* out, void* stream);

/* Coupled two-level samples (Sec. 6.2, multilevel sampler): the white noise
 * is drawn once on the fine level and restricted to the coarse one by
 * summing the 8 children of every coarse cell (the restricted noise has
 * exactly the coarse covariance); the coarse level is solved first and the
 * fine solve starts from its piecewise-constant prolongation.  Sample i is
 * Philox sample first_sample + i on the FINE grid, so out_fine equals
 * spde_sample(fine_level, ...) up to the solver tolerance.
 *   coarse_level must have n_c = n_f / 2 on the same box;
 *   out_fine   device [nsamples][fine outputs], out_coarse device
 *   [nsamples][coarse outputs] (layout of out_kind on each level).
 * Asynchronous as spde_sample (outcome by spde_wait). */
spde_status spde_sample_coupled(spde_ctx* ctx, int fine_level, int coarse_level, int nsamples, double kappa,
                                double sigma, uint64_t seed, uint64_t first_sample, int out_kind, void* out_fine,
                                void* out_coarse, void* stream);

/* ---- serving (continuous batching) ---------------------------------------
 * Requests for samples from several levels, kappas and sigmas are served
 * concurrently.  Samples of one level run as columns of one batch ("lane":
 * its own stream, host thread and workspace), each column with its own kappa
 * and sigma (the operator and the V-cycle take kappa per column); a lane works in
 * refinement steps and, at every step boundary, retires converged columns
 * into their requests' outputs and admits queued samples into the freed
 * columns.  Lanes are created on demand within opts.serve_budget_bytes and
 * released after 200 ms idle.  Every sample follows exactly the arithmetic of
 * spde_sample, so its result is the same alone or in any mix.
 *
 * Submit one request (non-blocking).  Arguments as spde_sample; `out` must
 * be device memory and stay valid until the request is done; the context's
 * precision must be SPDE_PREC_MIXED.  *request receives its id.  While any
 * request is in flight, spde_level_add / spde_mesh_attach return SPDE_EBUSY. */
spde_status spde_submit(spde_ctx* ctx, int level, int nsamples, double kappa, double sigma, uint64_t seed,
                        uint64_t first_sample, int out_kind, void* out, int64_t* request);

/* Poll a request: *done = 1 once all its samples are written (then *result
 * holds its status -- SPDE_OK, SPDE_ENOCONV, SPDE_ECANCELED or a failure --
 * and the request is forgotten), else 0.  *latency_ms: submit-to-completion
 * time once done, else the time waited so far.  latency_ms and result may be
 * NULL.  Unknown ids give SPDE_EINVAL. */
spde_status spde_poll(spde_ctx* ctx, int64_t request, int* done, double* latency_ms, int* result);

/* Cancel a request: samples not yet started are dropped, running ones are
 * discarded at the next step boundary; spde_poll then reports SPDE_ECANCELED.
 * The output buffer may hold partial results. */
spde_status spde_cancel(spde_ctx* ctx, int64_t request);

/* Bytes of device memory spde_sample(level, nsamples) needs beyond what the
 * level already holds (workspace of the selected precision path). */
spde_status spde_query_footprint(spde_ctx* ctx, int level, int nsamples, int64_t* bytes);

/* Statistics of the last call / mesh attach on this context (waits for the
 * context's enqueued calls; after asynchronous calls not yet collected by
 * spde_wait, the maxima over those calls). */
spde_status spde_get_stats(spde_ctx* ctx, spde_stats* stats);

/* Wait until every call enqueued on this context has finished and return the
 * worst outcome of the asynchronous calls since the previous spde_wait:
 * SPDE_OK, SPDE_ENOCONV (some solve stopped above the tolerance: its output
 * holds the last iterate, spde_get_stats the residual) or SPDE_ETIMEOUT (a
 * multigrid sweep gave up waiting for a plane copy: those outputs are
 * invalid).  No paper counterpart: the collection point of the asynchronous
 * calls. */
spde_status spde_wait(spde_ctx* ctx);

/* Size of the coupling matrix of `level`. */
spde_status spde_mesh_info(spde_ctx* ctx, int level, int64_t* ntets, int64_t* nnz);

/* Copy the coupling matrix G of `level` to host arrays (CSR, rows = tets):
 * row_ptr [ntets+1], col [nnz] (cell index), gval [nnz] (|tau cap c|, FP64),
 * vol [ntets] (|tau|).  Any pointer may be NULL to skip it. */
spde_status spde_mesh_copy_csr(spde_ctx* ctx, int level, int64_t* row_ptr, int32_t* col,
                               double* gval, double* vol);

/* Per-kernel timing of this context (CUDA events recorded around every
 * launch on the launching stream; the device time between them is that
 * launch's duration).  enable != 0 clears the counters and starts
 * recording, 0 stops.  Recording adds two event records per launch and no
 * synchronisation. */
spde_status spde_profile_enable(spde_ctx* ctx, int enable);

/* Counters of kernel class k (0 <= k < 18, in launch order of the path:
 * noise, sumsq, residual64, minres_A, alpha, minres_B, mg_down, mg_coarse,
 * mg_up, givens, minres_D, add_correction, transpose_theta, project_exp,
 * flux_from_theta, schur_apply, cg_update, other (reductions, column flags,
 * solver start)):
 * *name its name, *launches its launches, *ms their summed device time,
 * *bytes their summed algorithmic bytes (each launch's inputs read once and
 * outputs written once, for the columns active when it was enqueued).
 * Any output pointer may be NULL. */
spde_status spde_profile_read(spde_ctx* ctx, int k, const char** name, int64_t* launches, double* ms,
                              double* bytes);

/* Autotuner (no paper counterpart; the sampler's own schedule choice).  Times
 * whole spde_sample calls of `nsamples` columns on `level` (kappa, sigma;
 * grid output, a fixed seed, one warm-up and one timed call per candidate)
 * and searches, one knob at a time and twice over, the V-cycle smoother
 * weight omega in {0.7, 0.8, 0.9}, the inner reduction in {1e-4, 1e-5,
 * 1e-6}, the flux-block diagonal in {1.25, 1.5, 2} and the sweep planes per
 * CTA in {0, 8, 16, 32}; a candidate replaces the current choice only when
 * it is at least 1 % faster and the call reaches the tolerance.  The best
 * schedule is kept on the level (every later call on it, serving included,
 * runs with it) and returned in *best.  Synchronises the device; allocates a
 * temporary output buffer of nsamples x cells floats. */
spde_status spde_autotune(spde_ctx* ctx, int level, int nsamples, double kappa, double sigma, spde_tuning* best);

/* Set the schedule of `level` (e.g. an entry of a stored tuning table; only
 * omega, inner_tol, flux_diag and sweep_planes are read), or return it to
 * the context's options with tuning = NULL.  Waits for calls still using the
 * level; SPDE_EBUSY while serving requests are in flight. */
spde_status spde_level_set_tuning(spde_ctx* ctx, int level, const spde_tuning* tuning);

/* Message of the last failed call on this thread ("" if none). */
const char* spde_last_error(void);

/* Free every device and host resource of the context. */
spde_status spde_destroy(spde_ctx* ctx);

/* ---------------------------------------------------------------------
 * Step-level entry points: one step of the path each, on device buffers,
 * so every step can be checked on its own.  `opts` may be NULL.
 * ------------------------------------------------------------------- */

/* White noise (Sec. 4.2: f = W^{1/2} xi, xi ~ N(0, I)).  Writes
 * out[s][c] = scale * xi_c of sample first_sample + s, s < nsamples,
 * c < ncells (device, double, contiguous [nsamples][ncells]).
 * xi from Philox4x32-10: key = (seed mod 2^32, seed >> 32), counter =
 * (p, 0, sample mod 2^32, sample >> 32) for the cell pair (2p, 2p+1);
 * 53-bit uniforms u1 = ((w0:w1 >> 11) + 1) 2^-53, u2 = (w2:w3 >> 11) 2^-53;
 * Box-Muller xi_2p = r cos(2 pi u2), xi_2p+1 = r sin(2 pi u2),
 * r = sqrt(-2 ln u1). */
spde_status spde_noise(int64_t ncells, int nsamples, uint64_t seed, uint64_t first_sample,
                       double scale, double* out, void* stream);

/* Raw Philox4x32-10 words of the noise stream: out[p][0..3] (device, uint32)
 * for counters (p, 0, sample mod 2^32, sample >> 32), p < npairs, key as
 * spde_noise.  The integer stage of spde_noise, exposed for checking. */
spde_status spde_noise_words(int64_t npairs, uint64_t seed, uint64_t sample, uint32_t* out, void* stream);

/* y = (D A D) x, the scaled mixed operator (Eq. linsys_blocks) on an n^3 grid
 * of spacing h, for nsamples stacked vectors of 4 n^3 entries (layout above).
 * prec SPDE_PREC_FP64: x, y are double; SPDE_PREC_MIXED: float.  n is a
 * power of two in [4, 512]; x and y are 16-byte aligned.
 * Wall entries of y are written as 0. */
spde_status spde_apply(int n, double h, double kappa, int nsamples, int prec, const void* x,
                       void* y, void* stream);

/* spde_apply on a box of n[0] x n[1] x n[2] cells (each a power of two in
 * [4, 1024], at most 2^29 cells); every block of a vector has n[0] n[1] n[2] entries, cell
 * (i, j, k) at i + n[0] (j + n[1] k), wall entries at i = n[0]-1 (ux),
 * j = n[1]-1 (uy), k = n[2]-1 (uz). */
spde_status spde_apply_box(const int n[3], double h, double kappa, int nsamples, int prec, const void* x,
                           void* y, void* stream);

/* z = P^{-1} r for the block-diagonal MINRES preconditioner: flux block
 * opts->flux_diag * I, field block one symmetric V-cycle (damped Jacobi,
 * cell-centred linear prolongation, R = P^T, coarse operators
 * 2^l ((kappa h)^2 4^l I + c L_l), exact one-cell solve).  Layout and prec
 * as spde_apply.  Uses library-allocated scratch (allocated on first use per
 * (n, nsamples, prec), kept until process exit). */
spde_status spde_precond(int n, double h, double kappa, int nsamples, int prec,
                         const spde_opts* opts, const void* r, void* z, void* stream);

/* spde_precond on a box grid (layout as spde_apply_box; shape rules as
 * spde_level_add_box).  The level operators are s_l ((kappa h)^2 4^l I +
 * c L_l), where s_l multiplies by (children per coarse cell) / 4 at each
 * coarsening (2^l while all three extents halve). */
spde_status spde_precond_box(const int n[3], double h, double kappa, int nsamples, int prec,
                             const spde_opts* opts, const void* r, void* z, void* stream);

/* spde_precond for callers that cannot allocate device memory: the same
 * preconditioner on the same arguments, with the V-cycle's coarse-level
 * scratch taken from a 16 MiB array compiled into the library instead of
 * cudaMalloc.  (The paper has no counterpart; this serves callers whose
 * device memory belongs to another allocator, such as a framework's caching
 * pool, or whose loop cannot afford the device synchronisation cudaMalloc
 * and cudaFree imply.)  No call allocates or frees device memory.
 *   - Every GPU that loads the library holds the 16 MiB until the process
 *     exits.
 *   - Requests needing more scratch than that are rejected with
 *     SPDE_EINVAL before any work (spde_last_error gives the need): the
 *     need is 2 sum_{l=1..L} (n/2^l)^3 elements per sample over the levels
 *     with n/2^(l-1) >= 32, e.g. about 2.4 MB per sample at n = 128 in FP32.
 *   - n is a power of two in [4, 512], as for spde_precond.
 *   - The first call in a CUDA context looks up the array's device address
 *     (with that device current) and caches it under the context's id; make
 *     that first call before any stream capture.
 *   - A timeout of a V-cycle sweep is reported by spde_precond_status, not by
 *     this call (z's field block is then unspecified); the fault word it uses
 *     is static as well and cleared at the start of every call.
 *   - All calls share the array: calls that overlap on the GPU race.  No
 *     scratch element needs clearing between calls (each call writes every
 *     element it reads). */
spde_status spde_precond_noalloc(int n, double h, double kappa, int nsamples, int prec,
                                 const spde_opts* opts, const void* r, void* z, void* stream);

/* Outcome of the step-level preconditioner calls (spde_precond,
 * spde_precond_box, spde_precond_noalloc) on the current device.  Those calls
 * return once their kernels are enqueued and never report SPDE_ETIMEOUT
 * themselves.  If a V-cycle sweep of a call waits about one second for a
 * plane copy and gives up, that call's z keeps a correct flux block, but
 * its field block is unspecified (tiles skipped, or partly written).  Each
 * call clears its fault word when it starts, so a timeout never makes a
 * later call skip work.  This function synchronises `stream` and returns
 * SPDE_ETIMEOUT when the last spde_precond / spde_precond_box call, or the
 * last spde_precond_noalloc call, timed out (clearing the word), else SPDE_OK.
 * Solves inside a context (spde_sample and the rest) check their own fault
 * word and return SPDE_ETIMEOUT directly. */
spde_status spde_precond_status(void* stream);

/* Self-check of the bounded device waits (no paper counterpart: a safety
 * property of this implementation).  The multigrid sweeps wait on mbarriers
 * for their plane copies; every such wait gives up after about one second,
 * raises the fault word of its solve (one per workspace) and returns, and
 * that solve then reports SPDE_ETIMEOUT.  This call launches one CTA whose
 * barrier never completes, on a stream of its own with a fault word of its
 * own, and checks that path on `device`: SPDE_OK when the wait gave up and
 * its fault word was raised, *waited_ms the time the wait took (about 1000).
 * Solves running meanwhile are not affected; the device stays usable.
 * Synchronises its own stream only. */
spde_status spde_check_wait_limit(int device, double* waited_ms);

/* y = S x with the scaled Schur complement S = (kappa h)^2 I + D1 T^{-1} D1^T of
 * the cell unknowns (Sec. 4.2: kappa^2 W + B M^{-1} B^T, scaled by h^{-1}),
 * T^{-1} applied exactly by tridiagonal line solves.  x, y: device
 * [nsamples][n^3], double (SPDE_PREC_FP64) or float.  Synchronises `stream`. */
spde_status spde_schur_apply(int n, double h, double kappa, int nsamples, int prec, const void* x, void* y,
                             void* stream);

/* Solve the scaled system (D A D) X = [0; rhs] for nsamples right-hand sides
 * with the context's precision path (opts given at spde_grid_create).
 *   rhs  device double [nsamples][n^3] (cell block of the scaled RHS)
 *   x    device double [nsamples][4 n^3] solution (scaled unknowns)
 * Synchronises `stream`; SPDE_ENOCONV as spde_sample. */
spde_status spde_solve(spde_ctx* ctx, int level, int nsamples, double kappa, const double* rhs,
                       double* x, void* stream);

/* Project grid fields onto the tets of `level` (Eq. proj_op) and apply the
 * output map of out_kind (SPDE_OUT_LOGNORMAL or SPDE_OUT_GAUSSIAN, with
 * optional SPDE_OUT_F64).
 *   theta device double [nsamples][n^3] physical cell values
 *   out   device [nsamples][ntets] */
spde_status spde_project(spde_ctx* ctx, int level, int nsamples, const double* theta, int out_kind,
                         void* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPDE_H */
