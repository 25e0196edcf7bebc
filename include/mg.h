/*
 * mg.h -- C ABI of the GB300 multigrid solver for the cell-centred
 * variable-coefficient Poisson equation
 *
 *        div(beta grad phi) = f        on a box,
 *
 * each wall either Dirichlet (phi given on the wall; 0 unless lifted, see
 * mg_bc_lift) or Neumann (outward flux beta dphi/dn given; 0 unless lifted).
 *
 * This is the linear solve of a MAESTRO time step (paper Sec. 1: the
 * velocity constraint of the low-Mach approximation gives a variable-
 * coefficient Poisson equation to be solved every step; paper Sec. 3: these
 * solves are what limits MAESTRO's scaling).  The paper does not name a
 * discretisation; the library implements:
 *
 *   - cell (i, j, k) of an (nx, ny, nz) box with spacing dx has its centre at
 *     ((i+1/2)dx, (j+1/2)dx, (k+1/2)dx); arrays are C order (nz, ny, nx),
 *     x fastest (the torch shape (nz, ny, nx));
 *   - face coefficients: harmonic mean 2 a b / (a + b) of the two cells' beta;
 *     a face on a Dirichlet wall takes 2 beta of its cell (the wall is dx/2
 *     from the centre), a face on a Neumann wall 0 (no flux);
 *   - (A phi)_c = sum over the 6 faces of beta_face (phi_nbr - phi_c) / dx^2,
 *     phi_nbr = 0 outside the box; A is symmetric negative definite, or
 *     negative semi-definite with the constants as null space when every
 *     wall is Neumann (then f loses its mean and phi is returned with zero
 *     mean: the compatible problem and its zero-mean solution);
 *   - geometric multigrid V(nu1, nu2) cycles, red-black Gauss-Seidel
 *     smoothing (red = (i+j+k) even first), restriction = mean of 8 children,
 *     piecewise-constant prolongation, coarse face = mean of 4 fine faces,
 *     all dimensions halved while all are even and >= 4, coarsest level
 *     (at most MG_MAX_BOTTOM cells) solved exactly with a dense inverse;
 *   - convergence: ||f - A phi||_2 <= tol * ||f||_2 (unweighted discrete L2).
 *
 * Conventions for every call below.
 *   - Pointers to f, phi, beta and gradients are float64, contiguous, C order
 *     (nz, ny, nx) (batched calls: boxes packed back to back).  They may be
 *     device pointers on the context's device or host pointers (pageable or
 *     pinned); host buffers are copied in and out inside the call.  The
 *     caller owns them; the library never frees or retains them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     ordered on it; calls that return a convergence status synchronise it.
 *   - The library owns its hierarchy (allocated in *_create with cudaMalloc)
 *     and frees it in *_destroy.
 *   - Every int-returning call returns an mg_status; mg_last_error() gives a
 *     thread-local message for the last failure.  On MG_ERR_CUDA the CUDA
 *     error is in the message; the context must then be destroyed.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef MG_H
#define MG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;
typedef struct mg_batch mg_batch;

enum mg_status {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,   /* bad size, pointer, option or call order */
    MG_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    MG_ERR_OOM = 3,           /* device allocation failed */
    MG_ERR_NOT_CONVERGED = 4, /* max_cycles reached or the residual stalled; phi = last iterate */
    MG_ERR_DIVERGED = 5,      /* residual grew by more than 1e3 over its start */
    MG_ERR_NONFINITE = 6,     /* NaN/Inf in f, beta or the residual */
    MG_ERR_TIMEOUT = 7,       /* a bounded device wait gave up */
    MG_ERR_UNSUPPORTED = 8    /* shape or option outside what is implemented */
};

/* Boundary conditions: the bc argument of mg_create / mg_batch_create is a
 * mask with bit w set when wall w is Neumann, walls numbered x-, x+, y-, y+,
 * z-, z+ (0..5); a clear bit is a Dirichlet wall.  0 = every wall Dirichlet.
 * Bits 6, 7, 8 make the x, y, z axis periodic instead (its two wall bits
 * must be clear): cells n-1 and 0 of that axis are neighbours across one
 * face (harmonic mean).  Periodic axes are implemented for one box per
 * context (mg_create; not mg_solve_multi, mg_adjoint, mg_project_correct or
 * batches: MG_ERR_UNSUPPORTED); such a context smooths with single-colour
 * passes and fills the periodic guard cells by an exchange before every
 * stencil.  With every axis periodic or Neumann on both walls, A is
 * singular: the solve removes the mean of f and returns the zero-mean phi. */
enum {
    MG_BC_DIRICHLET0 = 0,
    MG_BC_NEUMANN_XLO = 1, MG_BC_NEUMANN_XHI = 2,
    MG_BC_NEUMANN_YLO = 4, MG_BC_NEUMANN_YHI = 8,
    MG_BC_NEUMANN_ZLO = 16, MG_BC_NEUMANN_ZHI = 32,
    MG_BC_NEUMANN_ALL = 63,
    MG_BC_PERIODIC_X = 64, MG_BC_PERIODIC_Y = 128, MG_BC_PERIODIC_Z = 256
};

/* precision of the V-cycles */
enum {
    MG_FP64 = 0,  /* everything in FP64 */
    MG_MIXED = 1  /* FP32 V-cycles inside an FP64 iterative-refinement loop:
                     FP64 residual, solution update and norm; FP32 smoothing,
                     residual, transfers and coarsest solve */
};

#define MG_MAX_BOTTOM 1024   /* most cells allowed on the coarsest level */
#define MG_MAX_HIST 128      /* residual-history entries kept in mg_stats */

typedef struct {
    int precision;    /* MG_FP64 (default) or MG_MIXED */
    int nu1, nu2;     /* pre- and post-smoothing sweeps (default 2, 2; 0..8) */
    int max_cycles;   /* V-cycles (FP64) or refinement steps (mixed); default 100 */
    int use_graph;    /* 1 (default): replay each V-cycle as a captured CUDA graph */
    int smoother;     /* 0 auto (default), 1 single-colour in-place passes,
                         2 fused two-colour out-of-place sweeps (FP32 levels;
                         FP64 levels always use passes: their f, 1/D and D
                         are stored colour-split, each row's red cells
                         before its black ones, so that a pass reads only
                         its own colour of them) */
    int coarse_cells; /* levels of at most this many cells run inside one CTA
                         per box (the coarse end of the V-cycle as a single
                         launch); 0 default (4096 in FP32 V-cycles, 1024 in
                         FP64 ones, whose FP64 rate per SM is low), -1 off */
    int inner_cycles; /* MG_MIXED: FP32 V-cycles per FP64 refinement step.
                         1..8: that many.  0 (default): adaptive, up to 8:
                         the step solves A e = r32 for a scaled copy r32 of
                         the FP64 residual r, and the finest level's
                         restriction after pre-smoothing also gives
                         ||r32 - A e|| of the smoothed iterate; a box leaves
                         the step's cycles there (its e is that iterate)
                         once the update is expected to bring ||r|| to
                         tol ||f|| / 2, or the step has reduced ||r32 - A e||
                         by 1e6, the most asked of FP32 arithmetic.  With
                         nu1 = 0 or
                         full_residual = 1 (no red-only restriction) the
                         default is 2 fixed cycles */
    int full_residual;/* 0 (default): right after a red-black sweep the black
                         cells satisfy their equations, so the restricted
                         residual and the cycle's residual norm are formed
                         from the red cells only; 1: always every cell */
    int tma;          /* 0 (default) or 1: FP32 fused sweeps are fed by the
                         Tensor Memory Accelerator: a producer warp copies
                         each plane's tiles into a shared-memory ring that
                         eleven consumer warps compute from (on levels
                         whose rows and planes hold a whole 72 x 12 copy
                         box, when the driver can encode tensor maps;
                         elsewhere plain loads); -1: every fused sweep
                         reads its operands with plain loads.  Both give
                         bitwise the same result */
    int krylov;       /* 0 (default): the iteration is V-cycles (FP64) or
                         iterative refinement (mixed); 1: conjugate gradients
                         preconditioned by one symmetric V-cycle per iteration
                         (zero start, nu1 red-then-black sweeps going down,
                         nu2 = nu1 black-then-red sweeps coming up), for
                         high-contrast beta.  With MG_MIXED the V-cycle
                         runs in FP32 on r / ||r|| (CG, its vectors and the
                         residual stay FP64).  Independent boxes with
                         Dirichlet or Neumann walls (not every wall
                         Neumann), no periodic axis, not on a coupled level;
                         otherwise mg_create returns UNSUPPORTED.  cycles in
                         mg_stats counts CG iterations; the solve ends at
                         tol, divergence or max_cycles (the rule that stops
                         V-cycles after 5 cycles without a 10% gain does
                         not apply: a CG residual is not monotone). */
    int max_norm;     /* 1: also report rel_resid_max in mg_stats (one more
                         pass over the level after the solve); 0 (default) */
    int wait_limit;   /* bounded device waits (the TMA sweep's tile-copy
                         waits): polls of the barrier before a wait gives
                         up, sets the context's error word and the solve
                         returns MG_ERR_TIMEOUT.  0 (default): 2^22 polls;
                         n > 0: n polls; -1: give up at the first wait
                         (exercises the timeout path; the CTA still drains
                         the copies it issued before it exits) */
    int persistent;   /* 0 (default): one launch per stage and level.
                         2: every level smoothed with single-colour passes
                         runs as two persistent launches per V-cycle, one
                         going down (pre-smoothing, residual, restriction)
                         and one coming up (prolongation, post-smoothing),
                         each CTA walking the tiles of all active boxes of a
                         stage and a bounded grid barrier between stages
                         (a cooperative launch of at most the resident CTA
                         count; a barrier that gives up after wait_limit
                         polls returns MG_ERR_TIMEOUT).  1: only the levels
                         whose largest stage fits in one wave of resident
                         CTAs (the launch-bound ones); larger levels keep
                         per-stage launches.  Levels smoothed with fused
                         FP32 sweeps keep their own launches. */
    int sweep_zc;     /* tile depth of the fused FP32 sweep: planes of z a
                         CTA marches through (its tile is 64 x 8 cells in
                         x, y).  0 (default): chosen by a model that fills
                         whole waves of resident CTAs; n in 1..4096: n */
    int level_ctas;   /* persistent = 1: CTAs per SM of the persistent
                         launches.  0 (default): as many as can be
                         resident; n in 1..64: at most n */
    int fp32_setup;   /* MG_MIXED on independent boxes: 0 (default): the
                         finest level's FP32 weights are its FP64 ones rounded,
                         every coarser level is set up in FP32 only (averages
                         of the finer FP32 weights, 1/D from its own), since
                         the FP64 levels below the finest are never read;
                         1: every level is set up in FP64 and rounded */
    int reserved;
    /* Device memory of the context (its arena, launch descriptors and host
     * staging buffers) comes from dev_alloc(bytes, alloc_user) when set (NULL
     * on failure: MG_ERR_OOM) and goes back through dev_free(ptr,
     * alloc_user), e.g. a framework's caching allocator; NULL: cudaMalloc /
     * cudaFree.  Called on the host, with the context's device current, from
     * mg_create, the first host-buffer solve and mg_destroy (never while a
     * stream is being captured).  Pinned host buffers are not affected. */
    void *(*dev_alloc)(size_t bytes, void *alloc_user);
    void (*dev_free)(void *ptr, void *alloc_user);
    void *alloc_user;
} mg_opts;

typedef struct {
    int cycles;                /* V-cycles (FP64) or refinement steps (mixed) run */
    int status;                /* mg_status of the solve */
    double norm_f;             /* ||f||_2 */
    double rel_resid0;         /* ||f - A phi0|| / ||f|| before the first cycle */
    double rel_resid;          /* ||f - A phi|| / ||f|| at return */
    double hist[MG_MAX_HIST];  /* rel_resid after cycle c (hist[0] = rel_resid0) */
    float t_setup_ms;          /* device time of the last mg_set_beta set-up on its stream */
    float t_solve_ms;          /* wall time of this call */
    double rel_resid_max;      /* max |f - A phi| / max |f| at return (opts.max_norm = 1;
                                  else 0) */
} mg_stats;

/* Fill *opts with the defaults above. */
void mg_default_opts(mg_opts *opts);

/* Create a solver for an n = {nx, ny, nz} box with spacing dx > 0 on the
 * current CUDA device, walls of the mask bc.  Builds the level list and
 * allocates the hierarchy; runs no kernel.  opts may be NULL (defaults).
 * Errors: INVALID_ARG (n < 1, dx <= 0, bc outside 0..511, a periodic axis
 * with a Neumann bit, bad options),
 * UNSUPPORTED (a coarsest level above MG_MAX_BOTTOM cells, e.g. a 33^3 box),
 * OOM, CUDA. */
int mg_create(mg_ctx **out, const int n[3], double dx, int bc, const mg_opts *opts);

/* Set cell beta (nx*ny*nz values, all > 0 and finite).  Computes face
 * coefficients on every level, inverse diagonals and the coarsest-level
 * inverse, and keeps a device copy of beta for mg_adjoint.  Asynchronous.
 * Errors: INVALID_ARG (NULL). Non-positive or non-finite beta is not checked
 * here; it surfaces as MG_ERR_NONFINITE in the next solve. */
int mg_set_beta(mg_ctx *ctx, const double *beta_cell, void *stream);

/* Solve A phi = f.  phi holds the initial guess on entry (zeros for none)
 * and the solution on return.  tol > 0 is the relative residual target.
 * st may be NULL.  With use_graph (default) the whole cycle loop runs on the
 * device and the call synchronises the stream once at the end; otherwise once
 * per cycle.  Host (not device) f and phi are copied in and out inside the
 * call; host inputs are read on the context's own copy stream, concurrently
 * with work already queued on `stream` (a set-up from mg_set_beta), so they
 * must hold their values when the call is made.  Returns OK, NOT_CONVERGED
 * or DIVERGED (phi = last iterate), NONFINITE (phi unspecified), INVALID_ARG
 * (no beta set, NULL, tol <= 0), CUDA.  f = 0 gives phi = 0 and OK. */
int mg_solve(mg_ctx *ctx, const double *f, double *phi, double tol, mg_stats *st,
             void *stream);

/* Flags of the _ex solves. */
#define MG_ZERO_GUESS 1  /* phi is output only: the iteration starts from 0
                            (host phi is then not copied in) */

/* mg_solve / mg_solve_multi (nrhs >= 1) with flags. */
int mg_solve_ex(mg_ctx *ctx, int nrhs, const double *f, double *phi, double tol, int flags,
                mg_stats *st, void *stream);

/* Same as mg_solve for nrhs right-hand sides packed back to back (each
 * nx*ny*nz values) that share beta; st may be NULL or an array of nrhs.
 * Returns the worst status over the right-hand sides. */
int mg_solve_multi(mg_ctx *ctx, int nrhs, const double *f, double *phi, double tol,
                   mg_stats *st, void *stream);

/* Adjoint of mg_solve for a loss L(phi) with dL/dphi = g (nrhs right-hand
 * sides packed as in mg_solve_multi, phi the forward solutions):
 *   dLdf  (written)      = lambda, the solution of A lambda = g (A = A^T);
 *   dLdbeta (ADDED TO)   += sum over right-hand sides and over the 6 faces of
 *       each cell of dL/dbeta_face * d beta_face / d beta_cell, with
 *       dL/dbeta_face = (lambda_n - lambda_c)(phi_n - phi_c)/dx^2 inside and
 *       lambda_c phi_c / dx^2 on Dirichlet walls (0 on Neumann walls),
 *       d beta_face/d beta_c = 2 beta_n^2 / (beta_c + beta_n)^2 inside and 2
 *       on Dirichlet walls.
 * The forward beta must still be the one set.  Returns as mg_solve_multi;
 * UNSUPPORTED when every wall is Neumann (singular A). */
int mg_adjoint(mg_ctx *ctx, int nrhs, const double *phi, const double *g, double *dLdf,
               double *dLdbeta, double tol, mg_stats *st, void *stream);

/* ---- projection steps around the solve: the velocity constraint the
 * solve enforces (paper Sec. 1).  Face velocities in natural C layouts:
 * u (nz, ny, nx+1) on x faces, v (nz, ny+1, nx), w (nz+1, ny, nx); cell
 * arrays (nz, ny, nx).  Device pointers on the context's device; async.
 *   mg_project_rhs:     f = div(u, v, w) - S, div = sum of the face
 *                       differences / dx (S may be NULL for 0);
 *   mg_project_correct: u, v, w -= beta_face * (phi_high - phi_low) / dx on
 *                       every face, phi = 0 outside and the operator's own
 *                       wall faces (2 beta on Dirichlet walls, 0 on Neumann
 *                       walls, whose velocities are left as they are), using
 *                       the beta of the last mg_set_beta; then
 *                       div(u, v, w) = S up to the solve's residual.
 * Errors: INVALID_ARG (NULL, no beta set), CUDA. */
int mg_project_rhs(mg_ctx *ctx, const double *u, const double *v, const double *w,
                   const double *S, double *f, void *stream);
int mg_project_correct(mg_ctx *ctx, const double *phi, double *u, double *v, double *w,
                       void *stream);

/* Non-zero wall values, lifted into the right-hand side:
 *   f_out = f - sum over the walls next to each cell of
 *           2 beta_c g / dx^2   (Dirichlet wall, g = phi on the wall), or
 *           q / dx              (Neumann wall, q = outward flux beta dphi/dn),
 * so that mg_solve(f_out) returns the solution with those wall values.
 * vals packs one value per wall face, walls in the order x-, x+, y-, y+,
 * z-, z+: an x wall is an (nz, ny) array, a y wall (nz, nx), a z wall
 * (ny, nx), C order; 2 (ny nz + nz nx + ny nx) values in all.  Each value is
 * read as Dirichlet or Neumann by the context's wall mask.  Uses the beta of
 * the last mg_set_beta.  f and f_out (may be equal) are (nz, ny, nx).
 * Device pointers on the context's device; async.  With every wall Neumann
 * the problem is compatible when the fluxes balance the integral of f; the
 * solve removes whatever mean is left.  Errors: INVALID_ARG (NULL, no beta
 * set), CUDA. */
int mg_bc_lift(mg_ctx *ctx, const double *vals, const double *f, double *f_out, void *stream);

/* Level list of a context: *nlev levels, dims[3*l .. 3*l+2] = (nx, ny, nz)
 * of level l (dims may be NULL; room for 32 levels). */
int mg_levels(const mg_ctx *ctx, int *nlev, int *dims);

/* How the context smooths level `level` of its V-cycles (FP32 levels in
 * mixed precision, else FP64): *kind = 0 single-colour passes (or the
 * level is in the one-CTA coarse kernel, or is the coarsest), 1 fused
 * sweeps with plain loads, 2 fused sweeps fed by the Tensor Memory
 * Accelerator.  Host only.  INVALID_ARG for a level outside the list. */
int mg_smoother_kind(const mg_ctx *ctx, int level, int *kind);

void mg_destroy(mg_ctx *ctx);

/* ---- many independent boxes (the grids of one MultiFAB level, paper Sec. 2:
 * a level is a union of disjoint rectangular grids whose data are distributed
 * and worked on independently).  Every stage of a V-cycle runs as one launch
 * over the tiles of all boxes still active at that level; a box whose
 * residual meets tol stops being updated.  Box b has dims n[b] and spacing
 * dx[b]; its arrays are packed at element offset off[b] = sum_{c<b} cells(c). */
int mg_batch_create(mg_batch **out, int nbox, const int (*n)[3], const double *dx, int bc,
                    const mg_opts *opts);
int mg_batch_set_beta(mg_batch *b, const double *beta_packed, void *stream);
/* st may be NULL or an array of nbox; returns the worst status over boxes. */
int mg_solve_batched(mg_batch *b, const double *f_packed, double *phi_packed, double tol,
                     mg_stats *st, void *stream);
int mg_solve_batched_ex(mg_batch *b, const double *f_packed, double *phi_packed, double tol,
                        int flags, mg_stats *st, void *stream);
void mg_batch_destroy(mg_batch *b);

/* ---- a coupled level: boxes of one level solved as one domain ----------
 * The union of disjoint boxes (paper Sec. 2: the grids of one MultiFAB
 * level) is one domain: faces between cells of two boxes are interior faces
 * (harmonic mean), faces on the union's boundary are Dirichlet walls.  Box b
 * covers cells lo[b] .. lo[b] + n[b] - 1 of a common index space (spacing
 * dx); its arrays are packed at element offset off[b] = sum_{c<b} cells(c),
 * each (nz, ny, nx) in C order.  Every box's V-cycle level is coupled to its
 * neighbours by ghost-cell exchanges before each smoothing pass and residual;
 * the exchange patterns come from a hash-binned intersection of the boxes
 * (regions at least as large as any box, keyed by a box's lowest corner,
 * search of the own and the 26 neighbouring regions: O(N + N^2/M)) and are
 * computed once at create.  Levels halve while every box's dims and lower
 * corners are even (boxes may end as single cells); the coarsest levels of
 * all boxes are solved together with a dense inverse (at most MG_MAX_BOTTOM
 * cells in all).  Smoothing uses single-colour passes with a global red-black
 * colouring ((i + j + k) of the common index space even = red).
 * Errors: INVALID_ARG (overlapping boxes, n < 1, dx <= 0, bc != 0),
 * UNSUPPORTED (coarsest union above MG_MAX_BOTTOM cells), OOM, CUDA.  The
 * level solve reports one status and one residual history (the union's);
 * st receives it for every box. */
typedef struct mg_level mg_level;
int mg_level_create(mg_level **out, int nbox, const int (*lo)[3], const int (*n)[3], double dx,
                    int bc, const mg_opts *opts);
int mg_level_set_beta(mg_level *lv, const double *beta_packed, void *stream);
int mg_level_solve(mg_level *lv, const double *f_packed, double *phi_packed, double tol,
                   mg_stats *st, void *stream);
int mg_level_solve_ex(mg_level *lv, const double *f_packed, double *phi_packed, double tol,
                      int flags, mg_stats *st, void *stream);
int mg_level_levels(const mg_level *lv, int *nlev);
void mg_level_destroy(mg_level *lv);

/* Host-only (no device work): the ghost-exchange records of boxes
 * (lo[b], n[b]) at one level.  *nrec = number of records; out (nullable)
 * receives min(*nrec, cap) records of 11 ints: dst box, src box, the patch
 * origin in dst's local coordinates (a guard position: -1 or n on the face
 * axis), the same cells in src's local coordinates, and the extents
 * (ex, ey, ez).  brute != 0 tests all pairs instead of the region bins (for
 * checking).  INVALID_ARG if two boxes overlap. */
int mg_level_intersections(int nbox, const int (*lo)[3], const int (*n)[3], int brute,
                           int *nrec, int *out, int cap);

/* ---- one box split in z into slabs, one GPU per slab ----------------------
 * The paper's codes distribute a level's grids over MPI ranks and fill their
 * ghost cells from the neighbouring grids before each stencil (paper Sec. 2);
 * the linear solves are what limits MAESTRO's scaling (Sec. 3).  This is the
 * same for one large box over several GPUs.  Slab r holds planes
 * z0[r] .. z0[r+1]-1 (equal slabs: nz must be a multiple of nslab) on
 * device devices[r].  Levels are smoothed slab by slab, each slab pulling its
 * neighbours' boundary planes of phi into its guard planes before every
 * single-colour pass and residual (peer copies into a local halo buffer);
 * the first level with at most 32^3 cells (or where a slab or the box stops
 * halving) is gathered: the slabs' restriction writes into one coarse
 * context on devices[0], which runs the rest of the V-cycle, and their
 * prolongation reads its correction from there (slabs on other devices reach
 * it by peer access, which mg_slab_create enables).  The residual norm is the
 * sum of the slabs' squares, judged on the host once per cycle.  The result
 * is the single-box solution of the same operator (interface faces are
 * harmonic means across the two slabs' cells).  FP64 V-cycles only
 * (opts->precision, krylov and persistent must be 0: MG_ERR_UNSUPPORTED).
 * All arrays are device memory of the slab's device, (nz_r, ny, nx) C order;
 * the calls synchronise before they return (their own streams: the
 * caller's work producing the inputs must be complete when they are made). */
typedef struct mg_slab mg_slab;
/* Host only: the slab plan of an n = {nx, ny, nz} box in nslab slabs: z0
 * (nullable) receives nslab + 1 plane offsets, *gather_level (nullable) the
 * level solved by the coarse context (levels 0 .. gather_level - 1 are
 * smoothed slab by slab).  UNSUPPORTED when nz is not a multiple of nslab or
 * no level can be smoothed slab by slab. */
int mg_slab_plan(const int n[3], int nslab, int *z0, int *gather_level);
/* Host only: the halo copies of slab level `level` (< gather_level): *nrec
 * records of 4 ints into out (nullable; at most cap records): source slab,
 * its plane (local k), destination slab, its guard plane (-1 below, the
 * slab's thickness at that level above). */
int mg_slab_halo(const int n[3], int nslab, int level, int *nrec, int *out, int cap);
int mg_slab_create(mg_slab **out, const int n[3], double dx, int nslab, const int *devices,
                   const mg_opts *opts);
/* beta[r]: slab r's cell beta. */
int mg_slab_set_beta(mg_slab *sl, const double *const *beta);
/* f[r], phi[r]: slab r's right-hand side and solution (initial guess unless
 * flags has MG_ZERO_GUESS); st (nullable) gets the whole box's history. */
int mg_slab_solve(mg_slab *sl, const double *const *f, double *const *phi, double tol, int flags,
                  mg_stats *st);
void mg_slab_destroy(mg_slab *sl);

/* ---- measurement -------------------------------------------------------
 * With profiling on, the solver records CUDA events around each stage class
 * below (as event nodes inside the captured V-cycle graph, so the times are
 * those of the real solve) and accumulates the device time between them.
 * Back-to-back launches of one class (the ν sweeps or the 2ν passes of a
 * smoothing step) share one pair of events, and `launches` counts each of
 * them, so ms / launches is a launch's average time.  `kernels` counts every kernel launched by the context (graph nodes count
 * once per replay).  Profiling takes effect at the next solve. */
enum {
    MG_PROF_SWEEP = 0,     /* finest level: fused red+black sweeps */
    MG_PROF_PASS = 1,      /* finest level: single-colour passes */
    MG_PROF_RESTRICT = 2,  /* finest level: residual + restriction */
    MG_PROF_PROLONG = 3,   /* finest level: prolongation + correction */
    MG_PROF_NORM = 4,      /* finest level: residual norm */
    MG_PROF_COARSE = 5,    /* every coarser level and the coarsest solve */
    MG_PROF_REFINE = 6,    /* mixed precision: FP64 refinement step */
    MG_PROF_KRYLOV = 7,    /* krylov = 1: the CG vector updates and dot products */
    MG_PROF_LEVEL = 8,     /* persistent = 1: the finest level's persistent launches
                              (each a whole level sweep, down or up) */
    MG_PROF_SWEEP_PROLONG = 9, /* finest level: the first post-smoothing fused sweep
                              with the prolongation applied to what it reads */
    MG_PROF_NKIND = 16
};
typedef struct {
    double ms[MG_PROF_NKIND];          /* summed device time per stage class */
    long long launches[MG_PROF_NKIND]; /* timed launches per stage class */
    long long kernels;                 /* kernels launched (all classes) */
    long long cells[MG_PROF_NKIND];    /* cells processed per launch (finest level) */
} mg_profile;
int mg_profile_enable(mg_ctx *ctx, int on);
int mg_profile_read(mg_ctx *ctx, mg_profile *out, int reset);
int mg_batch_profile_enable(mg_batch *b, int on);
int mg_batch_profile_read(mg_batch *b, mg_profile *out, int reset);
int mg_level_profile_enable(mg_level *lv, int on);
int mg_level_profile_read(mg_level *lv, mg_profile *out, int reset);

const char *mg_error_string(int status);
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
