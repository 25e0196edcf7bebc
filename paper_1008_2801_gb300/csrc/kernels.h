// kernels.h -- host launchers of the solver's CUDA kernels (kernels.cu).
#pragma once

#include "common.cuh"

namespace mg {

// Kernels launched by this library so far (all threads, all contexts).
long long launch_counter();

// ---- V-cycle stages over a set of boxes (one CTA per tile) --------------
// `active` (nullable, indexed by Box::box) skips boxes whose flag is 0.

// One red (0) or black (1) Gauss-Seidel pass in place on Box::phi.
template <class T>
cudaError_t launch_rbgs_pass(const BoxSet<T> &S, const int *active, int color, cudaStream_t st);
// One colour out of place (from2: phi2 -> phi, else phi -> phi2); partials
// (FP64, nullable): per TK_PCOLZ tile, the sum of the squared residuals of the
// source at the updated cells (finish with launch_norm_finish mode 2).
template <class T>
cudaError_t launch_rbgs_pass_oop(const BoxSet<T> &S, const int *active, int color, int from2,
                                 double *partials, cudaStream_t st);

// The boxes of S are right-hand sides of one box (same dims, one set of
// weights, 1/D and D): one colour pass in every active box, in place
// (oop = 0) or out of place (oop = 1, from2 as launch_rbgs_pass_oop), each
// cell's weights read once for all of them.  Same arithmetic per cell as
// the per-box passes.
template <class T>
cudaError_t launch_rbgs_pass_multi(const BoxSet<T> &S, const int *active, int color, int oop,
                                   int from2, cudaStream_t st);

// ---- FP32 fused sweep fed by the Tensor Memory Accelerator (sweep_tma.cu)
struct SweepMaps;  // seven tensor maps of one box level (device memory, 128-B aligned)
size_t sweep_maps_size();
// The TMA sweep serves levels whose rows and planes hold a whole copy box.
bool sweep_tma_fits(int nx, int ny);
// The fused prolongation also needs the coarse level to hold its copy box.
bool sweep_tma_prol_fits(int nx, int ny, int cx, int cy);
// Encode the maps from the arrays' allocation bases (logical (0, 0, -1));
// phic_base (or null): the coarse level's phi, cx x cy x cz, for the fused
// prolongation.  False if the driver offers no encoder or a box does not fit.
bool encode_sweep_maps(SweepMaps *out, int nx, int ny, int nz, const float *phi_base,
                       const float *phi2_base, const float *f_base, const float *wx_base,
                       const float *wy_base, const float *wz_base,
                       const float *phic_base = nullptr, int cx = 0, int cy = 0, int cz = 0);
int sweep_tma_ctas_per_sm();
// Same result as launch_rbgs_sweep<float>; *err is set to 1 if a bounded
// wait on a tile copy gave up after wait_polls polls (the CTA then waits,
// with the default bound, for the copies it issued and stops).
// prolong: first apply the level's prolongation phi += e(parent) (the coarse
// correction in each box's phic) to the tiles read, as launch_prolong would
// (maps encoded with the coarse level's phi).
cudaError_t launch_rbgs_sweep_tma(const BoxSet<float> &S, const SweepMaps *maps,
                                  const int *active, int src_is_phi2, int *err, cudaStream_t st,
                                  long long wait_polls, bool prolong = false);
// Polls of a tile-copy wait for mg_opts.wait_limit (0: the default bound;
// -1: none, the first wait gives up).
long long sweep_wait_polls(int wait_limit);

// Resident CTAs per SM of the fused sweep kernel (occupancy query).
template <class T>
int sweep_ctas_per_sm();

// Fused red+black sweep, out of place: Box::phi -> Box::phi2 (src_is_phi2
// swaps the roles).
template <class T>
cudaError_t launch_rbgs_sweep(const BoxSet<T> &S, const int *active, int src_is_phi2,
                              cudaStream_t st);

// fc = mean over 8 children of (f - A phi); phic = 0.
template <class T>
cudaError_t launch_resid_restrict(const BoxSet<T> &S, const int *active, cudaStream_t st);

// Same, right after a red-black sweep: only the 4 red children carry a
// residual (black cells satisfy their equations), half the stencil work.
template <class T>
cudaError_t launch_resid_restrict_red(const BoxSet<T> &S, const int *active, cudaStream_t st,
                                      double *partials = nullptr);
// Adaptive inner cycles (mixed precision): the exit test after a restriction
// with partials; the start of a step's inner cycles (flags copied, counter
// reset, loop condition set) and, in the graph WHILE form, the end of each.
cudaError_t launch_inner_judge(const BoxSet<float> &S, int *active32, const double *partials,
                               const int *cstart, int nchunks, int chunk_tiles, double *chunks,
                               const double *se, const double *sr, const double *normf,
                               const double *tol, double floor_rel, int coupled, cudaStream_t st);
cudaError_t launch_inner_begin(int nbox, const int *src, int *dst, int *count,
                               cudaGraphConditionalHandle handle, int use_handle, cudaStream_t st);
cudaError_t launch_inner_end(int nbox, const int *flags, int *count, int max_cycles,
                             cudaGraphConditionalHandle handle, cudaStream_t st);

// phi += phic[parent].
template <class T>
cudaError_t launch_prolong(const BoxSet<T> &S, const int *active, cudaStream_t st);

// r = f - A phi written to Box::phi2 (used by the single-stage entry point).
template <class T>
cudaError_t launch_residual_field(const BoxSet<T> &S, cudaStream_t st);

// Residual norm of level 0: partial sums, then out[Box::box] (see below).

// Per-tile partial sums of squares: mode 0 = residual f - A phi, mode 1 = f,
// mode 2 = residual at red cells only (right after a red-black sweep).
template <class T>
cudaError_t launch_norm_partials(const BoxSet<T> &S, const int *active, int mode,
                                 double *partials, cudaStream_t st);

// out[Box::box] = sqrt(sum of the box's partials), fixed order; inactive
// boxes keep their old value.  copy and inv (nullable) receive the same value
// and its reciprocal (0 for a zero norm).
// mult (nullable, per box) scales the norm before it is stored; mode is the
// partials' tiling, as in launch_norm_partials (0/1 TK_COLZ, 2 TK_PCOLZ).
template <class T>
cudaError_t launch_norm_finish(const BoxSet<T> &S, const int *active, const double *partials,
                               double *out, double *copy, double *inv, cudaStream_t st,
                               const double *mult = nullptr, int mode = 0);

// Coarsest level: phi = Ainv f (dense, one warp per row).
template <class T>
cudaError_t launch_bottom(const BoxSet<T> &S, const int *active, int max_cells, cudaStream_t st);

// The coarse end of the V-cycle of each job's box in one CTA per job.
// post_first: colour of the first pass of each post-smoothing sweep (0 red,
// the default; 1 black: the post-smoother is the pre-smoother's adjoint).
template <class T>
cudaError_t launch_coarse_vcycle(const CoarseJob<T> *jobs, int njobs, const int *active, int nu1,
                                 int nu2, cudaStream_t st, int post_first = 0);

// Mixed-precision refinement on the finest level of every box (FP64 phi = x,
// f, weights, D in S64; FP32 phi = e, f = r32 in S32):
//   update:   x += c_e[b] e
//   residual: r = f - A x; r32 = r * c_r_inv[b]; partial sums of r32^2
//   (x_zero: x = 0, so r = f, read without the stencil)
cudaError_t launch_refine_update(const BoxSet<double> &S64, const BoxSet<float> &S32,
                                 const int *active, const double *c_e, cudaStream_t st);
cudaError_t launch_refine_residual(const BoxSet<double> &S64, const BoxSet<float> &S32,
                                   const int *active, const double *c_r_inv, double *partials,
                                   cudaStream_t st, bool x_zero = false);

// One convergence decision per active box after a cycle (see k_judge); sets
// the graph condition to "any box still active" when use_handle is 1.
cudaError_t launch_judge(int nbox, const double *norm, const double *normf, int *active,
                         const JudgeState &J, cudaGraphConditionalHandle handle, int use_handle,
                         cudaStream_t st);

// ---- persistent level sweeps (one launch per level and direction) -------
// Bounded grid-wide barrier of a persistent launch: `word` (device, zero when
// a solve starts) is shared by every barrier of the solve; a CTA that polls
// it `polls` times without seeing it complete sets *err to 1 and returns.
struct GridSync {
    unsigned *word;
    int *err;
    long long polls;
};
// What one level's persistent launch does.  Down (k_level_down): nu sweeps
// of single-colour passes (red, black), then the residual and restriction.
// Up (k_level_up): prolongation, then nu sweeps.  A grid barrier separates
// consecutive stages.
struct LevelOps {
    int nu;              // sweeps (each a red and a black pass)
    int head_done;       // down, finest level after the look-ahead red pass (phi -> phi2): the
                         // first sweep ends with the black pass phi2 -> phi
    int red;             // down: restrict the residual of the red children only
    int reverse;         // up: black before red in each sweep (symmetric cycle)
    const ExchRec *rec;  // ghost exchange before every pass and the residual (nrec = 0: none)
    int nrec, chunks;    // records, and CTAs' worth of work per record
    int flat;            // the set tiles TK_COARSE flat (its flat bit)
    double *partials;    // down, red restriction: per-tile sums of squared residuals (or null)
};
// Resident CTAs per SM of the persistent level kernels (occupancy query).
template <class T>
int level_ctas_per_sm();
// One cooperative launch of `grid` CTAs (at most level_ctas_per_sm x SMs).
template <class T>
cudaError_t launch_level(const BoxSet<T> &S, const int *active, int up, const LevelOps &op,
                         const GridSync &g, int grid, cudaStream_t st);

// ---- coarsest level too large for a dense inverse: conjugate gradients ----
// One cooperative launch over box 0 of S (its coarsest level): diagonally
// preconditioned CG on -A from x = 0 into phi (r in phi2; p, q level arrays
// of that level with zero guards; part: 2 x grid doubles of scratch), until
// <r, D^-1 r> falls by tol^2 or maxit iterations; stages separated by the
// bounded grid barrier g.
template <class T>
int cg_bottom_ctas_per_sm();
template <class T>
cudaError_t launch_cg_bottom(const BoxSet<T> &S, const int *active, T *p, T *q, double *part,
                             const GridSync &g, int grid, double tol, int maxit, cudaStream_t st);

// ---- moving data between packed user arrays and the level layout --------
// user[off[b] + (k*ny + j)*nx + i] -> level 0 f (to_f) or phi of box b.
// partials (f only): also the TK_COLZ partial sums of f^2 that
// launch_norm_partials(S, NULL, 1, partials) would write, bit for bit.
cudaError_t launch_pack(const BoxSet<double> &S, const long long *off, const double *user,
                        int to_f, cudaStream_t st, double *partials = nullptr);
// level 0 phi (side[b] == 0, or side == NULL) or phi2 (side[b] == 1) -> user.
cudaError_t launch_unpack(const BoxSet<double> &S, const long long *off, double *user,
                          const int *side, cudaStream_t st);
// phi = 0 inside the box (active boxes only).
template <class T>
cudaError_t launch_zero(const BoxSet<T> &S, const int *active, cudaStream_t st);
// Mixed-precision scales per box: init -> se = 0, sr = normf, sr_inv = 1/normf;
// otherwise (active boxes) se = sr, sr = norm, sr_inv = 1/norm.
cudaError_t launch_scales(int nbox, const int *active, int init, const double *norm,
                          const double *normf, double *se, double *sr, double *sr_inv,
                          cudaStream_t st);

// ---- set-up (one box per launch) -----------------------------------------
// bcm: bit w set = wall w (x-, x+, y-, y+, z-, z+) is Neumann (weight 0).
cudaError_t launch_face_weights(int nx, int ny, int nz, double inv_h2, int bcm, const double *beta,
                                double *wx, double *wy, double *wz, cudaStream_t st);
cudaError_t launch_coarsen(int nx, int ny, int nz, const double *wx, const double *wy,
                           const double *wz, double *cwx, double *cwy, double *cwz,
                           cudaStream_t st);
// invD = 1 / D and (D nullable) D = sum of the six weights.
cudaError_t launch_inv_diag(int nx, int ny, int nz, const double *wx, const double *wy,
                            const double *wz, double *invD, double *D, cudaStream_t st);
cudaError_t launch_round_f32(int nx, int ny, int nz, const double *wx, const double *wy,
                             const double *wz, const double *invD, float *wx32, float *wy32,
                             float *wz32, float *invD32, cudaStream_t st);
// singular != 0: every wall Neumann; the constants are shifted out.
cudaError_t launch_bottom_inverse(int nx, int ny, int nz, const double *wx, const double *wy,
                                  const double *wz, int singular, double *work, double *inv64,
                                  float *inv32, cudaStream_t st);
// ---- set-up of every box of a level in one launch ------------------------
// step 0: face weights from beta; 1: coarse weights; 2: D and 1/D; 3: FP32
// copies; 4: coupled faces from betaL; 5: faces with their FP32 copies; 6: D
// with the FP32 1/D; 8: FP32 1/D from the FP32 weights; 9: FP32 coarse
// weights from the finer FP32 ones.
cudaError_t launch_setup(const SetupSet &S, int step, cudaStream_t st);
// Tiles [t0, t1) of one step (tiles are numbered plane by plane, so a range
// of whole planes of a one-box set is a range of tiles).
cudaError_t launch_setup_tiles(const SetupSet &S, int step, int t0, int t1, cudaStream_t st);
// The coarsest level's dense inverse, one CTA per box.
// packed_bytes: dynamic shared memory for the packed upper triangles (the
// largest packed_bottom_bytes over the boxes; 0: every matrix in scratch)
cudaError_t launch_setup_bottom(const SetupSet &S, int packed_bytes, cudaStream_t st);
// Bytes of the packed upper triangle of an n-cell coarsest matrix if it is
// inverted in shared memory, else 0.
int packed_bottom_bytes(int n, bool fp64);

// Projection steps (natural layouts): f = div(u, v, w) - S (S nullable), and
// u, v, w -= beta_face grad(phi) using the level-0 weights.
cudaError_t launch_project_rhs(int nx, int ny, int nz, double h, const double *u, const double *v,
                               const double *w, const double *S, double *f, cudaStream_t st);
cudaError_t launch_project_correct(int nx, int ny, int nz, double h, const double *wx,
                                   const double *wy, const double *wz, const double *phi,
                                   double *u, double *v, double *w, cudaStream_t st,
                                   bool wide = false);

cudaError_t launch_beta_grad(int nx, int ny, int nz, double inv_h2, int bcm, const double *beta,
                             const double *phi, const double *lam, double *dbeta, cudaStream_t st);
// fout = f - lift of the packed wall values (level-0 FP64 weights, layout of mg.h).
cudaError_t launch_bc_lift(int nx, int ny, int nz, double inv_h, int bcm, const double *wx,
                           const double *wy, const double *wz, const double *vals,
                           const double *f, double *fout, cudaStream_t st,
                           bool wide = false);
// Every box of S: field (0 = f, 1 = phi) -= its mean over the box's cells.
// partials: TK_COLZ tiles of S; mean: one double per box (written).
cudaError_t launch_remove_mean(const BoxSet<double> &S, int field, double *partials, double *mean,
                               cudaStream_t st);

// ---- coupled levels (the boxes of one level solved as one domain) ---------
// Copy each record's source patch into the destination box's guard cells.
template <class T>
cudaError_t launch_exchange(const BoxSet<T> &S, const int *active, const ExchRec *rec, int nrec,
                            int max_cells, cudaStream_t st, int second = 0);
// The guard cells of the six faces of every box of S = v (phi arrays).
template <class T>
cudaError_t launch_guard_fill(const BoxSet<T> &S, T v, cudaStream_t st);
// Dense inverse of the union of the coarsest levels (S in union order).
cudaError_t launch_union_inverse(const SetupSet &S, const UnionBottom &U, double *work,
                                 double *inv64, float *inv32, cudaStream_t st);
// phi = Ainv f on the union of the coarsest levels.
template <class T>
cudaError_t launch_union_bottom(const BoxSet<T> &S, const UnionBottom &U, const T *ainv,
                                const int *active, cudaStream_t st);
// norm[b] <- sqrt(sum over b of norm[b]^2), for every b.
cudaError_t launch_norm_combine(int nbox, double *norm, cudaStream_t st);

// ---- preconditioned CG (level-0 FP64 arrays; see kernels.cu) -------------
struct PcgScalars {
    double *rz, *rzn, *pq, *beta, *alpha;  // [nbox] each
};
// op 0: <r, z> -> sum_out; 1: p = z + beta p; 2: q = A p and <p, q> -> sum_out;
// 3: x += alpha p, r -= alpha q, phi = 0 and ||r|| -> sum_out;
// 4: x = phi, r = f - A x, p = 0 and ||r|| -> sum_out (nullable); 5: phi = x.
cudaError_t launch_pcg(const BoxSet<double> &S, const int *active, int op, double *const *pv,
                       double *const *qv, const PcgScalars &sc, double *partials,
                       double *sum_out, cudaStream_t st);
// step 0: beta = rzn / rz (0 first), rz = rzn; step 1: alpha = rz / pq.
// out[box] = max |f| (field 0) or max |f - A phi| (field 1; phi2 where
// side[box] is set) over the box's level-0 cells.
cudaError_t launch_max_norm(const BoxSet<double> &S, const int *side, int field,
                            double *partials, double *out, cudaStream_t st);
// Mixed precision: op 0: FP32 f = r / nrm, FP32 phi = 0; op 1: FP64 phi =
// nrm * FP32 phi (the preconditioned residual z).
cudaError_t launch_pcg_mixed(const BoxSet<double> &S64, const BoxSet<float> &S32, const int *active,
                             int op, const double *nrm, cudaStream_t st);
cudaError_t launch_pcg_scalars(int nbox, const int *active, int step, const PcgScalars &sc,
                               cudaStream_t st);

}  // namespace mg
