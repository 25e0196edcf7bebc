/*
 * mg_ops.h -- single-stage entry points of the multigrid solver in mg.h.
 *
 * Each call runs one stage of the V-cycle on one box, on arrays the caller
 * owns, so the stages can be checked one at a time and reused by callers
 * that drive their own cycle.  Definitions are the ones stated in mg.h
 * (paper Sec. 1 names the variable-coefficient Poisson solve; the stage
 * definitions are this library's reading of it).
 *
 * LEVEL LAYOUT.  Every array of an (nx, ny, nz) level holds
 * mg_layout_elems(n) elements of the stage's precision and uses
 *     row pitch  P = round_up(nx + 1, 8),  plane pitch Q = P * (ny + 1),
 *     element (i, j, k) at offset (k + 1) * Q + j * P + i.
 * Cell arrays (phi, f, invD, r) use i < nx, j < ny, k < nz; x-face weights
 * use i <= nx (face i lies between cells i-1 and i), y-face weights j <= ny,
 * z-face weights k <= nz.  Every element outside those ranges (the guard
 * plane below k = 0, the row j = ny, the columns i >= nx, the plane k = nz
 * of cell arrays) must be zero in phi arrays; the library never writes them.
 * Face "weights" are beta_face / h^2, so A phi = sum_f w_f (phi_nbr - phi_c).
 *
 * Precision: `prec` is MG_OPS_F64 (double arrays) or MG_OPS_F32 (float).
 * All calls are asynchronous on `stream`; pointers are device pointers.
 * Return: MG_OK, MG_ERR_INVALID_ARG (bad size/pointer/precision), MG_ERR_CUDA.
 */
#ifndef MG_OPS_H
#define MG_OPS_H

#include "mg.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { MG_OPS_F64 = 0, MG_OPS_F32 = 1 };

/* Pitches and total elements of the level layout of an n = {nx, ny, nz} box. */
int mg_layout(const int n[3], long long *P, long long *Q, long long *elems);

/* Face weights from cell beta (contiguous (nz, ny, nx) float64):
 * w = harmonic mean of the two cells' beta / h^2; a wall face has 2 beta / h^2
 * (Dirichlet wall) or 0 (Neumann wall), per the wall mask bc of mg.h
 * (0..63; 0 = every wall Dirichlet).  Writes FP64 weights wx, wy, wz in the
 * level layout.  The harmonic mean 2ab/(a+b) is taken as (2a/h^2) b times a
 * reciprocal of a + b within one ulp (see mg_op_inv_diag), so a weight is
 * within a few ulp of the correctly rounded value. */
int mg_op_face_weights(const int n[3], double h, int bc, const double *beta, double *wx,
                       double *wy, double *wz, void *stream);

/* Coarse weights of an all-even fine level n: w_c = (mean of the 4 fine faces
 * covering the coarse face) / 4, i.e. the coarse face beta is the mean of the
 * fine ones and the coarse spacing is 2h.  FP64. */
int mg_op_coarsen_weights(const int n_fine[3], const double *wx, const double *wy,
                          const double *wz, double *cwx, double *cwy, double *cwz,
                          void *stream);

/* D = sum of the 6 face weights of each cell (the negated diagonal of A),
 * invD = 1 / D, FP64, within one ulp (no FP64 division: the FP32
 * reciprocal refined by one cubic Newton step; D outside FP32's normal
 * range takes the division).  D may be NULL. */
int mg_op_inv_diag(const int n[3], const double *wx, const double *wy, const double *wz,
                   double *invD, double *D, void *stream);

/* Round FP64 level arrays to FP32 (weights and inverse diagonal). */
int mg_op_round_f32(const int n[3], const double *wx, const double *wy, const double *wz,
                    const double *invD, float *wx32, float *wy32, float *wz32,
                    float *invD32, void *stream);

/* One red (color 0) or black (color 1) Gauss-Seidel pass in place: every cell
 * with (i+j+k) % 2 == color gets phi = (sum_f w_f phi_nbr - f) * invD. */
int mg_op_rbgs_pass(int prec, const int n[3], const void *wx, const void *wy, const void *wz,
                    const void *invD, const void *f, void *phi, int color, void *stream);

/* One full red-then-black sweep as the solver runs it on large levels
 * (fused, out of place: reads phi_in, writes phi_out; phi_in is not
 * modified).  Equal to a red pass followed by a black pass.  The sweep reads
 * no inverse diagonal: each update takes the reciprocal of
 * D = ((wx- + wx+) + (wy- + wy+)) + (wz- + wz+), summed from the six weights
 * it loads (FP32: correctly rounded; FP64: the value mg_op_inv_diag
 * stores).  Each CTA marches
 * through zc planes (zc <= 0: 32).  UNSUPPORTED for levels of 2^31 or more
 * elements (the kernel indexes with 32-bit offsets). */
int mg_op_rbgs_sweep(int prec, const int n[3], const void *wx, const void *wy, const void *wz,
                     const void *f, const void *phi_in, void *phi_out, int zc, void *stream);

/* The same sweep in FP32 with its operand tiles staged by the Tensor Memory
 * Accelerator (bulk tensor copies into shared memory, completion counted by
 * mbarriers).  Bitwise equal to mg_op_rbgs_sweep with MG_OPS_F32.  Waits on
 * the copies are bounded: MG_ERR_TIMEOUT if one gave up.  Synchronises the
 * stream (to read the error word); MG_ERR_UNSUPPORTED if the driver cannot
 * encode tensor maps or the level is too small for one copy box (needs
 * nx >= 64 and ny >= 11). */
int mg_op_rbgs_sweep_tma(const int n[3], const float *wx, const float *wy, const float *wz,
                         const float *f, const float *phi_in, float *phi_out, int zc,
                         void *stream);

/* The TMA-fed sweep with the level's prolongation fused (the V-cycle's
 * first post-smoothing sweep): the result is bitwise that of
 * mg_op_prolong_add(phic, phi_in) followed by mg_op_rbgs_sweep_tma, but
 * phi_in is left as it is.  phic: the coarse level's phi (n / 2 cells, level
 * layout); n must be even.  Same errors as mg_op_rbgs_sweep_tma, and
 * UNSUPPORTED if the coarse level is too small for its copy box (n / 2 >= 32
 * in x, >= 5 in y). */
int mg_op_rbgs_sweep_tma_prolong(const int n[3], const float *wx, const float *wy,
                                 const float *wz, const float *f, const float *phic,
                                 const float *phi_in, float *phi_out, int zc, void *stream);

/* In the residual stages below, D (nullable) is the stored diagonal of
 * mg_op_inv_diag in the stage precision; when NULL it is summed from the six
 * weights of each cell. */

/* r = f - A phi (cell array). */
int mg_op_residual(int prec, const int n[3], const void *wx, const void *wy, const void *wz,
                   const void *D, const void *f, const void *phi, void *r, void *stream);

/* Fused residual and restriction of an all-even level n: fc = mean over the
 * 8 children of (f - A phi); phic (coarse solution) is set to zero. */
int mg_op_residual_restrict(int prec, const int n_fine[3], const void *wx, const void *wy,
                            const void *wz, const void *D, const void *f, const void *phi,
                            void *fc, void *phic, void *stream);

/* The same right after a red-black sweep (the last operation on phi was a
 * black pass): the black cells then satisfy their own equations, so only the
 * 4 red children of each coarse cell are evaluated and the black ones count
 * as zero.  Equal to mg_op_residual_restrict to rounding in that state. */
int mg_op_residual_restrict_red(int prec, const int n_fine[3], const void *wx, const void *wy,
                                const void *wz, const void *D, const void *f, const void *phi,
                                void *fc, void *phic, void *stream);

/* phi += coarse value of each cell's parent (piecewise-constant
 * prolongation) for an all-even fine level n. */
int mg_op_prolong_add(int prec, const int n_fine[3], const void *phic, void *phi,
                      void *stream);

/* Exact coarsest-level solve set-up: Ainv = A^{-1} as a dense row-major
 * (N, N) FP64 matrix, N = nx*ny*nz <= MG_MAX_BOTTOM, dense index
 * (k*ny + j)*nx + i.  work: N*N doubles of scratch.  singular != 0 (every
 * wall Neumann, A singular on the constants): Ainv = -(M + c 1 1^T)^{-1} with
 * M = -A and c = trace(M) / N^2, so that x = Ainv r solves
 * A x = r - mean(r); x has zero mean when r has. */
int mg_op_bottom_inverse(const int n[3], int singular, const double *wx, const double *wy,
                         const double *wz, double *work, double *Ainv, void *stream);

/* phi = Ainv f on the coarsest level (Ainv in the stage precision). */
int mg_op_bottom_solve(int prec, const int n[3], const void *Ainv, const void *f, void *phi,
                       void *stream);

/* Residual norm: *out (device double) = ||f - A phi||_2, reduced in a fixed
 * order.  `partials` is caller-owned device scratch of at least
 * mg_op_norm_scratch(n) doubles. */
long long mg_op_norm_scratch(const int n[3]);
int mg_op_residual_norm(int prec, const int n[3], const void *wx, const void *wy,
                        const void *wz, const void *D, const void *f, const void *phi,
                        double *partials, double *out, void *stream);

/* Residual norm that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory, such as
 * an application whose device memory all belongs to its own pool allocator
 * (nothing may call cudaMalloc beside it) or a time-critical loop that cannot
 * take the implicit synchronisation of cudaMalloc/cudaFree.  It computes the
 * same *out = ||f - A phi||_2 as mg_op_residual_norm, but its per-tile partial
 * sums live in a file-scope device array of 65536 doubles (512 KiB, held on
 * every GPU that loads the library until the process exits) instead of
 * caller scratch; it calls no cudaMalloc, cudaFree or allocating routine.
 * Limit: column tiles <= 65536, a tile being 32 x 8 columns of 16 planes
 * (ceil(nx/32) * ceil(ny/8) * ceil(nz/16) when nx is a multiple of 32, else
 * ceil(nx*ny/256) * ceil(nz/16); e.g. 512^3 uses 32768); larger boxes return
 * MG_ERR_INVALID_ARG before anything runs.
 * The first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  The address is cached per device for the life of the
 * process: do not use this entry point after a cudaDeviceReset (the
 * module, and with it the array, may then sit elsewhere).  Every call
 * reuses the array and overwrites the slots it
 * reads, so nothing needs clearing, but calls that overlap on the GPU race on
 * it: order them (same stream, or synchronise).  Arguments as
 * mg_op_residual_norm without `partials`. */
int mg_op_residual_norm_noalloc(int prec, const int n[3], const void *wx, const void *wy,
                                const void *wz, const void *D, const void *f, const void *phi,
                                double *out, void *stream);

/* Mixed-precision refinement step on the finest level (FP64 x, f, weights,
 * D; FP32 correction e and scaled residual r32):
 *   x += (*c_e) e  (in place), then e = 0;  r = f - A64 x;
 *   r32 = float(r) * float(1/(*c_r));
 *   *out = (*c_r) * ||r32||_2  (= ||r||_2 to FP32 accuracy; fixed-order
 *   reduction through `partials`).
 * c_e and c_r are device doubles, c_r > 0. */
int mg_op_refine(const int n[3], const double *wx, const double *wy, const double *wz,
                 const double *D, const double *f, double *x, float *e, float *r32,
                 const double *c_e, const double *c_r, double *partials, double *out,
                 void *stream);

/* Beta gradient of one right-hand side (see mg_adjoint): dbeta += chain of
 * the face products of phi and lambda; Neumann wall faces of the mask bc add
 * nothing.  beta, phi, lambda, dbeta are contiguous (nz, ny, nx) float64. */
int mg_op_beta_grad(const int n[3], double h, int bc, const double *beta, const double *phi,
                    const double *lambda, double *dbeta, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MG_OPS_H */
