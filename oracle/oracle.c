/*
 * oracle.c -- plain, slow FP64 CPU reference for the cell-centred
 * variable-coefficient Poisson solve div(beta grad phi) = f.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or constant with the CUDA solver and never calls it.
 *
 * The problem is the one the paper names in Sec. 1: each MAESTRO time step
 * solves a variable-coefficient Poisson equation that enforces the low-Mach
 * velocity constraint (the paper's Sec. 3 blames these linear solves for
 * MAESTRO's weaker scaling).  The paper gives no discretisation, so this file
 * writes out the standard cell-centred reading, one definition per function:
 *
 *   cells        (i, j, k), centre ((i+1/2)h, (j+1/2)h, (k+1/2)h), C order
 *                (nz, ny, nx) with x fastest;
 *   faces        bx (nz, ny, nx+1): face i lies between cells i-1 and i;
 *                by (nz, ny+1, nx); bz (nz+1, ny, nx);
 *   face beta    harmonic mean 2 a b / (a + b) of the two cells; a face on
 *                the box wall carries 2 beta of its one cell (the wall sits
 *                h/2 from the cell centre where phi = 0);
 *   operator     (A phi)_c = (1/h^2) sum over the 6 faces of
 *                beta_face (phi_neighbour - phi_c), phi_neighbour = 0 outside;
 *   smoother     red-black Gauss-Seidel, red = (i+j+k) even first; each
 *                update solves row c of A phi = f for phi_c;
 *   multigrid    V(nu1, nu2) cycles; all dimensions halved while all are even
 *                and at least 4; restriction = mean of the 8 children;
 *                prolongation = piecewise-constant add; coarse face beta =
 *                mean of the 4 fine faces it covers; coarse h = 2h; the
 *                coarsest level is solved exactly (dense Cholesky up to 1024
 *                cells, else conjugate gradients to 1e-15);
 *   convergence  ||f - A phi||_2 / ||f||_2 <= tol (unweighted discrete L2);
 *   adjoint      for L with dL/dphi = g: A lambda = g (A is symmetric),
 *                dL/df = lambda, dL/dbeta_face = (lambda_n - lambda_c)
 *                (phi_n - phi_c)/h^2 (wall face: lambda_c phi_c / h^2), chained
 *                to cell beta through the harmonic mean;
 *   projection   f = div(u) - S from face velocities; after the solve each
 *                face velocity loses beta_face (phi_high - phi_low) / h, so
 *                the corrected field has div = S;
 *   walls        a mask bc selects each wall's condition, bit w for wall w in
 *                the order x-, x+, y-, y+, z-, z+: bit clear = Dirichlet (the
 *                wall face carries 2 beta, as above), bit set = Neumann (no
 *                flux through the wall: the wall face carries 0).  Non-zero
 *                wall values move to the right-hand side (a lift): a
 *                Dirichlet value g adds 2 beta (g - phi_c)/h^2 to row c, a
 *                Neumann outward flux q (beta dphi/dn) adds q/h, so the solve
 *                runs on f - 2 beta g/h^2 - q/h with homogeneous walls.  With
 *                every wall Neumann, A is singular (constants): the solve
 *                removes the mean of f (the compatibility condition) and
 *                returns the zero-mean solution; its coarsest level is solved
 *                with M + c 1 1^T, which is positive definite and exact on
 *                zero-mean right-hand sides;
 *   periodic     bits 6, 7, 8 of the wall mask make the x, y or z axis
 *                periodic: cell n-1 and cell 0 of that axis are neighbours
 *                across one face (harmonic mean of their beta, stored at
 *                both face positions 0 and n).  With every axis periodic or
 *                with Neumann walls on both ends, A is singular and the
 *                solve is the zero-mean one, as above.  The oracle solves
 *                periodic boxes by conjugate gradients on the operator;
 *   krylov       (a variant the paper does not describe) conjugate gradients
 *                on the symmetric positive definite -A, preconditioned by
 *                one V-cycle from a zero start whose post-smoothing sweeps
 *                run black then red (the adjoint of the red-then-black
 *                pre-smoother) with nu1 = nu2: then the cycle is a symmetric
 *                linear map of its right-hand side, and -V approximates
 *                (-A)^{-1};
 *   level        a level of several boxes (paper Sec. 2: the union of
 *                disjoint rectangular grids of a MultiFAB) is one domain:
 *                the same operator on the union, faces between cells of two
 *                boxes are interior faces (harmonic mean), faces on the
 *                union's boundary are Dirichlet walls.  The oracle takes the
 *                union as a mask over its bounding box and solves by
 *                conjugate gradients on the masked operator.
 *
 * Loops over cells run under OpenMP where each iteration is independent; all
 * reductions are serial, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXLEV 32

/* ---------------------------------------------------------------- indexing */

static size_t cell(int i, int j, int k, int nx, int ny)
{
    return ((size_t)k * ny + j) * nx + i;
}
static size_t xface(int i, int j, int k, int nx, int ny)   /* i in 0..nx */
{
    return ((size_t)k * ny + j) * (nx + 1) + i;
}
static size_t yface(int i, int j, int k, int nx, int ny)   /* j in 0..ny */
{
    return ((size_t)k * (ny + 1) + j) * nx + i;
}
static size_t zface(int i, int j, int k, int nx, int ny)   /* k in 0..nz */
{
    return ((size_t)k * ny + j) * nx + i;
}

/* phi outside the box is the homogeneous Dirichlet value 0 */
static double value_at(const double *phi, int i, int j, int k, int nx, int ny, int nz)
{
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return 0.0;
    return phi[cell(i, j, k, nx, ny)];
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------- face beta */

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

/* Wall w (0..5 = x-, x+, y-, y+, z-, z+) is Neumann when bit w of bc is set. */
static int neumann(int bc, int w) { return (bc >> w) & 1; }

/* The coefficient of a wall face next to a cell of coefficient b. */
static double wall_face(int bc, int w, double b) { return neumann(bc, w) ? 0.0 : 2.0 * b; }

/* Face coefficients from cell beta: harmonic mean inside; on walls 2 beta
 * (Dirichlet) or 0 (Neumann) as the mask bc says. */
void oracle_face_beta_bc(int nx, int ny, int nz, const double *beta, int bc,
                         double *bx, double *by, double *bz)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                double v;
                if (i == 0) v = wall_face(bc, 0, beta[cell(0, j, k, nx, ny)]);
                else if (i == nx) v = wall_face(bc, 1, beta[cell(nx - 1, j, k, nx, ny)]);
                else v = harmonic(beta[cell(i - 1, j, k, nx, ny)], beta[cell(i, j, k, nx, ny)]);
                bx[xface(i, j, k, nx, ny)] = v;
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double v;
                if (j == 0) v = wall_face(bc, 2, beta[cell(i, 0, k, nx, ny)]);
                else if (j == ny) v = wall_face(bc, 3, beta[cell(i, ny - 1, k, nx, ny)]);
                else v = harmonic(beta[cell(i, j - 1, k, nx, ny)], beta[cell(i, j, k, nx, ny)]);
                by[yface(i, j, k, nx, ny)] = v;
            }
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double v;
                if (k == 0) v = wall_face(bc, 4, beta[cell(i, j, 0, nx, ny)]);
                else if (k == nz) v = wall_face(bc, 5, beta[cell(i, j, nz - 1, nx, ny)]);
                else v = harmonic(beta[cell(i, j, k - 1, nx, ny)], beta[cell(i, j, k, nx, ny)]);
                bz[zface(i, j, k, nx, ny)] = v;
            }
}

/* Face coefficients with every wall Dirichlet. */
void oracle_face_beta(int nx, int ny, int nz, const double *beta,
                      double *bx, double *by, double *bz)
{
    oracle_face_beta_bc(nx, ny, nz, beta, 0, bx, by, bz);
}

/* Right-hand-side lift of non-zero wall values.  vals holds one value per
 * wall face, walls in the order x-, x+, y-, y+, z-, z+; an x wall is an
 * (nz, ny) array, a y wall (nz, nx), a z wall (ny, nx), C order.  For a
 * Dirichlet wall the value is phi on the wall and the adjacent cell's row
 * gains 2 beta_c (g - phi_c)/h^2, of which the known part 2 beta_c g/h^2 is
 * subtracted from f; for a Neumann wall it is the outward flux beta dphi/dn
 * and q/h is subtracted from f. */
void oracle_bc_lift(int nx, int ny, int nz, double h, const double *beta, int bc,
                    const double *vals, double *f)
{
    double ih = 1.0 / h, ih2 = 1.0 / (h * h);
    size_t off = 0;
    for (int w = 0; w < 6; ++w) {
        int axis = w / 2, hi = w & 1;
        int na = axis == 0 ? ny : nx;                 /* fastest wall index */
        int nb = axis == 2 ? ny : nz;                 /* slowest wall index */
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                int i, j, k;
                if (axis == 0) { i = hi ? nx - 1 : 0; j = a; k = b; }
                else if (axis == 1) { i = a; j = hi ? ny - 1 : 0; k = b; }
                else { i = a; j = b; k = hi ? nz - 1 : 0; }
                size_t c = cell(i, j, k, nx, ny);
                double v = vals[off + (size_t)b * na + a];
                if (neumann(bc, w)) f[c] -= v * ih;
                else f[c] -= 2.0 * beta[c] * v * ih2;
            }
        off += (size_t)na * nb;
    }
}

/* Coarse face beta = mean of the 4 fine faces that make up the coarse face.
 * (nx, ny, nz) are the fine dimensions, all even. */
void oracle_coarsen_faces(int nx, int ny, int nz,
                          const double *bx, const double *by, const double *bz,
                          double *cbx, double *cby, double *cbz)
{
    int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    for (int K = 0; K < cz; ++K)
        for (int J = 0; J < cy; ++J)
            for (int I = 0; I <= cx; ++I) {
                double s = 0.0;
                for (int b = 0; b < 2; ++b)
                    for (int c = 0; c < 2; ++c)
                        s += bx[xface(2 * I, 2 * J + b, 2 * K + c, nx, ny)];
                cbx[xface(I, J, K, cx, cy)] = s / 4.0;
            }
    for (int K = 0; K < cz; ++K)
        for (int J = 0; J <= cy; ++J)
            for (int I = 0; I < cx; ++I) {
                double s = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int c = 0; c < 2; ++c)
                        s += by[yface(2 * I + a, 2 * J, 2 * K + c, nx, ny)];
                cby[yface(I, J, K, cx, cy)] = s / 4.0;
            }
    for (int K = 0; K <= cz; ++K)
        for (int J = 0; J < cy; ++J)
            for (int I = 0; I < cx; ++I) {
                double s = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        s += bz[zface(2 * I + a, 2 * J + b, 2 * K, nx, ny)];
                cbz[zface(I, J, K, cx, cy)] = s / 4.0;
            }
}

/* --------------------------------------------------------------- operator */

/* Sum over the 6 faces of beta_face * phi_neighbour, and the sum of the
 * 6 face coefficients (the negated diagonal times h^2). */
static void neighbour_sums(int i, int j, int k, int nx, int ny, int nz,
                           const double *bx, const double *by, const double *bz,
                           const double *phi, double *sum_bphi, double *sum_b)
{
    double bw = bx[xface(i, j, k, nx, ny)], be = bx[xface(i + 1, j, k, nx, ny)];
    double bs = by[yface(i, j, k, nx, ny)], bn = by[yface(i, j + 1, k, nx, ny)];
    double bd = bz[zface(i, j, k, nx, ny)], bu = bz[zface(i, j, k + 1, nx, ny)];
    *sum_bphi = bw * value_at(phi, i - 1, j, k, nx, ny, nz)
              + be * value_at(phi, i + 1, j, k, nx, ny, nz)
              + bs * value_at(phi, i, j - 1, k, nx, ny, nz)
              + bn * value_at(phi, i, j + 1, k, nx, ny, nz)
              + bd * value_at(phi, i, j, k - 1, nx, ny, nz)
              + bu * value_at(phi, i, j, k + 1, nx, ny, nz);
    *sum_b = bw + be + bs + bn + bd + bu;
}

/* out = A phi */
void oracle_apply(int nx, int ny, int nz, double h,
                  const double *bx, const double *by, const double *bz,
                  const double *phi, double *out)
{
    double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double sbp, sb;
                neighbour_sums(i, j, k, nx, ny, nz, bx, by, bz, phi, &sbp, &sb);
                out[cell(i, j, k, nx, ny)] = (sbp - sb * phi[cell(i, j, k, nx, ny)]) * ih2;
            }
}

/* r = f - A phi */
void oracle_residual(int nx, int ny, int nz, double h,
                     const double *bx, const double *by, const double *bz,
                     const double *f, const double *phi, double *r)
{
    double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double sbp, sb;
                size_t c = cell(i, j, k, nx, ny);
                neighbour_sums(i, j, k, nx, ny, nz, bx, by, bz, phi, &sbp, &sb);
                r[c] = f[c] - (sbp - sb * phi[c]) * ih2;
            }
}

/* One colour of red-black Gauss-Seidel, in place: every cell with
 * (i+j+k) % 2 == color is set so that its own row of A phi = f holds:
 * (sum_f b_f phi_n - phi_c sum_f b_f) / h^2 = f_c. */
void oracle_rbgs_pass(int nx, int ny, int nz, double h,
                      const double *bx, const double *by, const double *bz,
                      const double *f, double *phi, int color)
{
    double h2 = h * h;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (((i + j + k) & 1) != color) continue;
                double sbp, sb;
                size_t c = cell(i, j, k, nx, ny);
                neighbour_sums(i, j, k, nx, ny, nz, bx, by, bz, phi, &sbp, &sb);
                phi[c] = (sbp - h2 * f[c]) / sb;
            }
}

/* coarse = mean of the 8 children; (nx, ny, nz) fine, all even */
void oracle_restrict(int nx, int ny, int nz, const double *fine, double *coarse)
{
    int cx = nx / 2, cy = ny / 2, cz = nz / 2;
#pragma omp parallel for schedule(static)
    for (int K = 0; K < cz; ++K)
        for (int J = 0; J < cy; ++J)
            for (int I = 0; I < cx; ++I) {
                double s = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a)
                            s += fine[cell(2 * I + a, 2 * J + b, 2 * K + c, nx, ny)];
                coarse[cell(I, J, K, cx, cy)] = s / 8.0;
            }
}

/* fine += coarse value of the parent cell; (nx, ny, nz) fine, all even */
void oracle_prolong_add(int nx, int ny, int nz, const double *coarse, double *fine)
{
    int cx = nx / 2, cy = ny / 2;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                fine[cell(i, j, k, nx, ny)] += coarse[cell(i / 2, j / 2, k / 2, cx, cy)];
}

static double norm2(size_t n, const double *x)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += x[i] * x[i];
    return sqrt(s);
}

double oracle_norm2(long long n, const double *x) { return norm2((size_t)n, x); }

/* ---------------------------------------------------------- level builder */

/* Level dimensions: halve every dimension while all are even and >= 4.
 * Writes up to MAXLEV triples (nx, ny, nz) and returns the level count. */
int oracle_levels(int nx, int ny, int nz, int *dims)
{
    int n = 0;
    dims[0] = nx; dims[1] = ny; dims[2] = nz; n = 1;
    while (n < MAXLEV && nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 &&
           nx >= 4 && ny >= 4 && nz >= 4) {
        nx /= 2; ny /= 2; nz /= 2;
        dims[3 * n] = nx; dims[3 * n + 1] = ny; dims[3 * n + 2] = nz;
        ++n;
    }
    return n;
}

typedef struct {
    int nx, ny, nz;
    double h;
    double *bx, *by, *bz, *phi, *f, *r;
} level_t;

typedef struct {
    int nlev, nu1, nu2;
    int post_first;          /* colour of each post-smoothing sweep's first pass (0 red) */
    int singular;            /* every wall Neumann: A has the constants as null space */
    level_t L[MAXLEV];
    /* coarsest level: dense Cholesky factor of M = -h^2 A (SPD), plus
     * c 1 1^T when A is singular */
    int dense_n;
    double *chol;
} hier_t;

static size_t ncell(const level_t *l) { return (size_t)l->nx * l->ny * l->nz; }

static void free_hier(hier_t *H)
{
    for (int l = 0; l < H->nlev; ++l) {
        free(H->L[l].bx); free(H->L[l].by); free(H->L[l].bz);
        free(H->L[l].phi); free(H->L[l].f); free(H->L[l].r);
    }
    free(H->chol);
    H->nlev = 0;
    H->chol = NULL;
}

/* Dense M = -h^2 A on the coarsest level, built column by column from the
 * operator applied to unit vectors, then factored M = L L^T in place
 * (lower triangle).  When A is singular, c 1 1^T with c = trace(M)/n^2 is
 * added first: M + c 1 1^T is positive definite, and for a right-hand side
 * of zero sum its solution is the zero-mean solution of M x = rhs.
 * Returns 0, or -1 if the matrix is not positive definite. */
static int factor_bottom(hier_t *H)
{
    level_t *b = &H->L[H->nlev - 1];
    int n = (int)ncell(b);
    H->dense_n = n;
    H->chol = (double *)calloc((size_t)n * n, sizeof(double));
    double *e = (double *)calloc((size_t)n, sizeof(double));
    double *col = (double *)calloc((size_t)n, sizeof(double));
    for (int c = 0; c < n; ++c) {
        memset(e, 0, sizeof(double) * n);
        e[c] = 1.0;
        oracle_apply(b->nx, b->ny, b->nz, b->h, b->bx, b->by, b->bz, e, col);
        for (int r = 0; r < n; ++r) H->chol[(size_t)r * n + c] = -b->h * b->h * col[r];
    }
    free(e);
    free(col);
    double *a = H->chol;
    if (H->singular) {
        double tr = 0.0;
        for (int c = 0; c < n; ++c) tr += a[(size_t)c * n + c];
        double shift = tr / ((double)n * n);
        for (size_t q = 0; q < (size_t)n * n; ++q) a[q] += shift;
    }
    for (int j = 0; j < n; ++j) {
        double d = a[(size_t)j * n + j];
        for (int p = 0; p < j; ++p) d -= a[(size_t)j * n + p] * a[(size_t)j * n + p];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        a[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = a[(size_t)i * n + j];
            for (int p = 0; p < j; ++p) s -= a[(size_t)i * n + p] * a[(size_t)j * n + p];
            a[(size_t)i * n + j] = s / d;
        }
    }
    return 0;
}

static double mean(size_t n, const double *x)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += x[i];
    return s / (double)n;
}

static void remove_mean(size_t n, double *x)
{
    double m = mean(n, x);
    for (size_t i = 0; i < n; ++i) x[i] -= m;
}

/* Conjugate gradients on M x = rhs with M = -h^2 A, for coarsest levels too
 * large for a dense factor.  Iterates until ||rhs - M x|| <= 1e-15 ||rhs||.
 * When A is singular the right-hand side loses its mean first (CG then stays
 * in the zero-mean subspace, where M is positive definite). */
static void cg_bottom(level_t *b, int singular)
{
    size_t n = ncell(b);
    double *x = b->phi, *rhs = b->r;
    if (singular) remove_mean(n, rhs);
    double *res = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    double mh2 = -b->h * b->h;
    for (size_t i = 0; i < n; ++i) { x[i] = 0.0; res[i] = rhs[i]; p[i] = rhs[i]; }
    double rr = 0.0, r0;
    for (size_t i = 0; i < n; ++i) rr += res[i] * res[i];
    r0 = rr;
    for (int it = 0; it < 100000 && rr > 1e-30 * r0; ++it) {
        oracle_apply(b->nx, b->ny, b->nz, b->h, b->bx, b->by, b->bz, p, q);
        double pq = 0.0;
        for (size_t i = 0; i < n; ++i) { q[i] *= mh2; pq += p[i] * q[i]; }
        double alpha = rr / pq;
        double rr1 = 0.0;
        for (size_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            res[i] -= alpha * q[i];
            rr1 += res[i] * res[i];
        }
        double beta = rr1 / rr;
        rr = rr1;
        for (size_t i = 0; i < n; ++i) p[i] = res[i] + beta * p[i];
    }
    free(res); free(p); free(q);
}

/* Exact solve A e = f on the coarsest level: e = -M^{-1} h^2 f. */
static void bottom_solve(hier_t *H)
{
    level_t *b = &H->L[H->nlev - 1];
    size_t n = ncell(b);
    double h2 = b->h * b->h;
    if (H->chol) {
        int m = H->dense_n;
        double *y = b->phi;
        for (int i = 0; i < m; ++i) {           /* L y = -h^2 f */
            double s = -h2 * b->f[i];
            for (int p = 0; p < i; ++p) s -= H->chol[(size_t)i * m + p] * y[p];
            y[i] = s / H->chol[(size_t)i * m + i];
        }
        for (int i = m - 1; i >= 0; --i) {      /* L^T e = y */
            double s = y[i];
            for (int p = i + 1; p < m; ++p) s -= H->chol[(size_t)p * m + i] * y[p];
            y[i] = s / H->chol[(size_t)i * m + i];
        }
    } else {
        for (size_t i = 0; i < n; ++i) b->r[i] = -h2 * b->f[i];
        cg_bottom(b, H->singular);
    }
}

/* Build the hierarchy (faces on every level) from cell beta and the wall
 * mask. */
static int build_hier(hier_t *H, int nx, int ny, int nz, double h, const double *beta,
                      int bc, int nu1, int nu2)
{
    int dims[3 * MAXLEV];
    memset(H, 0, sizeof(*H));
    H->nlev = oracle_levels(nx, ny, nz, dims);
    H->nu1 = nu1;
    H->nu2 = nu2;
    H->singular = (bc & 63) == 63;
    for (int l = 0; l < H->nlev; ++l) {
        level_t *L = &H->L[l];
        L->nx = dims[3 * l]; L->ny = dims[3 * l + 1]; L->nz = dims[3 * l + 2];
        L->h = (l == 0) ? h : 2.0 * H->L[l - 1].h;
        size_t n = ncell(L);
        L->bx = (double *)calloc((size_t)L->nz * L->ny * (L->nx + 1), sizeof(double));
        L->by = (double *)calloc((size_t)L->nz * (L->ny + 1) * L->nx, sizeof(double));
        L->bz = (double *)calloc((size_t)(L->nz + 1) * L->ny * L->nx, sizeof(double));
        L->phi = (double *)calloc(n, sizeof(double));
        L->f = (double *)calloc(n, sizeof(double));
        L->r = (double *)calloc(n, sizeof(double));
        if (l == 0)
            oracle_face_beta_bc(L->nx, L->ny, L->nz, beta, bc, L->bx, L->by, L->bz);
        else {
            level_t *F = &H->L[l - 1];
            oracle_coarsen_faces(F->nx, F->ny, F->nz, F->bx, F->by, F->bz, L->bx, L->by, L->bz);
        }
    }
    level_t *b = &H->L[H->nlev - 1];
    if (ncell(b) <= 1024) {
        if (factor_bottom(H) != 0) { free(H->chol); H->chol = NULL; return -1; }
    }
    return 0;
}

static void vcycle(hier_t *H, int l)
{
    level_t *L = &H->L[l];
    if (l == H->nlev - 1) { bottom_solve(H); return; }
    for (int s = 0; s < H->nu1; ++s) {
        oracle_rbgs_pass(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->f, L->phi, 0);
        oracle_rbgs_pass(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->f, L->phi, 1);
    }
    oracle_residual(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->f, L->phi, L->r);
    level_t *C = &H->L[l + 1];
    oracle_restrict(L->nx, L->ny, L->nz, L->r, C->f);
    memset(C->phi, 0, sizeof(double) * ncell(C));
    vcycle(H, l + 1);
    oracle_prolong_add(L->nx, L->ny, L->nz, C->phi, L->phi);
    for (int s = 0; s < H->nu2; ++s) {
        oracle_rbgs_pass(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->f, L->phi,
                         H->post_first);
        oracle_rbgs_pass(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->f, L->phi,
                         1 - H->post_first);
    }
}

/* ---------------------------------------------------------------- solvers */

/* Status codes of the oracle's solve. */
enum { OR_OK = 0, OR_NOT_CONVERGED = 1, OR_NONFINITE = 2, OR_BAD = 3 };

static int run_cycles(hier_t *H, const double *f, double *phi, double tol, int max_cycles,
                      double *hist, int *cycles_out)
{
    level_t *L = &H->L[0];
    size_t n = ncell(L);
    memcpy(L->f, f, sizeof(double) * n);
    memcpy(L->phi, phi, sizeof(double) * n);
    if (H->singular) remove_mean(n, L->f);
    double nf = norm2(n, L->f);
    if (cycles_out) *cycles_out = 0;
    if (!isfinite(nf)) return OR_NONFINITE;
    if (nf == 0.0) {
        memset(phi, 0, sizeof(double) * n);
        if (hist) hist[0] = 0.0;
        return OR_OK;
    }
    oracle_residual(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->f, L->phi, L->r);
    double rn = norm2(n, L->r);
    if (hist) hist[0] = rn / nf;
    int status = (rn <= tol * nf) ? OR_OK : OR_NOT_CONVERGED;
    int c = 0;
    while (status == OR_NOT_CONVERGED && c < max_cycles) {
        vcycle(H, 0);
        ++c;
        oracle_residual(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, L->f, L->phi, L->r);
        rn = norm2(n, L->r);
        if (hist) hist[c] = rn / nf;
        if (!isfinite(rn)) { status = OR_NONFINITE; break; }
        if (rn <= tol * nf) status = OR_OK;
    }
    if (H->singular) remove_mean(n, L->phi);
    memcpy(phi, L->phi, sizeof(double) * n);
    if (cycles_out) *cycles_out = c;
    return status;
}

/* Solve A phi = f (homogeneous walls of the mask bc) by V(nu1, nu2) cycles
 * from the initial guess in phi until ||f - A phi|| <= tol ||f|| or
 * max_cycles.  hist (nullable, length max_cycles + 1) receives the relative
 * residual before each cycle and after the last one.  With every wall
 * Neumann, f is taken without its mean and phi is returned with zero mean.
 * Returns 0 converged, 1 not converged, 2 non-finite, 3 bad hierarchy. */
int oracle_solve_bc(int nx, int ny, int nz, double h, const double *beta, int bc,
                    const double *f, double *phi, double tol, int max_cycles, int nu1,
                    int nu2, double *hist, int *cycles)
{
    hier_t H;
    if (build_hier(&H, nx, ny, nz, h, beta, bc, nu1, nu2) != 0) {
        free_hier(&H);
        return OR_BAD;
    }
    int s = run_cycles(&H, f, phi, tol, max_cycles, hist, cycles);
    free_hier(&H);
    return s;
}

/* The solve with every wall Dirichlet. */
int oracle_solve(int nx, int ny, int nz, double h, const double *beta, const double *f,
                 double *phi, double tol, int max_cycles, int nu1, int nu2,
                 double *hist, int *cycles)
{
    return oracle_solve_bc(nx, ny, nz, h, beta, 0, f, phi, tol, max_cycles, nu1, nu2, hist,
                           cycles);
}

/* dL/dbeta_cell += chain rule of the face products for one right-hand side:
 * dL/dbeta_face = (lambda_n - lambda_c)(phi_n - phi_c)/h^2 on inner faces and
 * lambda_c phi_c / h^2 on Dirichlet wall faces, times d beta_face /
 * d beta_cell = 2 beta_other^2 / (beta_c + beta_other)^2 inside and 2 on
 * Dirichlet walls; a Neumann wall face (coefficient 0) contributes nothing. */
void oracle_beta_grad_bc(int nx, int ny, int nz, double h, const double *beta, int bc,
                         const double *phi, const double *lam, double *dbeta)
{
    double ih2 = 1.0 / (h * h);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = cell(i, j, k, nx, ny);
                double b_c = beta[c], pc = phi[c], lc = lam[c];
                double acc = 0.0;
                int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k},
                                {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
                for (int q = 0; q < 6; ++q) {
                    int a = nb[q][0], b = nb[q][1], d = nb[q][2];
                    int inside = a >= 0 && b >= 0 && d >= 0 && a < nx && b < ny && d < nz;
                    if (inside) {
                        size_t o = cell(a, b, d, nx, ny);
                        double g = (lam[o] - lc) * (phi[o] - pc) * ih2;
                        double s = b_c + beta[o];
                        acc += g * 2.0 * beta[o] * beta[o] / (s * s);
                    } else if (!neumann(bc, q)) {
                        acc += 2.0 * lc * pc * ih2;
                    }
                }
                dbeta[c] += acc;
            }
}

void oracle_beta_grad(int nx, int ny, int nz, double h, const double *beta,
                      const double *phi, const double *lam, double *dbeta)
{
    oracle_beta_grad_bc(nx, ny, nz, h, beta, 0, phi, lam, dbeta);
}

/* Adjoint of the solve for one right-hand side: lambda solves A lambda = g
 * (written to lam, which is also dL/df), and dbeta (cell beta gradient) is
 * accumulated.  Returns the solve status of the adjoint solve. */
int oracle_adjoint_bc(int nx, int ny, int nz, double h, const double *beta, int bc,
                      const double *phi, const double *g, double *lam, double *dbeta,
                      double tol, int max_cycles, int *cycles)
{
    size_t n = (size_t)nx * ny * nz;
    memset(lam, 0, sizeof(double) * n);
    if ((bc & 63) == 63) return OR_BAD;   /* singular A: no adjoint of the gauge */
    int s = oracle_solve_bc(nx, ny, nz, h, beta, bc, g, lam, tol, max_cycles, 2, 2, NULL,
                            cycles);
    if (s == OR_NONFINITE || s == OR_BAD) return s;
    oracle_beta_grad_bc(nx, ny, nz, h, beta, bc, phi, lam, dbeta);
    return s;
}

int oracle_adjoint(int nx, int ny, int nz, double h, const double *beta,
                   const double *phi, const double *g, double *lam, double *dbeta,
                   double tol, int max_cycles, int *cycles)
{
    return oracle_adjoint_bc(nx, ny, nz, h, beta, 0, phi, g, lam, dbeta, tol, max_cycles,
                             cycles);
}

/* ------------------------------------------------------------ projection */

/* The velocity constraint around the solve (paper Sec. 1): with face
 * velocities u (x faces, (nz, ny, nx+1)), v (y faces), w (z faces) and a cell
 * source S (nullable = 0), the right-hand side is the discrete divergence
 * minus the source,
 *     f_c = (u_{i+1} - u_i + v_{j+1} - v_j + w_{k+1} - w_k) / h - S_c. */
void oracle_divergence(int nx, int ny, int nz, double h, const double *u, const double *v,
                       const double *w, const double *S, double *f)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double d = (u[xface(i + 1, j, k, nx, ny)] - u[xface(i, j, k, nx, ny)]) +
                           (v[yface(i, j + 1, k, nx, ny)] - v[yface(i, j, k, nx, ny)]) +
                           (w[zface(i, j, k + 1, nx, ny)] - w[zface(i, j, k, nx, ny)]);
                size_t c = cell(i, j, k, nx, ny);
                f[c] = d / h - (S ? S[c] : 0.0);
            }
}

/* Velocity correction after the solve: every face velocity loses the face
 * flux beta_face (phi_high - phi_low) / h, with phi = 0 outside the box and
 * the wall faces' coefficients of the mask bc (Neumann wall faces keep their
 * velocity), so that div(u') = div(u) - A phi. */
void oracle_correct_bc(int nx, int ny, int nz, double h, const double *beta, int bc,
                       const double *phi, double *u, double *v, double *w)
{
    size_t nfx = (size_t)nz * ny * (nx + 1), nfy = (size_t)nz * (ny + 1) * nx,
           nfz = (size_t)(nz + 1) * ny * nx;
    double *bx = (double *)malloc(sizeof(double) * nfx);
    double *by = (double *)malloc(sizeof(double) * nfy);
    double *bz = (double *)malloc(sizeof(double) * nfz);
    oracle_face_beta_bc(nx, ny, nz, beta, bc, bx, by, bz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                size_t q = xface(i, j, k, nx, ny);
                u[q] -= bx[q] * (value_at(phi, i, j, k, nx, ny, nz) -
                                 value_at(phi, i - 1, j, k, nx, ny, nz)) / h;
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t q = yface(i, j, k, nx, ny);
                v[q] -= by[q] * (value_at(phi, i, j, k, nx, ny, nz) -
                                 value_at(phi, i, j - 1, k, nx, ny, nz)) / h;
            }
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t q = zface(i, j, k, nx, ny);
                w[q] -= bz[q] * (value_at(phi, i, j, k, nx, ny, nz) -
                                 value_at(phi, i, j, k - 1, nx, ny, nz)) / h;
            }
    free(bx);
    free(by);
    free(bz);
}

void oracle_correct(int nx, int ny, int nz, double h, const double *beta, const double *phi,
                    double *u, double *v, double *w)
{
    oracle_correct_bc(nx, ny, nz, h, beta, 0, phi, u, v, w);
}

/* ------------------------------------------------------ masked domains */

/* Face coefficients of the domain {mask != 0} inside an (nx, ny, nz) box:
 * between two domain cells the harmonic mean, between a domain cell and a
 * cell outside the domain (or the box wall) 2 beta of the domain cell (a
 * Dirichlet wall), between two outside cells 0. */
void oracle_masked_face_beta(int nx, int ny, int nz, const double *beta, const int *mask,
                             double *bx, double *by, double *bz)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                int a = i > 0 && mask[cell(i - 1, j, k, nx, ny)];
                int b = i < nx && mask[cell(i, j, k, nx, ny)];
                double v = 0.0;
                if (a && b) v = harmonic(beta[cell(i - 1, j, k, nx, ny)], beta[cell(i, j, k, nx, ny)]);
                else if (a) v = 2.0 * beta[cell(i - 1, j, k, nx, ny)];
                else if (b) v = 2.0 * beta[cell(i, j, k, nx, ny)];
                bx[xface(i, j, k, nx, ny)] = v;
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int a = j > 0 && mask[cell(i, j - 1, k, nx, ny)];
                int b = j < ny && mask[cell(i, j, k, nx, ny)];
                double v = 0.0;
                if (a && b) v = harmonic(beta[cell(i, j - 1, k, nx, ny)], beta[cell(i, j, k, nx, ny)]);
                else if (a) v = 2.0 * beta[cell(i, j - 1, k, nx, ny)];
                else if (b) v = 2.0 * beta[cell(i, j, k, nx, ny)];
                by[yface(i, j, k, nx, ny)] = v;
            }
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int a = k > 0 && mask[cell(i, j, k - 1, nx, ny)];
                int b = k < nz && mask[cell(i, j, k, nx, ny)];
                double v = 0.0;
                if (a && b) v = harmonic(beta[cell(i, j, k - 1, nx, ny)], beta[cell(i, j, k, nx, ny)]);
                else if (a) v = 2.0 * beta[cell(i, j, k - 1, nx, ny)];
                else if (b) v = 2.0 * beta[cell(i, j, k, nx, ny)];
                bz[zface(i, j, k, nx, ny)] = v;
            }
}

/* Solve A phi = f on the domain {mask != 0} by conjugate gradients on
 * M = -h^2 A (symmetric positive definite on the domain), phi = 0 outside.
 * Iterates from phi = 0 until ||f - A phi|| <= tol ||f|| over the domain.
 * Returns 0 converged, 1 not converged within maxit, 2 non-finite. */
int oracle_masked_solve(int nx, int ny, int nz, double h, const double *beta, const int *mask,
                        const double *f, double *phi, double tol, int maxit, int *iters)
{
    size_t n = (size_t)nx * ny * nz;
    double *bx = (double *)malloc(sizeof(double) * (size_t)nz * ny * (nx + 1));
    double *by = (double *)malloc(sizeof(double) * (size_t)nz * (ny + 1) * nx);
    double *bz = (double *)malloc(sizeof(double) * (size_t)(nz + 1) * ny * nx);
    double *r = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    oracle_masked_face_beta(nx, ny, nz, beta, mask, bx, by, bz);
    double h2 = h * h, rr = 0.0, ff = 0.0;
    for (size_t c = 0; c < n; ++c) {
        phi[c] = 0.0;
        r[c] = mask[c] ? -h2 * f[c] : 0.0;      /* M phi = -h^2 f */
        p[c] = r[c];
        rr += r[c] * r[c];
    }
    ff = rr;
    int status = 1, it = 0;
    if (!isfinite(ff)) status = 2;
    else if (ff == 0.0) status = 0;
    for (; status == 1 && it < maxit; ++it) {
        if (rr <= tol * tol * ff) { status = 0; break; }
        oracle_apply(nx, ny, nz, h, bx, by, bz, p, q);
        double pq = 0.0;
        for (size_t c = 0; c < n; ++c) {
            q[c] = mask[c] ? -h2 * q[c] : 0.0;
            pq += p[c] * q[c];
        }
        double alpha = rr / pq, rr1 = 0.0;
        for (size_t c = 0; c < n; ++c) {
            phi[c] += alpha * p[c];
            r[c] -= alpha * q[c];
            rr1 += r[c] * r[c];
        }
        if (!isfinite(rr1)) { status = 2; break; }
        double b = rr1 / rr;
        rr = rr1;
        for (size_t c = 0; c < n; ++c) p[c] = r[c] + b * p[c];
    }
    if (status == 1 && rr <= tol * tol * ff) status = 0;
    if (iters) *iters = it;
    free(bx); free(by); free(bz); free(r); free(p); free(q);
    return status;
}

/* ------------------------------------------------------- periodic axes */

/* Axis d (0 = x, 1 = y, 2 = z) is periodic when bit 6 + d of bc is set. */
static int periodic(int bc, int d) { return (bc >> (6 + d)) & 1; }

/* Face coefficients with periodic axes: as oracle_face_beta_bc, except that
 * on a periodic axis the faces 0 and n are the one face between cells n-1
 * and 0 (harmonic mean). */
void oracle_face_beta_periodic(int nx, int ny, int nz, const double *beta, int bc,
                               double *bx, double *by, double *bz)
{
    oracle_face_beta_bc(nx, ny, nz, beta, bc & 63, bx, by, bz);
    if (periodic(bc, 0))
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j) {
                double v = harmonic(beta[cell(nx - 1, j, k, nx, ny)], beta[cell(0, j, k, nx, ny)]);
                bx[xface(0, j, k, nx, ny)] = v;
                bx[xface(nx, j, k, nx, ny)] = v;
            }
    if (periodic(bc, 1))
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) {
                double v = harmonic(beta[cell(i, ny - 1, k, nx, ny)], beta[cell(i, 0, k, nx, ny)]);
                by[yface(i, 0, k, nx, ny)] = v;
                by[yface(i, ny, k, nx, ny)] = v;
            }
    if (periodic(bc, 2))
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double v = harmonic(beta[cell(i, j, nz - 1, nx, ny)], beta[cell(i, j, 0, nx, ny)]);
                bz[zface(i, j, 0, nx, ny)] = v;
                bz[zface(i, j, nz, nx, ny)] = v;
            }
}

/* phi at (i, j, k) with periodic axes wrapped and 0 outside otherwise. */
static double value_wrapped(const double *phi, int i, int j, int k, int nx, int ny, int nz, int bc)
{
    if (periodic(bc, 0)) i = (i + nx) % nx;
    if (periodic(bc, 1)) j = (j + ny) % ny;
    if (periodic(bc, 2)) k = (k + nz) % nz;
    return value_at(phi, i, j, k, nx, ny, nz);
}

/* out = A phi with the faces of oracle_face_beta_periodic and wrapped
 * neighbours on periodic axes. */
void oracle_apply_periodic(int nx, int ny, int nz, double h, const double *bx, const double *by,
                           const double *bz, int bc, const double *phi, double *out)
{
    double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double bw = bx[xface(i, j, k, nx, ny)], be = bx[xface(i + 1, j, k, nx, ny)];
                double bs = by[yface(i, j, k, nx, ny)], bn = by[yface(i, j + 1, k, nx, ny)];
                double bd = bz[zface(i, j, k, nx, ny)], bu = bz[zface(i, j, k + 1, nx, ny)];
                double c = phi[cell(i, j, k, nx, ny)];
                double s = bw * (value_wrapped(phi, i - 1, j, k, nx, ny, nz, bc) - c) +
                           be * (value_wrapped(phi, i + 1, j, k, nx, ny, nz, bc) - c) +
                           bs * (value_wrapped(phi, i, j - 1, k, nx, ny, nz, bc) - c) +
                           bn * (value_wrapped(phi, i, j + 1, k, nx, ny, nz, bc) - c) +
                           bd * (value_wrapped(phi, i, j, k - 1, nx, ny, nz, bc) - c) +
                           bu * (value_wrapped(phi, i, j, k + 1, nx, ny, nz, bc) - c);
                out[cell(i, j, k, nx, ny)] = s * ih2;
            }
}

/* Solve A phi = f with the walls and periodic axes of bc by conjugate
 * gradients on M = -h^2 A.  When A is singular (every axis periodic or with
 * Neumann walls on both ends) f loses its mean first and phi is returned
 * with zero mean.  Returns 0 converged, 1 not converged, 2 non-finite. */
int oracle_periodic_solve(int nx, int ny, int nz, double h, const double *beta, int bc,
                          const double *f, double *phi, double tol, int maxit, int *iters)
{
    size_t n = (size_t)nx * ny * nz;
    double *bx = (double *)malloc(sizeof(double) * (size_t)nz * ny * (nx + 1));
    double *by = (double *)malloc(sizeof(double) * (size_t)nz * (ny + 1) * nx);
    double *bz = (double *)malloc(sizeof(double) * (size_t)(nz + 1) * ny * nx);
    double *r = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    oracle_face_beta_periodic(nx, ny, nz, beta, bc, bx, by, bz);
    int singular = 1;
    for (int d = 0; d < 3; ++d)
        if (!periodic(bc, d) && !(neumann(bc, 2 * d) && neumann(bc, 2 * d + 1))) singular = 0;
    double h2 = h * h, rr = 0.0;
    for (size_t c = 0; c < n; ++c) {
        phi[c] = 0.0;
        r[c] = -h2 * f[c];
    }
    if (singular) remove_mean(n, r);
    for (size_t c = 0; c < n; ++c) {
        p[c] = r[c];
        rr += r[c] * r[c];
    }
    double ff = rr;
    int status = 1, it = 0;
    if (!isfinite(ff)) status = 2;
    else if (ff == 0.0) status = 0;
    for (; status == 1 && it < maxit; ++it) {
        if (rr <= tol * tol * ff) { status = 0; break; }
        oracle_apply_periodic(nx, ny, nz, h, bx, by, bz, bc, p, q);
        double pq = 0.0;
        for (size_t c = 0; c < n; ++c) {
            q[c] *= -h2;
            pq += p[c] * q[c];
        }
        double alpha = rr / pq, rr1 = 0.0;
        for (size_t c = 0; c < n; ++c) {
            phi[c] += alpha * p[c];
            r[c] -= alpha * q[c];
            rr1 += r[c] * r[c];
        }
        if (!isfinite(rr1)) { status = 2; break; }
        double b = rr1 / rr;
        rr = rr1;
        for (size_t c = 0; c < n; ++c) p[c] = r[c] + b * p[c];
    }
    if (status == 1 && rr <= tol * tol * ff) status = 0;
    if (singular) remove_mean(n, phi);
    if (iters) *iters = it;
    free(bx); free(by); free(bz); free(r); free(p); free(q);
    return status;
}

/* ----------------------------------------------- V-cycle-preconditioned CG */

/* One V(nu, nu) cycle from phi = 0 on the right-hand side r: z = V r.
 * sym = 1: post-smoothing sweeps black then red (the symmetric cycle);
 * sym = 0: red then black (the cycle of oracle_solve).  Returns 0, or 3 for
 * a bad hierarchy. */
int oracle_vcycle_apply(int nx, int ny, int nz, double h, const double *beta, int bc, int nu,
                        int sym, const double *r, double *z)
{
    hier_t H;
    if (build_hier(&H, nx, ny, nz, h, beta, bc, nu, nu) != 0) {
        free_hier(&H);
        return OR_BAD;
    }
    H.post_first = sym ? 1 : 0;
    level_t *L = &H.L[0];
    size_t n = ncell(L);
    memcpy(L->f, r, sizeof(double) * n);
    memset(L->phi, 0, sizeof(double) * n);
    vcycle(&H, 0);
    memcpy(z, L->phi, sizeof(double) * n);
    free_hier(&H);
    return OR_OK;
}

/* Solve A phi = f (homogeneous walls of the mask bc, not every wall Neumann)
 * by preconditioned conjugate gradients, in the textbook form for the
 * symmetric positive definite system B x = b with B = -A, b = -f and the
 * preconditioner C = -V (V the symmetric V(nu, nu) cycle from a zero start):
 *   r = b - B x, z = C r, p = z;  repeat: q = B p, alpha = <r, z> / <p, q>,
 *   x += alpha p, r -= alpha q, z = C r, beta = <r, z>_new / <r, z>_old,
 *   p = z + beta p;
 * from the initial guess in phi until ||r|| <= tol ||f|| (||r|| is the
 * recursively updated residual, which equals ||f - A phi|| in exact
 * arithmetic) or maxit iterations.  hist (nullable, maxit + 1) gets ||r|| /
 * ||f|| before the first iteration and after each.  Returns 0 converged,
 * 1 not converged, 2 non-finite, 3 bad hierarchy or every wall Neumann. */
int oracle_pcg_solve(int nx, int ny, int nz, double h, const double *beta, int bc,
                     const double *f, double *phi, double tol, int maxit, int nu,
                     double *hist, int *iters)
{
    if (iters) *iters = 0;
    if ((bc & 63) == 63) return OR_BAD;
    hier_t H;
    if (build_hier(&H, nx, ny, nz, h, beta, bc, nu, nu) != 0) {
        free_hier(&H);
        return OR_BAD;
    }
    H.post_first = 1;
    level_t *L = &H.L[0];
    size_t n = ncell(L);
    double *r = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    double nf = norm2(n, f);
    int status = OR_NOT_CONVERGED, it = 0;
    /* r = b - B x = -f + A x */
    oracle_apply(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, phi, q);
    for (size_t c = 0; c < n; ++c) r[c] = -f[c] + q[c];
    double rn = norm2(n, r);
    if (hist) hist[0] = nf > 0.0 ? rn / nf : 0.0;
    if (!isfinite(nf) || !isfinite(rn)) status = OR_NONFINITE;
    else if (nf == 0.0) {
        memset(phi, 0, sizeof(double) * n);
        status = OR_OK;
    } else if (rn <= tol * nf) status = OR_OK;
    double rz = 0.0;
    while (status == OR_NOT_CONVERGED && it < maxit) {
        /* z = C r = -V r */
        memcpy(L->f, r, sizeof(double) * n);
        memset(L->phi, 0, sizeof(double) * n);
        vcycle(&H, 0);
        double rz1 = 0.0;
        for (size_t c = 0; c < n; ++c) {
            z[c] = -L->phi[c];
            rz1 += r[c] * z[c];
        }
        if (it == 0) memcpy(p, z, sizeof(double) * n);
        else {
            double b = rz1 / rz;
            for (size_t c = 0; c < n; ++c) p[c] = z[c] + b * p[c];
        }
        rz = rz1;
        /* q = B p = -A p */
        oracle_apply(L->nx, L->ny, L->nz, L->h, L->bx, L->by, L->bz, p, q);
        double pq = 0.0;
        for (size_t c = 0; c < n; ++c) {
            q[c] = -q[c];
            pq += p[c] * q[c];
        }
        double alpha = rz / pq;
        for (size_t c = 0; c < n; ++c) {
            phi[c] += alpha * p[c];
            r[c] -= alpha * q[c];
        }
        ++it;
        rn = norm2(n, r);
        if (hist) hist[it] = rn / nf;
        if (!isfinite(rn)) status = OR_NONFINITE;
        else if (rn <= tol * nf) status = OR_OK;
    }
    if (iters) *iters = it;
    free(r); free(z); free(p); free(q);
    free_hier(&H);
    return status;
}
