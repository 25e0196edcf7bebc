// kernels.cu -- CUDA kernels (sm_103a) of the multigrid Poisson solver.
//
// Operator (the library's reading of the paper's Sec. 1 variable-coefficient
// Poisson equation): with face weights w = beta_face / h^2,
//     (A phi)_c = sum over the 6 faces f of w_f (phi_nbr(f) - phi_c),
// phi_nbr = 0 outside the box (homogeneous Dirichlet wall h/2 from the
// centre, whose face weight carries 2 beta).  A Gauss-Seidel update solves
// row c for phi_c: phi_c = (sum_f w_f phi_nbr - f_c) / sum_f w_f.
//
// Every stencil is a 7-point, HBM-bound pass (no dense contraction, so no
// tensor cores); kernels are written for coalesced row access with the
// guarded level layout described in common.cuh.
#include "kernels.h"

#include <atomic>

namespace mg {

static std::atomic<long long> g_launches{0};
long long launch_counter() { return g_launches.load(std::memory_order_relaxed); }
static inline cudaError_t counted(cudaError_t e)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

// ------------------------------------------------------------ helpers ----

template <class T>
__device__ __forceinline__ T fmadd(T a, T b, T c);
template <>
__device__ __forceinline__ double fmadd<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmadd<float>(float a, float b, float c) { return fmaf(a, b, c); }

// Gauss-Seidel value of cell c from its six neighbours in src.
template <class T>
__device__ __forceinline__ T gs_value(const T *__restrict__ src, const T *__restrict__ f,
                                      const T *__restrict__ invD, const T *__restrict__ wx,
                                      const T *__restrict__ wy, const T *__restrict__ wz,
                                      long long c, int P, long long Q)
{
    T s = wx[c] * src[c - 1];
    s = fmadd(wx[c + 1], src[c + 1], s);
    s = fmadd(wy[c], src[c - P], s);
    s = fmadd(wy[c + P], src[c + P], s);
    s = fmadd(wz[c], src[c - Q], s);
    s = fmadd(wz[c + Q], src[c + Q], s);
    return (s - f[c]) * invD[c];
}

// f_c - (A phi)_c.  The diagonal comes from the stored D when given (FP64
// levels: saves five FP64 adds on GB300's narrow FP64 pipe), else it is
// summed from the six weights.
template <class T>
__device__ __forceinline__ T residual_at(const T *__restrict__ phi, const T *__restrict__ f,
                                         const T *__restrict__ wx, const T *__restrict__ wy,
                                         const T *__restrict__ wz, const T *__restrict__ Dg,
                                         long long c, int P, long long Q)
{
    T a = wx[c], b = wx[c + 1], d = wy[c], e = wy[c + P], g = wz[c], h = wz[c + Q];
    T s = a * phi[c - 1];
    s = fmadd(b, phi[c + 1], s);
    s = fmadd(d, phi[c - P], s);
    s = fmadd(e, phi[c + P], s);
    s = fmadd(g, phi[c - Q], s);
    s = fmadd(h, phi[c + Q], s);
    const T D = Dg ? Dg[c] : ((a + b) + (d + e)) + (g + h);
    return f[c] - fmadd(-D, phi[c], s);
}

template <class T>
struct Vec2;
template <>
struct Vec2<double> { typedef double2 type; };
template <>
struct Vec2<float> { typedef float2 type; };

// ---------------------------------------------- single-colour GS pass ----

template <class T>
__global__ void __launch_bounds__(kThreads) k_rbgs_pass(BoxSet<T> S, const int *__restrict__ active,
                                                        int color)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_PAIR];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const int nx = B.nx, ny = B.ny, nz = B.nz, P = B.P;
    const long long Q = B.Q;
    TilePos p = tile_pos(TK_PAIR, nx, ny, nz, t - ts[b]);
    const int j = p.y, k = p.z;
    const int i = 2 * p.x + ((j + k + color) & 1);
    if (j >= ny || i >= nx) return;
    const long long c = (long long)k * Q + (long long)j * P + i;
    B.phi[c] = gs_value<T>(B.phi, B.f, B.invD, B.wx, B.wy, B.wz, c, P, Q);
}

// -------------------------------------- fused red+black sweep (z-march) ----
//
// dst = black pass of (red pass of src), out of place.  The CTA owns a tile
// of 64 x kTY columns and a chunk of kSweepZ planes; thread (tx, ty) owns the
// cell pair (x0 + 2tx, x0 + 2tx + 1) of row y0 + ty, which holds exactly one
// red and one black cell on every plane.  Marching k upward, step k computes
// the new red values of plane k (own column plus the red cells of a one-cell
// ring around the tile, recomputed here because the neighbouring CTA's values
// are not visible) into a 3-plane shared ring buffer, then the new black
// values of plane k-1 from the red values of planes k-2, k-1, k, and stores
// both cells of the pair for plane k-1.  Reading src and writing dst keeps
// every CTA's inputs unchanged while other CTAs run.
template <class T>
__global__ void __launch_bounds__(kThreads) k_rbgs_sweep(BoxSet<T> S, const int *__restrict__ active,
                                                         int src_is_phi2)
{
    __shared__ T red[3][kTY + 2][2 * kTX + 2];
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_SWEEP];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;  // uniform over the CTA
    const int nx = B.nx, ny = B.ny, nz = B.nz, P = B.P;
    const long long Q = B.Q;
    const T *__restrict__ src = src_is_phi2 ? B.phi2 : B.phi;
    T *__restrict__ dst = src_is_phi2 ? B.phi : B.phi2;
    const T *__restrict__ f = B.f;
    const T *__restrict__ invD = B.invD;
    const T *__restrict__ wx = B.wx;
    const T *__restrict__ wy = B.wy;
    const T *__restrict__ wz = B.wz;

    const int zc = B.zc;
    const TilePos tp = tile_pos(TK_SWEEP, nx, ny, nz, t - ts[b], zc);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = 2 * (tp.x - tx);
    const int y0 = tp.y - ty;
    const int xa = x0 + 2 * tx;
    const int y = y0 + ty;
    const int z0 = tp.z * zc;
    const int z1 = min(z0 + zc, nz);
    const bool rowin = y < ny;

    for (int k = z0 - 1; k <= z1; ++k) {
        const int s0 = (k - z0 + 3) % 3;
        const bool plane_in = k >= 0 && k < nz;
        // (1) red values of plane k: own column
        {
            const int xr = xa + ((y + k) & 1);
            T v = T(0);
            if (plane_in && rowin && xr < nx)
                v = gs_value<T>(src, f, invD, wx, wy, wz, (long long)k * Q + (long long)y * P + xr,
                                P, Q);
            red[s0][ty + 1][xr - x0 + 1] = v;
        }
        // ... and the red cells of the ring, needed by this plane's black cells
        if (k >= z0 && k < z1) {
            if (ty < 2) {
                const int yy = (ty == 0) ? y0 - 1 : y0 + kTY;
                const int xr = x0 + 2 * tx + ((yy + k) & 1);
                T v = T(0);
                if (yy >= 0 && yy < ny && xr < nx)
                    v = gs_value<T>(src, f, invD, wx, wy, wz,
                                    (long long)k * Q + (long long)yy * P + xr, P, Q);
                red[s0][ty == 0 ? 0 : kTY + 1][xr - x0 + 1] = v;
            } else if (ty == 2 && tx < kTY) {
                const int xx = (tx < kTY / 2) ? x0 - 1 : x0 + 2 * kTX;
                const int m = tx % (kTY / 2);
                const int yy = y0 + 2 * m + ((xx + y0 + k) & 1);
                T v = T(0);
                if (xx >= 0 && xx < nx && yy < ny)
                    v = gs_value<T>(src, f, invD, wx, wy, wz,
                                    (long long)k * Q + (long long)yy * P + xx, P, Q);
                red[s0][yy - y0 + 1][xx - x0 + 1] = v;
            }
        }
        __syncthreads();
        // (2) black values of plane k-1, then store the pair of plane k-1
        const int km = k - 1;
        if (km >= z0 && km < z1 && rowin) {
            const int sm = (km - z0 + 3) % 3;
            const int smm = (km - 1 - z0 + 3) % 3;
            const int parm = (y + km) & 1;        // red cell of plane k-1 is xa + parm
            const int xb = xa + (parm ^ 1);
            const int lb = xb - x0 + 1;
            const T rv = red[sm][ty + 1][xa + parm - x0 + 1];
            T bv = T(0);
            if (xb < nx) {
                const long long c = (long long)km * Q + (long long)y * P + xb;
                T s = wx[c] * red[sm][ty + 1][lb - 1];
                s = fmadd(wx[c + 1], red[sm][ty + 1][lb + 1], s);
                s = fmadd(wy[c], red[sm][ty][lb], s);
                s = fmadd(wy[c + P], red[sm][ty + 2][lb], s);
                s = fmadd(wz[c], red[smm][ty + 1][lb], s);
                s = fmadd(wz[c + Q], red[s0][ty + 1][lb], s);
                bv = (s - f[c]) * invD[c];
            }
            const long long c0 = (long long)km * Q + (long long)y * P + xa;
            const T va = parm ? bv : rv;
            const T vb = parm ? rv : bv;
            if (xa + 1 < nx) {
                typename Vec2<T>::type v2;
                v2.x = va;
                v2.y = vb;
                *reinterpret_cast<typename Vec2<T>::type *>(dst + c0) = v2;
            } else if (xa < nx) {
                dst[c0] = va;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------- residual + restriction ----

template <class T>
__global__ void __launch_bounds__(kThreads) k_resid_restrict(BoxSet<T> S, const int *__restrict__ active)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_COARSE];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const int nx = B.nx, ny = B.ny, nz = B.nz, P = B.P;
    const long long Q = B.Q;
    TilePos p = tile_pos(TK_COARSE, nx, ny, nz, t - ts[b]);
    const int I = p.x, J = p.y, K = p.z;
    if (I >= nx / 2 || J >= ny / 2) return;
    T sum = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const long long q = (long long)(2 * K + c) * Q + (long long)(2 * J + bb) * P + 2 * I + a;
                sum += residual_at<T>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, q, P, Q);
            }
    const long long cc = (long long)K * B.cQ + (long long)J * B.cP + I;
    B.fc[cc] = sum * T(0.125);
    B.phic[cc] = T(0);
}

// --------------------------------------------------------- prolongation ----

template <class T>
__global__ void __launch_bounds__(kThreads) k_prolong(BoxSet<T> S, const int *__restrict__ active)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_CELL];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const long long c = (long long)p.z * B.Q + (long long)p.y * B.P + p.x;
    const long long cc = (long long)(p.z >> 1) * B.cQ + (long long)(p.y >> 1) * B.cP + (p.x >> 1);
    B.phi[c] += B.phic[cc];
}

// -------------------------------------------------------- residual field ----

template <class T>
__global__ void __launch_bounds__(kThreads) k_residual_field(BoxSet<T> S)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_CELL];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const long long c = (long long)p.z * B.Q + (long long)p.y * B.P + p.x;
    B.phi2[c] = residual_at<T>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c, B.P, B.Q);
}

// ------------------------------------------------------------- norms ----

template <class T>
__global__ void __launch_bounds__(kThreads) k_norm_partials(BoxSet<T> S, const int *__restrict__ active,
                                                            int mode, double *__restrict__ partials)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_COLZ];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t - ts[b]);
    double v = 0.0;
    if (p.x < B.nx && p.y < B.ny) {
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
        for (int k = z0; k < z1; ++k) {
            const long long c = (long long)k * B.Q + (long long)p.y * B.P + p.x;
            const T r = mode ? B.f[c] : residual_at<T>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c, B.P, B.Q);
            v = fma((double)r, (double)r, v);
        }
    }
    double s = block_sum(v);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[t] = s;
}

// One CTA of 1024 threads per box: thread q adds partials q, q + 1024, ...
// in order, then a fixed shuffle tree and an ordered sum of the 32 warps.
template <class T>
__global__ void __launch_bounds__(1024) k_norm_finish(BoxSet<T> S, const int *__restrict__ active,
                                                      const double *__restrict__ partials,
                                                      double *__restrict__ out,
                                                      double *__restrict__ copy,
                                                      double *__restrict__ inv,
                                                      const double *__restrict__ mult)
{
    __shared__ double wsum[32];
    const int b = blockIdx.x;
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const int *ts = S.tstart[TK_COLZ];
    const int lo = ts[b], hi = ts[b + 1];
    double s = 0.0;
    for (int q = lo + (int)threadIdx.x; q < hi; q += 1024) s += partials[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 32; ++w) tot += wsum[w];
        const double nrm = mult ? sqrt(tot) * mult[B.box] : sqrt(tot);
        out[B.box] = nrm;
        if (copy) copy[B.box] = nrm;
        if (inv) inv[B.box] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    }
}

// ----------------------------------------------------- coarsest level ----

// Grid (nbox, row chunks of 32); 8 warps x 4 rows each.
template <class T>
__global__ void __launch_bounds__(kThreads) k_bottom(BoxSet<T> S, const int *__restrict__ active)
{
    __shared__ T fs[MG_BOTTOM_CELLS];
    const Box<T> &B = S.boxes[blockIdx.x];
    if (active && !active[B.box]) return;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const int n = nx * ny * nz;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    for (int q = tid; q < n; q += kThreads) {
        const int i = q % nx, j = (q / nx) % ny, k = q / (nx * ny);
        fs[q] = B.f[(long long)k * B.Q + (long long)j * B.P + i];
    }
    __syncthreads();
    const int lane = threadIdx.x, warp = threadIdx.y;
    for (int rr = 0; rr < 4; ++rr) {
        const int r = blockIdx.y * 32 + warp * 4 + rr;
        if (r >= n) break;
        const T *row = B.ainv + (long long)r * n;
        T acc = T(0);
        for (int q = lane; q < n; q += 32) acc = fmadd(row[q], fs[q], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const int i = r % nx, j = (r / nx) % ny, k = r / (nx * ny);
            B.phi[(long long)k * B.Q + (long long)j * B.P + i] = acc;
        }
    }
}

// --------------------------------------------- coarse V-cycle in one CTA ----
//
// Levels of a few thousand cells take microseconds of work but a kernel
// launch each; the coarse end of every box's V-cycle therefore runs inside
// one CTA per box, with block barriers between stages: nu1 red/black passes
// and residual + restriction going down, the dense coarsest solve, then
// prolongation and nu2 passes going up.  Same stage definitions as the
// per-level kernels; data stay in global memory (L1/L2 resident).

// FP32: 1024 threads; FP64: 512 (its register footprint is larger)
template <class T>
struct CoarseThreads { static constexpr int value = sizeof(T) == 8 ? 512 : 1024; };

template <class T>
__device__ __forceinline__ void cta_pass(const Box<T> &B, int color)
{
    const int npx = (B.nx + 1) >> 1;
    const int tot = npx * B.ny * B.nz;
    for (int q = threadIdx.x; q < tot; q += CoarseThreads<T>::value) {
        const int p = q % npx;
        const int r = q / npx;
        const int j = r % B.ny, k = r / B.ny;
        const int i = 2 * p + ((j + k + color) & 1);
        if (i >= B.nx) continue;
        const long long c = (long long)k * B.Q + (long long)j * B.P + i;
        B.phi[c] = gs_value<T>(B.phi, B.f, B.invD, B.wx, B.wy, B.wz, c, B.P, B.Q);
    }
}

template <class T>
__device__ __forceinline__ void cta_resid_restrict(const Box<T> &B)
{
    const int cx = B.nx / 2, cy = B.ny / 2, cz = B.nz / 2;
    const int tot = cx * cy * cz;
    for (int q = threadIdx.x; q < tot; q += CoarseThreads<T>::value) {
        const int I = q % cx, r = q / cx;
        const int J = r % cy, K = r / cy;
        T sum = T(0);
        for (int c = 0; c < 2; ++c)
            for (int bb = 0; bb < 2; ++bb)
                for (int a = 0; a < 2; ++a) {
                    const long long g =
                        (long long)(2 * K + c) * B.Q + (long long)(2 * J + bb) * B.P + 2 * I + a;
                    sum += residual_at<T>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, g, B.P, B.Q);
                }
        const long long cc = (long long)K * B.cQ + (long long)J * B.cP + I;
        B.fc[cc] = sum * T(0.125);
        B.phic[cc] = T(0);
    }
}

template <class T>
__device__ __forceinline__ void cta_prolong(const Box<T> &B)
{
    const int tot = B.nx * B.ny * B.nz;
    for (int q = threadIdx.x; q < tot; q += CoarseThreads<T>::value) {
        const int i = q % B.nx, r = q / B.nx;
        const int j = r % B.ny, k = r / B.ny;
        const long long c = (long long)k * B.Q + (long long)j * B.P + i;
        B.phi[c] += B.phic[(long long)(k >> 1) * B.cQ + (long long)(j >> 1) * B.cP + (i >> 1)];
    }
}

template <class T>
__device__ __forceinline__ void cta_bottom(const Box<T> &B, T *fs)
{
    const int nx = B.nx, ny = B.ny, n = nx * ny * B.nz;
    for (int q = threadIdx.x; q < n; q += CoarseThreads<T>::value) {
        const int i = q % nx, j = (q / nx) % ny, k = q / (nx * ny);
        fs[q] = B.f[(long long)k * B.Q + (long long)j * B.P + i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < n; r += CoarseThreads<T>::value / 32) {
        const T *row = B.ainv + (long long)r * n;
        T acc = T(0);
        for (int q = lane; q < n; q += 32) acc = fmadd(row[q], fs[q], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const int i = r % nx, j = (r / nx) % ny, k = r / (nx * ny);
            B.phi[(long long)k * B.Q + (long long)j * B.P + i] = acc;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(CoarseThreads<T>::value) k_coarse_vcycle(const CoarseJob<T> *__restrict__ jobs,
                                                                  const int *__restrict__ active,
                                                                  int nu1, int nu2)
{
    __shared__ CoarseJob<T> J;
    __shared__ T fs[MG_BOTTOM_CELLS];
    {
        const int words = (int)(sizeof(CoarseJob<T>) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(jobs + blockIdx.x);
        int *dst = reinterpret_cast<int *>(&J);
        for (int w = threadIdx.x; w < words; w += CoarseThreads<T>::value) dst[w] = src[w];
    }
    __syncthreads();
    if (active && !active[J.box]) return;  // uniform over the CTA
    const int nl = J.nlev;
    for (int l = 0; l + 1 < nl; ++l) {
        for (int s = 0; s < nu1; ++s) {
            cta_pass<T>(J.lv[l], 0);
            __syncthreads();
            cta_pass<T>(J.lv[l], 1);
            __syncthreads();
        }
        cta_resid_restrict<T>(J.lv[l]);
        __syncthreads();
    }
    cta_bottom<T>(J.lv[nl - 1], fs);
    __syncthreads();
    for (int l = nl - 2; l >= 0; --l) {
        cta_prolong<T>(J.lv[l]);
        __syncthreads();
        for (int s = 0; s < nu2; ++s) {
            cta_pass<T>(J.lv[l], 0);
            __syncthreads();
            cta_pass<T>(J.lv[l], 1);
            __syncthreads();
        }
    }
}

// ------------------------------------------------ mixed refinement step ----
//
// FP64 iterative refinement around FP32 V-cycles, in two passes per step:
//   k_refine_update:   x += c_e e               (in place, pointwise)
//   k_refine_residual: r = f - A64 x;  r32 = float(r) * float(1 / c_r);
//                      partial sums of r32^2 (FP32 per column, FP64 per CTA)
// so ||r|| = c_r * sqrt(sum r32^2).  Only the update, the residual and their
// conversions use the FP64 pipe (GB300 issues 2 FP64 FMA per SM per clock
// against 128 FP32): 11 FP64-pipe operations per cell.

__global__ void __launch_bounds__(kThreads) k_refine_update(BoxSet<double> S64, BoxSet<float> S32,
                                                            const int *__restrict__ active,
                                                            const double *__restrict__ c_e)
{
    const int t = blockIdx.x;
    const int *ts = S64.tstart[TK_CELL];
    const int b = find_box(ts, S64.nbox, t);
    const Box<double> &B = S64.boxes[b];
    const Box<float> &E = S32.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const long long c = (long long)p.z * B.Q + (long long)p.y * B.P + p.x;
    B.phi[c] = fma(c_e[B.box], (double)E.phi[c], B.phi[c]);
}

__global__ void __launch_bounds__(kThreads) k_refine_residual(BoxSet<double> S64, BoxSet<float> S32,
                                                              const int *__restrict__ active,
                                                              const double *__restrict__ c_r_inv,
                                                              double *__restrict__ partials)
{
    const int t = blockIdx.x;
    const int *ts = S64.tstart[TK_COLZ];
    const int b = find_box(ts, S64.nbox, t);
    const Box<double> &B = S64.boxes[b];
    const Box<float> &E = S32.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t - ts[b]);
    float acc = 0.f;
    if (p.x < B.nx && p.y < B.ny) {
        const float cri = (float)c_r_inv[B.box];
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
        for (int k = z0; k < z1; ++k) {
            const long long c = (long long)k * B.Q + (long long)p.y * B.P + p.x;
            const double r = residual_at<double>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c, B.P, B.Q);
            const float r32 = (float)r * cri;
            E.f[c] = r32;
            acc = fmaf(r32, r32, acc);
        }
    }
    double s = block_sum((double)acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[t] = s;
}

// ------------------------------------------------- packing and helpers ----

__global__ void __launch_bounds__(kThreads) k_pack(BoxSet<double> S, const long long *__restrict__ off,
                                                   const double *__restrict__ user, int to_f)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_CELL];
    const int b = find_box(ts, S.nbox, t);
    const Box<double> &B = S.boxes[b];
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const long long u = off[B.box] + ((long long)p.z * B.ny + p.y) * B.nx + p.x;
    const long long c = (long long)p.z * B.Q + (long long)p.y * B.P + p.x;
    (to_f ? B.f : B.phi)[c] = user[u];
}

__global__ void __launch_bounds__(kThreads) k_unpack(BoxSet<double> S, const long long *__restrict__ off,
                                                     double *__restrict__ user,
                                                     const int *__restrict__ side)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_CELL];
    const int b = find_box(ts, S.nbox, t);
    const Box<double> &B = S.boxes[b];
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const long long u = off[B.box] + ((long long)p.z * B.ny + p.y) * B.nx + p.x;
    const long long c = (long long)p.z * B.Q + (long long)p.y * B.P + p.x;
    const double *src = (side && side[B.box]) ? B.phi2 : B.phi;
    user[u] = src[c];
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_zero(BoxSet<T> S, const int *__restrict__ active)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_CELL];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    B.phi[(long long)p.z * B.Q + (long long)p.y * B.P + p.x] = T(0);
}

__global__ void k_scales(int nbox, const int *__restrict__ active, int init,
                         const double *__restrict__ norm, const double *__restrict__ normf,
                         double *__restrict__ se, double *__restrict__ sr, double *__restrict__ sr_inv)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    if (init) {
        const double v = normf[b];
        se[b] = 0.0;
        sr[b] = v;
        sr_inv[b] = v > 0.0 ? 1.0 / v : 0.0;
    } else if (!active || active[b]) {
        const double v = norm[b];
        se[b] = sr[b];
        sr[b] = v;
        sr_inv[b] = v > 0.0 ? 1.0 / v : 0.0;
    }
}

// ------------------------------------------------------------- set-up ----

__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

// Thread per position (i, j, k) in [0, nx] x [0, ny] x [0, nz].
__global__ void k_face_weights(int nx, int ny, int nz, int P, long long Q, double inv_h2,
                               const double *__restrict__ beta, double *__restrict__ wx,
                               double *__restrict__ wy, double *__restrict__ wz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i > nx || j > ny || k > nz) return;
    auto bc = [&](int a, int bb, int c) { return beta[((long long)c * ny + bb) * nx + a]; };
    const long long q = (long long)k * Q + (long long)j * P + i;
    if (j < ny && k < nz) {
        double v = (i == 0) ? 2.0 * bc(0, j, k)
                 : (i == nx) ? 2.0 * bc(nx - 1, j, k) : harmonic(bc(i - 1, j, k), bc(i, j, k));
        wx[q] = v * inv_h2;
    }
    if (i < nx && k < nz) {
        double v = (j == 0) ? 2.0 * bc(i, 0, k)
                 : (j == ny) ? 2.0 * bc(i, ny - 1, k) : harmonic(bc(i, j - 1, k), bc(i, j, k));
        wy[q] = v * inv_h2;
    }
    if (i < nx && j < ny) {
        double v = (k == 0) ? 2.0 * bc(i, j, 0)
                 : (k == nz) ? 2.0 * bc(i, j, nz - 1) : harmonic(bc(i, j, k - 1), bc(i, j, k));
        wz[q] = v * inv_h2;
    }
}

// Coarse position (I, J, K) in [0, cx] x [0, cy] x [0, cz]; coarse face
// beta = mean of the 4 fine faces, coarse h = 2h: w_c = (sum of 4 w) / 16.
__global__ void k_coarsen(int nx, int ny, int nz, int P, long long Q, const double *__restrict__ wx,
                          const double *__restrict__ wy, const double *__restrict__ wz, int cP,
                          long long cQ, double *__restrict__ cwx, double *__restrict__ cwy,
                          double *__restrict__ cwz)
{
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z;
    if (I > cx || J > cy || K > cz) return;
    auto at = [&](int i, int j, int k) { return (long long)k * Q + (long long)j * P + i; };
    const long long cq = (long long)K * cQ + (long long)J * cP + I;
    if (J < cy && K < cz)
        cwx[cq] = (wx[at(2 * I, 2 * J, 2 * K)] + wx[at(2 * I, 2 * J + 1, 2 * K)] +
                   wx[at(2 * I, 2 * J, 2 * K + 1)] + wx[at(2 * I, 2 * J + 1, 2 * K + 1)]) * 0.0625;
    if (I < cx && K < cz)
        cwy[cq] = (wy[at(2 * I, 2 * J, 2 * K)] + wy[at(2 * I + 1, 2 * J, 2 * K)] +
                   wy[at(2 * I, 2 * J, 2 * K + 1)] + wy[at(2 * I + 1, 2 * J, 2 * K + 1)]) * 0.0625;
    if (I < cx && J < cy)
        cwz[cq] = (wz[at(2 * I, 2 * J, 2 * K)] + wz[at(2 * I + 1, 2 * J, 2 * K)] +
                   wz[at(2 * I, 2 * J + 1, 2 * K)] + wz[at(2 * I + 1, 2 * J + 1, 2 * K)]) * 0.0625;
}

__global__ void k_inv_diag(int nx, int ny, int nz, int P, long long Q, const double *__restrict__ wx,
                           const double *__restrict__ wy, const double *__restrict__ wz,
                           double *__restrict__ invD, double *__restrict__ Dout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny || k >= nz) return;
    const long long c = (long long)k * Q + (long long)j * P + i;
    const double D = ((wx[c] + wx[c + 1]) + (wy[c] + wy[c + P])) + (wz[c] + wz[c + Q]);
    invD[c] = 1.0 / D;
    if (Dout) Dout[c] = D;
}

// Positions (i, j, k) in [0, nx] x [0, ny] x [0, nz]: every stored weight.
__global__ void k_round_f32(int nx, int ny, int nz, int P, long long Q, const double *__restrict__ wx,
                            const double *__restrict__ wy, const double *__restrict__ wz,
                            const double *__restrict__ invD, float *__restrict__ wx32,
                            float *__restrict__ wy32, float *__restrict__ wz32,
                            float *__restrict__ invD32)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i > nx || j > ny || k > nz) return;
    const long long q = (long long)k * Q + (long long)j * P + i;
    if (j < ny && k < nz) wx32[q] = (float)wx[q];
    if (i < nx && k < nz) wy32[q] = (float)wy[q];
    if (i < nx && j < ny) wz32[q] = (float)wz[q];
    if (i < nx && j < ny && k < nz) invD32[q] = (float)invD[q];
}

// One CTA: assemble M = -A (symmetric positive definite) densely in work,
// invert it by Gauss-Jordan elimination without pivoting (M is diagonally
// dominant), and write A^{-1} = -M^{-1}.
__global__ void __launch_bounds__(1024) k_bottom_inverse(int nx, int ny, int nz, int P, long long Q,
                                                         const double *__restrict__ wx,
                                                         const double *__restrict__ wy,
                                                         const double *__restrict__ wz,
                                                         double *__restrict__ a,
                                                         double *__restrict__ inv64,
                                                         float *__restrict__ inv32)
{
    __shared__ double col[MG_BOTTOM_CELLS];
    const int n = nx * ny * nz;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (long long e = tid; e < (long long)n * n; e += nt) a[e] = 0.0;
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
        const int i = r % nx, j = (r / nx) % ny, k = r / (nx * ny);
        const long long c = (long long)k * Q + (long long)j * P + i;
        const double ww = wx[c], we = wx[c + 1], ws = wy[c], wn = wy[c + P], wd = wz[c],
                     wu = wz[c + Q];
        a[(long long)r * n + r] = ((ww + we) + (ws + wn)) + (wd + wu);
        if (i > 0) a[(long long)r * n + r - 1] = -ww;
        if (i < nx - 1) a[(long long)r * n + r + 1] = -we;
        if (j > 0) a[(long long)r * n + r - nx] = -ws;
        if (j < ny - 1) a[(long long)r * n + r + nx] = -wn;
        if (k > 0) a[(long long)r * n + r - nx * ny] = -wd;
        if (k < nz - 1) a[(long long)r * n + r + nx * ny] = -wu;
    }
    __syncthreads();
    for (int p = 0; p < n; ++p) {
        for (int i = tid; i < n; i += nt) col[i] = a[(long long)i * n + p];
        __syncthreads();
        const double piv = col[p];
        for (int j = tid; j < n; j += nt) {
            const double v = (j == p) ? 1.0 : a[(long long)p * n + j];
            a[(long long)p * n + j] = v / piv;
        }
        __syncthreads();
        for (int i = warp; i < n; i += nw) {
            if (i == p) continue;
            const double ci = col[i];
            for (int j = lane; j < n; j += 32) {
                const double v = (j == p) ? 0.0 : a[(long long)i * n + j];
                a[(long long)i * n + j] = v - ci * a[(long long)p * n + j];
            }
        }
        __syncthreads();
    }
    for (long long e = tid; e < (long long)n * n; e += nt) {
        const double v = -a[e];
        inv64[e] = v;
        if (inv32) inv32[e] = (float)v;
    }
}

// dbeta += chain of dL/dbeta_face through the harmonic mean (see mg.h).
// Arrays are contiguous (nz, ny, nx).
__global__ void k_beta_grad(int nx, int ny, int nz, double inv_h2, const double *__restrict__ beta,
                            const double *__restrict__ phi, const double *__restrict__ lam,
                            double *__restrict__ dbeta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny || k >= nz) return;
    const long long sx = 1, sy = nx, sz = (long long)nx * ny;
    const long long c = k * sz + j * sy + i;
    const double bc = beta[c], pc = phi[c], lc = lam[c];
    double acc = 0.0;
    auto face = [&](bool inside, long long o) {
        if (inside) {
            const double bo = beta[o];
            const double g = (lam[o] - lc) * (phi[o] - pc) * inv_h2;
            const double s = bc + bo;
            acc += g * (2.0 * bo * bo / (s * s));
        } else {
            acc += 2.0 * lc * pc * inv_h2;
        }
    };
    face(i > 0, c - sx);
    face(i < nx - 1, c + sx);
    face(j > 0, c - sy);
    face(j < ny - 1, c + sy);
    face(k > 0, c - sz);
    face(k < nz - 1, c + sz);
    dbeta[c] += acc;
}

// ----------------------------------------------------------- launchers ----

static inline dim3 block2d() { return dim3(kTX, kTY); }

template <class T>
cudaError_t launch_rbgs_pass(const BoxSet<T> &S, const int *active, int color, cudaStream_t st)
{
    if (S.ntiles[TK_PAIR] == 0) return cudaSuccess;
    k_rbgs_pass<T><<<S.ntiles[TK_PAIR], block2d(), 0, st>>>(S, active, color);
    return counted(cudaGetLastError());
}

template <class T>
int sweep_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rbgs_sweep<T>, kThreads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 4;
    }
    return n > 0 ? n : 1;
}
template int sweep_ctas_per_sm<double>();
template int sweep_ctas_per_sm<float>();

template <class T>
cudaError_t launch_rbgs_sweep(const BoxSet<T> &S, const int *active, int src_is_phi2,
                              cudaStream_t st)
{
    if (S.ntiles[TK_SWEEP] == 0) return cudaSuccess;
    k_rbgs_sweep<T><<<S.ntiles[TK_SWEEP], block2d(), 0, st>>>(S, active, src_is_phi2);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_resid_restrict(const BoxSet<T> &S, const int *active, cudaStream_t st)
{
    if (S.ntiles[TK_COARSE] == 0) return cudaSuccess;
    k_resid_restrict<T><<<S.ntiles[TK_COARSE], block2d(), 0, st>>>(S, active);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_prolong(const BoxSet<T> &S, const int *active, cudaStream_t st)
{
    if (S.ntiles[TK_CELL] == 0) return cudaSuccess;
    k_prolong<T><<<S.ntiles[TK_CELL], block2d(), 0, st>>>(S, active);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_residual_field(const BoxSet<T> &S, cudaStream_t st)
{
    if (S.ntiles[TK_CELL] == 0) return cudaSuccess;
    k_residual_field<T><<<S.ntiles[TK_CELL], block2d(), 0, st>>>(S);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_norm_partials(const BoxSet<T> &S, const int *active, int mode, double *partials,
                                 cudaStream_t st)
{
    if (S.ntiles[TK_COLZ] == 0) return cudaSuccess;
    k_norm_partials<T><<<S.ntiles[TK_COLZ], block2d(), 0, st>>>(S, active, mode, partials);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_norm_finish(const BoxSet<T> &S, const int *active, const double *partials,
                               double *out, double *copy, double *inv, cudaStream_t st,
                               const double *mult)
{
    if (S.nbox == 0) return cudaSuccess;
    k_norm_finish<T><<<S.nbox, 1024, 0, st>>>(S, active, partials, out, copy, inv, mult);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_bottom(const BoxSet<T> &S, const int *active, int max_cells, cudaStream_t st)
{
    if (S.nbox == 0) return cudaSuccess;
    dim3 grid(S.nbox, (max_cells + 31) / 32);
    k_bottom<T><<<grid, block2d(), 0, st>>>(S, active);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_coarse_vcycle(const CoarseJob<T> *jobs, int njobs, const int *active, int nu1,
                                 int nu2, cudaStream_t st)
{
    if (njobs == 0) return cudaSuccess;
    k_coarse_vcycle<T><<<njobs, CoarseThreads<T>::value, 0, st>>>(jobs, active, nu1, nu2);
    return counted(cudaGetLastError());
}

cudaError_t launch_refine_update(const BoxSet<double> &S64, const BoxSet<float> &S32,
                                 const int *active, const double *c_e, cudaStream_t st)
{
    if (S64.ntiles[TK_CELL] == 0) return cudaSuccess;
    k_refine_update<<<S64.ntiles[TK_CELL], block2d(), 0, st>>>(S64, S32, active, c_e);
    return counted(cudaGetLastError());
}

cudaError_t launch_refine_residual(const BoxSet<double> &S64, const BoxSet<float> &S32,
                                   const int *active, const double *c_r_inv, double *partials,
                                   cudaStream_t st)
{
    if (S64.ntiles[TK_COLZ] == 0) return cudaSuccess;
    k_refine_residual<<<S64.ntiles[TK_COLZ], block2d(), 0, st>>>(S64, S32, active, c_r_inv,
                                                                  partials);
    return counted(cudaGetLastError());
}

cudaError_t launch_pack(const BoxSet<double> &S, const long long *off, const double *user,
                        int to_f, cudaStream_t st)
{
    if (S.ntiles[TK_CELL] == 0) return cudaSuccess;
    k_pack<<<S.ntiles[TK_CELL], block2d(), 0, st>>>(S, off, user, to_f);
    return counted(cudaGetLastError());
}

cudaError_t launch_unpack(const BoxSet<double> &S, const long long *off, double *user,
                          const int *side, cudaStream_t st)
{
    if (S.ntiles[TK_CELL] == 0) return cudaSuccess;
    k_unpack<<<S.ntiles[TK_CELL], block2d(), 0, st>>>(S, off, user, side);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_zero(const BoxSet<T> &S, const int *active, cudaStream_t st)
{
    if (S.ntiles[TK_CELL] == 0) return cudaSuccess;
    k_zero<T><<<S.ntiles[TK_CELL], block2d(), 0, st>>>(S, active);
    return counted(cudaGetLastError());
}

cudaError_t launch_scales(int nbox, const int *active, int init, const double *norm,
                          const double *normf, double *se, double *sr, double *sr_inv,
                          cudaStream_t st)
{
    k_scales<<<(nbox + 127) / 128, 128, 0, st>>>(nbox, active, init, norm, normf, se, sr, sr_inv);
    return counted(cudaGetLastError());
}

static inline dim3 grid3(int ex, int ey, int ez)
{
    return dim3((ex + kTX - 1) / kTX, (ey + kTY - 1) / kTY, ez);
}

cudaError_t launch_face_weights(int nx, int ny, int nz, double inv_h2, const double *beta,
                                double *wx, double *wy, double *wz, cudaStream_t st)
{
    k_face_weights<<<grid3(nx + 1, ny + 1, nz + 1), block2d(), 0, st>>>(
        nx, ny, nz, (int)pitch_row(nx), pitch_plane(nx, ny), inv_h2, beta, wx, wy, wz);
    return counted(cudaGetLastError());
}

cudaError_t launch_coarsen(int nx, int ny, int nz, const double *wx, const double *wy,
                           const double *wz, double *cwx, double *cwy, double *cwz, cudaStream_t st)
{
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    k_coarsen<<<grid3(cx + 1, cy + 1, cz + 1), block2d(), 0, st>>>(
        nx, ny, nz, (int)pitch_row(nx), pitch_plane(nx, ny), wx, wy, wz, (int)pitch_row(cx),
        pitch_plane(cx, cy), cwx, cwy, cwz);
    return counted(cudaGetLastError());
}

cudaError_t launch_inv_diag(int nx, int ny, int nz, const double *wx, const double *wy,
                            const double *wz, double *invD, double *D, cudaStream_t st)
{
    k_inv_diag<<<grid3(nx, ny, nz), block2d(), 0, st>>>(nx, ny, nz, (int)pitch_row(nx),
                                                        pitch_plane(nx, ny), wx, wy, wz, invD, D);
    return counted(cudaGetLastError());
}

cudaError_t launch_round_f32(int nx, int ny, int nz, const double *wx, const double *wy,
                             const double *wz, const double *invD, float *wx32, float *wy32,
                             float *wz32, float *invD32, cudaStream_t st)
{
    k_round_f32<<<grid3(nx + 1, ny + 1, nz + 1), block2d(), 0, st>>>(
        nx, ny, nz, (int)pitch_row(nx), pitch_plane(nx, ny), wx, wy, wz, invD, wx32, wy32, wz32,
        invD32);
    return counted(cudaGetLastError());
}

cudaError_t launch_bottom_inverse(int nx, int ny, int nz, const double *wx, const double *wy,
                                  const double *wz, double *work, double *inv64, float *inv32,
                                  cudaStream_t st)
{
    k_bottom_inverse<<<1, 1024, 0, st>>>(nx, ny, nz, (int)pitch_row(nx), pitch_plane(nx, ny), wx,
                                         wy, wz, work, inv64, inv32);
    return counted(cudaGetLastError());
}

cudaError_t launch_beta_grad(int nx, int ny, int nz, double inv_h2, const double *beta,
                             const double *phi, const double *lam, double *dbeta, cudaStream_t st)
{
    k_beta_grad<<<grid3(nx, ny, nz), block2d(), 0, st>>>(nx, ny, nz, inv_h2, beta, phi, lam,
                                                         dbeta);
    return counted(cudaGetLastError());
}

#define MG_INSTANTIATE(T)                                                                        \
    template cudaError_t launch_rbgs_pass<T>(const BoxSet<T> &, const int *, int, cudaStream_t);  \
    template cudaError_t launch_rbgs_sweep<T>(const BoxSet<T> &, const int *, int, cudaStream_t); \
    template cudaError_t launch_resid_restrict<T>(const BoxSet<T> &, const int *, cudaStream_t);  \
    template cudaError_t launch_prolong<T>(const BoxSet<T> &, const int *, cudaStream_t);         \
    template cudaError_t launch_residual_field<T>(const BoxSet<T> &, cudaStream_t);               \
    template cudaError_t launch_norm_partials<T>(const BoxSet<T> &, const int *, int, double *,   \
                                                 cudaStream_t);                                   \
    template cudaError_t launch_norm_finish<T>(const BoxSet<T> &, const int *, const double *,    \
                                               double *, double *, double *, cudaStream_t,        \
                                               const double *);                                   \
    template cudaError_t launch_bottom<T>(const BoxSet<T> &, const int *, int, cudaStream_t);   \
    template cudaError_t launch_zero<T>(const BoxSet<T> &, const int *, cudaStream_t);          \
    template cudaError_t launch_coarse_vcycle<T>(const CoarseJob<T> *, int, const int *, int, int, \
                                                 cudaStream_t);

MG_INSTANTIATE(double)
MG_INSTANTIATE(float)

}  // namespace mg
