// common.cuh -- level descriptors, tile bookkeeping and reductions shared by
// the solver's kernels and host driver.
//
// Storage of one (nx, ny, nz) level (any precision T): every array holds
// (nz + 2) * Q elements with row pitch P = round_up(nx + 1, 8) and plane pitch
// Q = P * (ny + 1); the element of logical position (i, j, k) sits at offset
// (k + 1) Q + j P + i.  Device pointers in the descriptors below point at
// logical (0, 0, 0), so position (i, j, k) is ptr[k Q + j P + i] for cell
// arrays and for face arrays alike (x face i between cells i-1 and i, y face j,
// z face k).  Outside the box (i = -1 or nx, j = -1 or ny, k = -1 or nz) the
// solution arrays hold zeros that are never written: the stencil reads the
// homogeneous Dirichlet neighbour value 0 there without a branch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mg.h"

namespace mg {

constexpr int MG_BOTTOM_CELLS = MG_MAX_BOTTOM;  // dense coarsest-level limit

constexpr int kTX = 32;   // tile width  (threads along x)
constexpr int kTY = 8;    // tile height (threads along y)
constexpr int kThreads = kTX * kTY;
constexpr int kSweepZ = 32;   // default planes per CTA of the fused red-black sweep
constexpr int kSweepTY = 8;   // tile height (rows) of the fused sweep: 64 x 8 cells
constexpr int kSweepWarps = kSweepTY + 3;        // row warps + 2 ring-row warps + 1 ring-column warp
constexpr int kSweepThreads = kTX * kSweepWarps;
// The fused sweep indexes a level with 32-bit offsets: levels of at least
// this many elements smooth with single-colour passes instead.
constexpr long long kSweepMaxElems = (1LL << 31) - 1;
constexpr int kColZ = 16;     // planes per thread of the column kernels (norms)

inline __host__ __device__ long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }
// wide: the layout of the boxes of a coupled level, whose guard cells hold
// neighbour values.  The default layout lets the guard at i = nx of one row
// share its element with the guard at i = -1 of the next (and likewise the
// guard rows j = ny and j = -1 of consecutive planes): both are 0 there.  The
// wide layout gives every guard cell of the six faces its own element:
// P >= nx + 2 and Q = P (ny + 2); element (i, j, k) is still at (k+1) Q + j P + i.
inline __host__ __device__ long long pitch_row(int nx, bool wide = false)
{
    return round_up((long long)nx + (wide ? 2 : 1), 8);
}
inline __host__ __device__ long long pitch_plane(int nx, int ny, bool wide = false)
{
    return pitch_row(nx, wide) * (ny + (wide ? 2 : 1));
}
inline __host__ __device__ long long level_elems(int nx, int ny, int nz, bool wide = false)
{
    return pitch_plane(nx, ny, wide) * (nz + 2);
}

// One box at one level, as the cycle kernels see it.
template <class T>
struct Box {
    T *phi;          // solution / correction
    T *phi2;         // second solution buffer (out-of-place sweeps)
    T *f;            // right-hand side
    const T *wx, *wy, *wz;   // face weights beta_face / h^2
    const T *invD;   // 1 / sum of the six weights
    const T *D;      // sum of the six weights (FP64 levels; NULL: summed on the fly)
    const T *ainv;   // coarsest level only: dense A^{-1}, row-major n x n
    T *phic;         // next-coarser level solution (zeroed by restriction)
    T *fc;           // next-coarser level right-hand side
    int nx, ny, nz;
    int P;           // row pitch
    long long Q;     // plane pitch
    int cP;          // coarse row pitch
    long long cQ;    // coarse plane pitch
    int box;         // index of the box in its batch
    int zc;          // planes per CTA of the fused sweep (chosen on the host)
    int par;         // colour of local cell (0,0,0): (sum of the box's lower corner) % 2 on a
                     // coupled level (red = global i+j+k even), else 0
    int rb;          // 1: f, invD and D are colour-split (see split_at); 0: natural layout
    int cpar;        // par of the next-coarser level (its f index when rb)
};

// Element of cell (i, j, k) in a colour-split array (FP64 levels' f, 1/D and
// D): each row keeps its cells of one colour together, red (i + j + k + par
// even) at [0, P/2) and black at [P/2, P), each in x order, so that a pass
// over one colour reads only that colour's sectors.  Guard positions are
// never addressed this way.
__host__ __device__ __forceinline__ long long split_at(int i, int j, int k, int par, int P,
                                                       long long Q)
{
    return (long long)k * Q + (long long)j * P + (((i + j + k + par) & 1) ? (P >> 1) : 0) + (i >> 1);
}

// Colour-split f / invD / D in use: only FP64 levels split (a compile-time
// false for FP32 boxes, so their kernels carry no split arithmetic).
template <class T>
__host__ __device__ __forceinline__ bool split_on(const Box<T> &B)
{
    return sizeof(T) == sizeof(double) && B.rb;
}

// Index of coarse cell (I, J, K) in the next-coarser level's f.
template <class T>
__host__ __device__ __forceinline__ long long cfidx(const Box<T> &B, int I, int J, int K)
{
    return split_on(B) ? split_at(I, J, K, B.cpar, B.cP, B.cQ)
                : (long long)K * B.cQ + (long long)J * B.cP + I;
}

// Index of cell (i, j, k) in the box's f / invD / D arrays.
template <class T>
__host__ __device__ __forceinline__ long long fidx(const Box<T> &B, int i, int j, int k)
{
    return split_on(B) ? split_at(i, j, k, B.par, B.P, B.Q)
                       : (long long)k * B.Q + (long long)j * B.P + i;
}

// Index spaces that kernels tile: all cells, red-black pairs along x
// (ceil(nx/2) per row), the cells of the next-coarser level, pairs along x
// with z cut into chunks of kSweepZ planes (the fused sweep marches in z), or
// cells with z cut into chunks of kColZ planes (one thread per column chunk).
enum TileKind {
    TK_CELL = 0,
    TK_PAIR = 1,
    TK_COARSE = 2,
    TK_SWEEP = 3,
    TK_COLZ = 4,
    TK_FACE = 5,   // positions [0, nx] x [0, ny] x [0, nz] (every stored face)
    TK_CFACE = 6,  // positions of the next-coarser level's faces
    TK_PCOLZ = 7,  // red-black pairs along x, z in chunks of kColZ planes
    TK_NKIND = 8
};

// zc: planes per CTA of the fused sweep (TK_SWEEP only).
inline __host__ __device__ void tile_extent(int kind, int nx, int ny, int nz, int &ex, int &ey,
                                            int &ez, int zc = kSweepZ)
{
    if (kind == TK_PAIR) { ex = (nx + 1) / 2; ey = ny; ez = nz; }
    else if (kind == TK_COARSE) { ex = nx / 2; ey = ny / 2; ez = nz / 2; }
    else if (kind == TK_SWEEP) { ex = (nx + 1) / 2; ey = ny; ez = (nz + zc - 1) / zc; }
    else if (kind == TK_COLZ) { ex = nx; ey = ny; ez = (nz + kColZ - 1) / kColZ; }
    else if (kind == TK_FACE) { ex = nx + 1; ey = ny + 1; ez = nz + 1; }
    else if (kind == TK_CFACE) { ex = nx / 2 + 1; ey = ny / 2 + 1; ez = nz / 2 + 1; }
    else if (kind == TK_PCOLZ) { ex = (nx + 1) / 2; ey = ny; ez = (nz + kColZ - 1) / kColZ; }
    else { ex = nx; ey = ny; ez = nz; }
}

inline __host__ __device__ int tile_rows(int kind) { return kind == TK_SWEEP ? kSweepTY : kTY; }

// A row that does not fill whole warps (ex not a multiple of kTX, as in the
// boxes of a batch with 48 or 96 cells a side) would leave lanes idle in
// every tile, so such index spaces are tiled flat: a CTA takes kTX * rows
// consecutive positions of a plane in row-major order (a warp may span two
// rows).  The fused sweep and the set-up faces keep their 2D tiles.
inline __host__ __device__ bool tile_flat(int kind, int ex)
{
    return kind != TK_SWEEP && kind != TK_FACE && kind != TK_CFACE && ex % kTX != 0;
}

inline __host__ __device__ int tiles_of(int kind, int nx, int ny, int nz, int zc = kSweepZ)
{
    int ex, ey, ez;
    tile_extent(kind, nx, ny, nz, ex, ey, ez, zc);
    const int ty = tile_rows(kind);
    if (tile_flat(kind, ex)) {
        const long long per = (long long)kTX * ty;
        return (int)(((long long)ex * ey + per - 1) / per) * ez;
    }
    return ((ex + kTX - 1) / kTX) * ((ey + ty - 1) / ty) * ez;
}

// A set of boxes launched together (one box, or every box of a batch that is
// active at a level).  tstart[kind] is a device prefix array of nbox + 1 tile
// offsets for each tile kind; one CTA handles one tile.
template <class D>
struct DescSet {
    const D *boxes;
    const int *tstart[TK_NKIND];
    int ntiles[TK_NKIND];
    int nbox;
    int flat;      // bit k: some box of the set tiles kind k flat (tile_flat)
};
template <class T>
using BoxSet = DescSet<Box<T>>;

// One box at one level as the set-up kernels see it (FP64 weights written
// from cell beta or from the finer level; FP32 copies for mixed precision;
// the dense inverse on the coarsest level).
struct SetupBox {
    double *wx, *wy, *wz, *invD, *D;
    double *cwx, *cwy, *cwz;           // next-coarser level's weights (coarsening)
    float *wx32, *wy32, *wz32, *invD32;  // NULL unless mixed precision
    const double *beta;                 // finest level: the box's cell beta
    double inv_h2;
    double *work, *inv64;               // coarsest level: scratch and A^{-1}
    float *inv32;
    int nx, ny, nz, P;
    long long Q;
    int cP;
    long long cQ;
    int zc;                             // unused (tile bookkeeping)
    int bc;                             // wall mask: bit w set = wall w Neumann
    const double *betaL;                // coupled level 0: beta in the level layout, guards
                                        // holding the neighbour box's beta or -1 (no neighbour)
    int par, rb;                        // colour parity; invD and D colour-split (split_at)
    // mixed precision with the coarser FP32 levels averaged in FP32: the
    // next-coarser level's FP32 weights, and w32src = 1 when the bottom
    // inverse assembles from the FP32 weights
    float *cwx32, *cwy32, *cwz32;
    int w32src;
};
typedef DescSet<SetupBox> SetupSet;

// The coarse end of one box's V-cycle, run by a single CTA: levels
// lv[0] (the first level small enough) down to lv[nlev-1] (the coarsest).
// Ghost exchange of a coupled level: copy the src box's cells of a patch
// (extents ex, ey, ez; one of them 1) into the dst box's guard cells (local
// coordinates, guard positions -1 or n).  Box indices refer to the level's
// launch set.
struct ExchRec {
    int dst, src;
    int di, dj, dk;  // patch origin in dst (guard layer)
    int si, sj, sk;  // the same cells in src's local coordinates
    int ex, ey, ez;
};

// The coarsest levels of a coupled level's boxes, solved together: cell c
// of box b is union unknown off[b] + c (c in C order of the box).
struct UnionBottom {
    int n;               // unknowns (<= MG_MAX_BOTTOM)
    int nbox;
    int singular;        // constants in the null space (no Dirichlet wall)
    const int *off;      // [nbox + 1]
    const ExchRec *rec;  // ghost exchange records of the coarsest level
    int nrec;
};

constexpr int kMaxCoarse = 10;
template <class T>
struct CoarseJob {
    int nlev;
    int box;
    Box<T> lv[kMaxCoarse];
    // periodic axes: the level's self-exchange records (copied into the
    // box's own guard cells before every pass and residual), else 0
    const ExchRec *rec[kMaxCoarse];
    int nrec[kMaxCoarse];
};

// Per-box convergence state of a solve, kept on the device so that the
// V-cycle loop can run as a conditional CUDA graph with no host round trip.
struct JudgeState {
    int *status;      // [nbox] mg_status (NOT_CONVERGED while running)
    int *cycles;      // [nbox] cycles (or refinement steps) done
    int *stall;       // [nbox] consecutive cycles without a 10% gain
    double *rel0;     // [nbox] starting relative residual
    double *best;     // [nbox] best relative residual so far
    double *hist;     // [nbox * MG_MAX_HIST] relative residual after each cycle
    int *step;        // [1] cycles run by the loop
    double *tol;      // [1] relative residual target
    int max_cycles;
    int stall_limit;  // cycles without a 10% gain that end the solve (0: no such rule)
};

// Last box b with tstart[b] <= t (tstart ascending, tstart[0] = 0).
__device__ __forceinline__ int find_box(const int *__restrict__ tstart, int nbox, int t)
{
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(tstart + mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Position of this thread inside tile `local` of a box (kind's index space).
struct TilePos {
    int x, y, z;
};
// FLAT = false: the caller knows that no box of its set is tiled flat (the
// set's flat bit for the kind is clear), which keeps the flat decode out of
// the kernel.
template <bool FLAT = true>
__device__ __forceinline__ TilePos tile_pos(int kind, int nx, int ny, int nz, int local,
                                            int zc = kSweepZ)
{
    int ex, ey, ez;
    tile_extent(kind, nx, ny, nz, ex, ey, ez, zc);
    const int rows = tile_rows(kind);
    if (FLAT && tile_flat(kind, ex)) {
        const int per = kTX * rows;
        const int tpp = (int)(((long long)ex * ey + per - 1) / per);   // tiles per plane
        const int q = (local % tpp) * per + (int)threadIdx.y * kTX + (int)threadIdx.x;
        TilePos p;
        p.x = q % ex;
        p.y = q / ex;      // ey or more past the plane's last position: no cell
        p.z = local / tpp;
        return p;
    }
    int ntx = (ex + kTX - 1) / kTX, nty = (ey + rows - 1) / rows;
    int tx = local % ntx;
    local /= ntx;
    int ty = local % nty;
    int tz = local / nty;
    TilePos p;
    p.x = tx * kTX + (int)threadIdx.x;
    p.y = ty * rows + (int)threadIdx.y;
    p.z = tz;
    return p;
}

// Fixed-order block sum of one double per thread (blockDim = kTX x kTY):
// warp shuffles, then warp 0 adds the 8 warp sums in order.  Result valid in
// thread (0, 0).
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double warp_part[kThreads / 32];
    int tid = threadIdx.y * kTX + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) warp_part[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += warp_part[w];
    return s;
}

}  // namespace mg
