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

#include <algorithm>
#include <type_traits>

#include <atomic>
#include <mutex>

namespace mg {

static std::atomic<long long> g_launches{0};
long long launch_counter() { return g_launches.load(std::memory_order_relaxed); }
static inline cudaError_t counted(cudaError_t e)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

// Programmatic dependent launch.  The kernels of the solve loop are launched
// with cudaLaunchAttributeProgrammaticStreamSerialization, so that a kernel's
// CTAs can be scheduled while its predecessor's last CTAs drain (the cycle is
// a chain of many short, dependent launches on the coarse levels); each such
// kernel first waits for the predecessor grid to complete and its writes to
// be visible.  The wait is a no-op in a plain launch.  MG_PDL=0 in the
// environment launches them plainly.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

static bool pdl_enabled()
{
    static const bool on = [] {
        const char *v = getenv("MG_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

template <typename... KArgs, typename... Args>
static cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return counted(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// ------------------------------------------------------------ helpers ----

template <class T>
__device__ __forceinline__ T fmadd(T a, T b, T c);
template <>
__device__ __forceinline__ double fmadd<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmadd<float>(float a, float b, float c) { return fmaf(a, b, c); }

// Gauss-Seidel value of cell c from its six neighbours in src:
// (sum_f w_f src_nbr - f_c) / D_c, with -f_c as the start of the FMA chain
// (six FMAs and one multiply: GB300's FP64 pipe is the narrow resource).
// cf: the cell's element in f and invD (c, or its colour-split position).
template <class T>
__device__ __forceinline__ T gs_sum(const T *__restrict__ src, const T *__restrict__ f,
                                    const T *__restrict__ wx, const T *__restrict__ wy,
                                    const T *__restrict__ wz, long long c, long long cf, int P,
                                    long long Q)
{
    T s = fmadd(wx[c], src[c - 1], -f[cf]);
    s = fmadd(wx[c + 1], src[c + 1], s);
    s = fmadd(wy[c], src[c - P], s);
    s = fmadd(wy[c + P], src[c + P], s);
    s = fmadd(wz[c], src[c - Q], s);
    return fmadd(wz[c + Q], src[c + Q], s);
}

template <class T>
__device__ __forceinline__ T gs_value(const T *__restrict__ src, const T *__restrict__ f,
                                      const T *__restrict__ invD, const T *__restrict__ wx,
                                      const T *__restrict__ wy, const T *__restrict__ wz,
                                      long long c, long long cf, int P, long long Q)
{
    return gs_sum<T>(src, f, wx, wy, wz, c, cf, P, Q) * invD[cf];
}

// f_c - (A phi)_c = f_c + D_c phi_c - sum_f w_f phi_nbr, one FMA chain (seven
// FP64 operations with the stored D).  HAS_D: the diagonal comes from the
// stored D (FP64 levels: saves five FP64 adds on GB300's narrow FP64 pipe),
// else it is summed from the six weights.  It is a template parameter, and
// kernels branch on it once per box, because a run-time choice inside the
// stencil is if-converted and then pays for both sides.
template <class T, bool HAS_D>
__device__ __forceinline__ T residual_at(const T *__restrict__ phi, const T *__restrict__ f,
                                         const T *__restrict__ wx, const T *__restrict__ wy,
                                         const T *__restrict__ wz, const T *__restrict__ Dg,
                                         long long c, long long cf, int P, long long Q)
{
    T a = wx[c], b = wx[c + 1], d = wy[c], e = wy[c + P], g = wz[c], h = wz[c + Q];
    const T D = HAS_D ? Dg[cf] : ((a + b) + (d + e)) + (g + h);
    T s = fmadd(D, phi[c], f[cf]);
    s = fmadd(-a, phi[c - 1], s);
    s = fmadd(-b, phi[c + 1], s);
    s = fmadd(-d, phi[c - P], s);
    s = fmadd(-e, phi[c + P], s);
    s = fmadd(-g, phi[c - Q], s);
    return fmadd(-h, phi[c + Q], s);
}

template <class T>
struct Vec2;
template <>
struct Vec2<double> { typedef double2 type; };
template <>
struct Vec2<float> { typedef float2 type; };

// FP64 <-> FP32 conversions by integer moves of the IEEE 754 fields
// (binary64: sign, 11-bit exponent biased by 1023, 52-bit fraction;
// binary32: sign, 8-bit exponent biased by 127, 23-bit fraction).  GB300
// executes the conversion instructions on its narrow FP64 pipe, where one
// conversion costs as much as an FMA; these use the integer pipe.

// exact widening of a float in FP32's normal range (exponent field 1..254):
// exponent + (1023 - 127), the fraction's top 20 bits in the high word, its
// low 3 bits at the top of the low word
__device__ __forceinline__ double normal_f32_to_f64(float x)
{
    const unsigned b = __float_as_uint(x);
    return __hiloint2double((int)((b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20))),
                            (int)(b << 29));
}

// The conversion instruction for the values the integer path below leaves
// out (zero, subnormal results, overflow, infinity, NaN): a call, so that the
// compiler cannot run it under a predicate for every value, which would put
// one FP64-pipe conversion into each call of f64_to_f32_rn.
__device__ __noinline__ float f64_to_f32_by_cvt(double x) { return __double2float_rn(x); }

// the float nearest to x, ties to even (IEEE round-to-nearest)
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned h = hi & 0x7fffffffu;
    // biased exponent 897..1150: FP32 exponent 1..254 (a round-up out of 254
    // carries into the exponent and gives infinity, as the rounding does)
    if (h - (897u << 20) >= (254u << 20)) return f64_to_f32_by_cvt(x);
    unsigned m = ((h - (896u << 20)) << 3) | (lo >> 29);   // truncated to 23 fraction bits
    const unsigned rest = lo & 0x1fffffffu;                 // the 29 bits dropped
    m += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(m | (hi & 0x80000000u));
}

// 1/d in FP64 without an FP64 division, whose iterations occupy GB300's
// narrow FP64 pipe: Newton-Raphson for the reciprocal (Muller et al.,
// Handbook of Floating-Point Arithmetic, on iterations for 1/d) from an FP32
// seed.  The seed: d's fraction truncated to 23 bits (relative error below
// 2^-23) and its FP32 reciprocal by the approximate instruction (at most one
// FP32 ulp), widened exactly, both by integer moves; then d y0 = 1 - e with
// |e| < 2^-21.9, and one cubic step y = y0 (1 + e + e^2) = (1 - e^3) / d,
// e computed by a fused multiply-add, is within 2^-65 of 1/d before its one
// rounding, hence within one ulp (and nearly always the correctly rounded
// value).  A d outside 2^-125 <= |d| < 2^126 (so that the seed and its
// reciprocal are normal FP32 numbers; d = 0, inf, NaN) takes the division.
__device__ __forceinline__ double rcp64(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned h = hi & 0x7fffffffu;
    if ((h >> 20) - 898u > 250u) return 1.0 / d;   // FP32 exponent of d outside 2..252
    const float f = __uint_as_float((((h - (896u << 20)) << 3) | (lo >> 29)) | (hi & 0x80000000u));
    float s;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(f));
    const double y = normal_f32_to_f64(s);   // s is normal: 2^-126 < |1/f| <= 2^125
    const double e = fma(-d, y, 1.0);
    return fma(fma(e, e, e), y, y);
}

// ---------------------------------------------- single-colour GS pass ----

template <class T>
__global__ void __launch_bounds__(kThreads) k_rbgs_pass(BoxSet<T> S, const int *__restrict__ active,
                                                        int color)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_PAIR];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const int nx = B.nx, ny = B.ny, nz = B.nz, P = B.P;
    const long long Q = B.Q;
    TilePos p = tile_pos(TK_PAIR, nx, ny, nz, t - ts[b]);
    const int j = p.y, k = p.z;
    const int i = 2 * p.x + ((j + k + color + B.par) & 1);
    if (j >= ny || i >= nx) return;
    const long long c = (long long)k * Q + (long long)j * P + i;
    const long long cf =
        split_on(B) ? (long long)k * Q + (long long)j * P + (color ? (P >> 1) : 0) + p.x : c;
    B.phi[c] = gs_value<T>(B.phi, B.f, B.invD, B.wx, B.wy, B.wz, c, cf, P, Q);
}

// One colour out of place: dst = src with the cells of `color` updated (a
// thread per red-black pair along x, which holds one cell of each colour; the
// pair is read and written as one vector, the other cell copied).  The norm
// variant also sums r_c^2 over the updated cells, where
// r_c = D_c (phi_c - phi'_c) = f_c - (A src)_c (phi'_c solves row c) is
// the residual of src at c, formed as D_c src_c - s_c from the update's own
// sum s_c = sum_f w_f src_nbr - f_c (one extra FMA).  Right after a black
// pass the black residuals vanish, so a red pass with partials yields
// ||f - A src||^2 as a by-product (the cycle's convergence norm, taken at the
// start of the next cycle).
template <class T>
__device__ __forceinline__ void oop_pair(const Box<T> &B, int color, int from2, int j, int k,
                                         int x0, bool norm, double &r2)
{
    const int P = B.P;
    const long long Q = B.Q;
    const T *__restrict__ src = from2 ? B.phi2 : B.phi;
    T *__restrict__ dst = from2 ? B.phi : B.phi2;
    typedef typename Vec2<T>::type V2;
    const long long c0 = (long long)k * Q + (long long)j * P + x0;
    V2 pair = *reinterpret_cast<const V2 *>(src + c0);
    const int odd = (j + k + color + B.par) & 1;   // the pair's cell of this colour
    if (x0 + odd < B.nx) {
        const long long c = c0 + odd;
        const long long cf =
            split_on(B) ? (long long)k * Q + (long long)j * P + (color ? (P >> 1) : 0) + (x0 >> 1)
                        : c;
        const T sc = gs_sum<T>(src, B.f, B.wx, B.wy, B.wz, c, cf, P, Q);
        const T nv = sc * B.invD[cf];
        if (norm) {
            const T r = fmadd(B.D[cf], odd ? pair.y : pair.x, -sc);
            r2 = fma((double)r, (double)r, r2);
        }
        if (odd) pair.y = nv;
        else pair.x = nv;
    }
    *reinterpret_cast<V2 *>(dst + c0) = pair;
}

template <class T>
__global__ void __launch_bounds__(kThreads, 8) k_rbgs_pass_oop(BoxSet<T> S,
                                                               const int *__restrict__ active,
                                                               int color, int from2)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_PAIR];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_PAIR, B.nx, B.ny, B.nz, t - ts[b]);
    double unused = 0.0;
    if (p.y < B.ny && 2 * p.x < B.nx) oop_pair(B, color, from2, p.y, p.z, 2 * p.x, false, unused);
}

// The same pass with the residual norm: each thread takes its pair through a
// column of kColZ planes (TK_PCOLZ tiles), so the block reduction of the
// partial sums (FP64 adds and shuffles, costly on GB300's narrow FP64 pipe)
// is paid once per kColZ cells instead of once per cell.
template <class T>
__global__ void __launch_bounds__(kThreads) k_rbgs_pass_oop_norm(BoxSet<T> S,
                                                                    const int *__restrict__ active,
                                                                    int color, int from2,
                                                                    double *__restrict__ partials)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_PCOLZ];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_PCOLZ, B.nx, B.ny, B.nz, t - ts[b]);
    double r2 = 0.0;
    if (p.y < B.ny && 2 * p.x < B.nx) {
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
#pragma unroll 1
        for (int k = z0; k < z1; ++k) oop_pair(B, color, from2, p.y, k, 2 * p.x, true, r2);
    }
    const double sum = block_sum(r2);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[t] = sum;
}

// -------------------------------------- fused red+black sweep (z-march) ----
//
// dst = black pass of (red pass of src), out of place.  The CTA owns a tile
// of 64 x kSweepTY columns and a chunk of zc planes; in row warp ty, lane tx
// owns the cell pair (x0 + 2tx, x0 + 2tx + 1) of row y0 + ty, which holds
// exactly one red and one black cell on every plane.  Marching k upward, step
// k computes the new red values of plane k (own columns, plus the red cells
// of a one-cell ring around the tile, recomputed by three ring warps because
// the neighbouring CTA's values are not visible) into a 4-plane shared ring
// buffer, then the new black values of plane k-1 from the red values of
// planes k-2, k-1, k, and stores both cells of the pair for plane k-1.
// Reading src and writing dst keeps every CTA's inputs unchanged while other
// CTAs run.
//
// Written for few instructions per cell (at 28 bytes a cell in FP32 the sweep
// is issue-bound before it is DRAM-bound): the ring is balanced over
// dedicated warps; every thread precomputes the offsets, shared-memory
// positions and validity of its cells for both colour parities, so a step
// only adds a plane offset; cells outside the box load from a harmless
// address and store 0 instead of branching; the march is unrolled by 4, so
// the ring-buffer slot and the parity are constants in each step; with 4
// slots one barrier per step suffices (a step writes the slot read two steps
// earlier, with a barrier between).  The black operands are loaded one step
// ahead; 56 registers keep 3 CTAs (33 warps) resident per SM.

// A red update's 13 operands and a black update's 7 global ones (its red
// neighbours come from shared memory).  The diagonal is the sum of the six
// face weights the update loads anyway, so its reciprocal is computed
// instead of read: 4 of 28 bytes a cell less in FP32 (the correctly rounded
// FP32 reciprocal), and for FP64 the set-up's rcp64, i.e. the stored 1/D.
template <class T>
struct SweepRed { T sw, se, ss, sn, sd, su, wxa, wxb, wya, wyb, wza, wzb, f; };
template <class T>
struct SweepBlack { T wxa, wxb, wya, wyb, wza, wzb, f; };

__device__ __forceinline__ float rcp_rn(float d) { return __frcp_rn(d); }
__device__ __forceinline__ double rcp_rn(double d) { return rcp64(d); }

// 1 / D from a cell's six face weights, summed in the set-up's order
template <class T>
__device__ __forceinline__ T inv_diag6(T wxa, T wxb, T wya, T wyb, T wza, T wzb)
{
    return rcp_rn(((wxa + wxb) + (wya + wyb)) + (wza + wzb));
}

template <class T>
__device__ __forceinline__ SweepRed<T> sweep_load_red(const T *__restrict__ src, const T *__restrict__ f,
                                          const T *__restrict__ wx,
                                          const T *__restrict__ wy, const T *__restrict__ wz,
                                          int c, int P, int Q)
{
    SweepRed<T> r;
    r.sw = src[c - 1]; r.se = src[c + 1]; r.ss = src[c - P]; r.sn = src[c + P];
    r.sd = src[c - Q]; r.su = src[c + Q];
    r.wxa = wx[c]; r.wxb = wx[c + 1]; r.wya = wy[c]; r.wyb = wy[c + P]; r.wza = wz[c]; r.wzb = wz[c + Q];
    r.f = f[c];
    return r;
}
template <class T>
__device__ __forceinline__ SweepBlack<T> sweep_load_black(const T *__restrict__ f,
                                            const T *__restrict__ wx, const T *__restrict__ wy,
                                            const T *__restrict__ wz, int c, int P, int Q)
{
    SweepBlack<T> b;
    b.wxa = wx[c]; b.wxb = wx[c + 1]; b.wya = wy[c]; b.wyb = wy[c + P]; b.wza = wz[c]; b.wzb = wz[c + Q];
    b.f = f[c];
    return b;
}
template <class T>
__device__ __forceinline__ T sweep_red_value(const SweepRed<T> &r)
{
    T s = fmadd(r.wxa, r.sw, -r.f);
    s = fmadd(r.wxb, r.se, s); s = fmadd(r.wya, r.ss, s); s = fmadd(r.wyb, r.sn, s);
    s = fmadd(r.wza, r.sd, s); s = fmadd(r.wzb, r.su, s);
    return s * inv_diag6(r.wxa, r.wxb, r.wya, r.wyb, r.wza, r.wzb);
}

template <class T>
__global__ void __launch_bounds__(kSweepThreads, sizeof(T) == 4 ? 3 : 1)
k_rbgs_sweep(BoxSet<T> S, const int *__restrict__ active, int src_is_phi2)
{
    pdl_wait();
    constexpr int W = 2 * kTX, SW = W + 2;            // smem row length
    constexpr int SROWS = kSweepTY + 2, SPLANE = SROWS * SW;
    __shared__ T red[4 * SPLANE];   // red values of 4 planes (slot = step % 4)
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_SWEEP];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const int nx = B.nx, ny = B.ny, nz = B.nz, P = B.P;
    const int Q = (int)B.Q;
    const T *__restrict__ src = src_is_phi2 ? B.phi2 : B.phi;
    T *__restrict__ dst = src_is_phi2 ? B.phi : B.phi2;
    const T *__restrict__ f = B.f;
    const T *__restrict__ wx = B.wx;
    const T *__restrict__ wy = B.wy;
    const T *__restrict__ wz = B.wz;
    const int zc = B.zc;
    const TilePos tp = tile_pos(TK_SWEEP, nx, ny, nz, t - ts[b], zc);
    const int lane = threadIdx.x, wid = threadIdx.y;
    const int x0 = 2 * (tp.x - lane), y0 = tp.y - wid;
    const int z0 = tp.z * zc, z1 = min(z0 + zc, nz);
    const int kf = z0 - 1;                            // first step's plane
    const bool own = wid < kSweepTY;
    const bool colw = wid == kSweepTY + 2;
    const int xa = x0 + 2 * lane;

    // this thread's red cell at even (rE) and odd (rO) steps: plane offset 0
    // (the first step's plane), smem position, validity in x and y
    int rE, rO, sE, sO;
    bool vE, vO;
    bool ractive;        // updates a red cell at every step (own) or at steps with k in [z0, z1)
    if (!colw) {
        const int y = own ? y0 + wid : wid == kSweepTY ? y0 - 1 : y0 + kSweepTY;
        const int srow = own ? wid + 1 : wid == kSweepTY ? 0 : kSweepTY + 1;
        const int p0 = (y + kf) & 1;                  // red x parity at the first step
        const bool rowin = y >= 0 && y < ny;
        rE = kf * Q + y * P + xa + p0;
        rO = kf * Q + y * P + xa + (p0 ^ 1);
        sE = srow * SW + 2 * lane + 1 + p0;
        sO = srow * SW + 2 * lane + 1 + (p0 ^ 1);
        vE = rowin && xa + p0 < nx;
        vO = rowin && xa + (p0 ^ 1) < nx;
        ractive = true;
    } else {
        const int xc = lane < kSweepTY / 2 ? x0 - 1 : x0 + W;
        const int ym = y0 + 2 * (lane % (kSweepTY / 2));
        const int q0 = (xc + y0 + kf) & 1;            // red row offset at the first step
        const bool cin = lane < kSweepTY && xc >= 0 && xc < nx;
        rE = kf * Q + (ym + q0) * P + xc;
        rO = kf * Q + (ym + (q0 ^ 1)) * P + xc;
        sE = (ym + q0 - y0 + 1) * SW + xc - x0 + 1;
        sO = (ym + (q0 ^ 1) - y0 + 1) * SW + xc - x0 + 1;
        vE = cin && ym + q0 < ny;
        vO = cin && ym + (q0 ^ 1) < ny;
        ractive = lane < kSweepTY;
    }
    const bool ringonly = !own;
    // own rows: the black cell is the pair's other cell; pair store position
    const int yo = y0 + wid;
    const bool orow = own && yo < ny;
    const int pairo = kf * Q + yo * P + xa;           // pair base at the first step
    const bool full = xa + 1 < nx, half = xa < nx;
    const int srowo = (wid + 1) * SW;
    const int po = (yo + kf) & 1;                     // own rows' p0
    const int cE = srowo + 2 * lane + 1 + po, cO = srowo + 2 * lane + 1 + (po ^ 1);

    // first step's red operands
    SweepBlack<T> bc{};
    // step j of a block of 6 starting at plane kb (j compile-time: slot j % 3,
    // parity j & 1).  Red work at plane k = kb + j, black work at plane k - 1.
    auto step = [&](int kb, int boff, auto J) {
        constexpr int j = decltype(J)::value, s0 = j % 4, sm = (j + 3) % 4, smm = (j + 2) % 4;
        constexpr bool odd = j & 1;
        const int k = kb + j, off = boff + j * Q;
        const bool vc = (odd ? vO : vE) && k >= 0 && k < nz;
        const SweepRed<T> rc = sweep_load_red(src, f, wx, wy, wz, vc ? (odd ? rO : rE) + off : 0, P, Q);
        // this plane's black operands (used at the next step)
        const bool bv_ok = orow && k >= z0 && k < z1 && (odd ? vE : vO);
        const SweepBlack<T> bn = sweep_load_black(f, wx, wy, wz, bv_ok ? (odd ? rE : rO) + off : 0, P, Q);
        if (ractive && (!ringonly || (k >= z0 && k < z1))) {
            const bool v = (odd ? vO : vE) && k >= 0 && k < nz;
            const T val = sweep_red_value(rc);
            red[s0 * SPLANE + (odd ? sO : sE)] = v ? val : T(0);
        }
        __syncthreads();
        const int km = k - 1;
        if (orow && km >= z0) {
            // plane km had parity !odd: its red cell sits at the (odd ? E : O) position
            const int rpos = odd ? cE : cO;           // red cell of plane km
            const int lb = odd ? cO : cE;             // black cell of plane km
            const T rv = red[sm * SPLANE + rpos];
            T s = fmadd(bc.wxa, red[sm * SPLANE + lb - 1], -bc.f);
            s = fmadd(bc.wxb, red[sm * SPLANE + lb + 1], s);
            s = fmadd(bc.wya, red[sm * SPLANE + lb - SW], s);
            s = fmadd(bc.wyb, red[sm * SPLANE + lb + SW], s);
            s = fmadd(bc.wza, red[smm * SPLANE + lb], s);
            s = fmadd(bc.wzb, red[s0 * SPLANE + lb], s);
            const bool bvalid = odd ? vO : vE;        // black cell of plane km
            const T bval =
                bvalid ? s * inv_diag6(bc.wxa, bc.wxb, bc.wya, bc.wyb, bc.wza, bc.wzb) : T(0);
            const bool redfirst = (odd ? po : (po ^ 1)) == 0;  // red is the pair's first cell
            const T va = redfirst ? rv : bval, vb = redfirst ? bval : rv;
            const int c0 = pairo + off - Q;
            if (full) {
                typename Vec2<T>::type v2; v2.x = va; v2.y = vb;
                *reinterpret_cast<typename Vec2<T>::type *>(dst + c0) = v2;
            } else if (half) dst[c0] = va;
        }
        bc = bn;
    };
    for (int kb = kf, boff = 0; kb <= z1; kb += 4, boff += 4 * Q) {
        step(kb, boff, std::integral_constant<int, 0>{});
        if (kb + 1 <= z1) step(kb, boff, std::integral_constant<int, 1>{});
        if (kb + 2 <= z1) step(kb, boff, std::integral_constant<int, 2>{});
        if (kb + 3 <= z1) step(kb, boff, std::integral_constant<int, 3>{});
    }
}

// ------------------------------------------- residual + restriction ----

// One coarse cell per thread, one tile of TK_COARSE: fc = mean over the 8
// children of f - A phi, phic = 0.
template <class T, bool FC>
__device__ __forceinline__ void restrict_tile(const BoxSet<T> &S, const int *__restrict__ active,
                                              int t)
{
    const int *ts = S.tstart[TK_COARSE];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const int nx = B.nx, ny = B.ny, nz = B.nz, P = B.P;
    const long long Q = B.Q;
    TilePos p = tile_pos<FC>(TK_COARSE, nx, ny, nz, t - ts[b]);
    const int I = p.x, J = p.y, K = p.z;
    if (I >= nx / 2 || J >= ny / 2) return;
    auto children = [&](auto has_d) {
        constexpr bool HD = decltype(has_d)::value;
        T sum = T(0);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const long long q =
                        (long long)(2 * K + c) * Q + (long long)(2 * J + bb) * P + 2 * I + a;
                    sum += residual_at<T, HD>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, q,
                                              fidx(B, 2 * I + a, 2 * J + bb, 2 * K + c), P, Q);
                }
        return sum;
    };
    const T sum = B.D ? children(std::true_type{}) : children(std::false_type{});
    const long long cc = (long long)K * B.cQ + (long long)J * B.cP + I;
    B.fc[cfidx(B, I, J, K)] = sum * T(0.125);
    B.phic[cc] = T(0);
}

template <class T, bool FC>
__global__ void __launch_bounds__(kThreads) k_resid_restrict(BoxSet<T> S, const int *__restrict__ active)
{
    pdl_wait();
    restrict_tile<T, FC>(S, active, blockIdx.x);
}

// The red-children restriction of coarse cell (I, J, K); returns the sum of
// the squared red residuals when NORM.
template <class T, bool NORM>
__device__ __forceinline__ T restrict_red_cell(const Box<T> &B, int I, int J, int K)
{
    const int P = B.P;
    const long long Q = B.Q;
    // red children of the 2x2x2 block at (2I, 2J, 2K): (a+b+c+par) even,
    // par the parity of the box's lower corner in the level's index space
    const long long o = (long long)(2 * K) * Q + (long long)(2 * J) * P + 2 * I;
    // colour-split f and D: a red child (i, j, k) of this block sits at
    // element I of row (j, k)'s red half
    const long long of = (long long)(2 * K) * Q + (long long)(2 * J) * P + I;
    T r2 = T(0);
    auto red4 = [&](auto has_d, auto odd) {
        constexpr bool HD = decltype(has_d)::value, OD = decltype(odd)::value;
        const long long c0 = OD ? o + 1 : o, c1 = OD ? o + P : o + P + 1,
                        c2 = OD ? o + Q : o + Q + 1, c3 = OD ? o + Q + P + 1 : o + Q + P;
        const bool sp = split_on(B);
        const long long f0 = sp ? of : c0, f1 = sp ? of + P : c1, f2 = sp ? of + Q : c2,
                        f3 = sp ? of + Q + P : c3;
        const T a0 = residual_at<T, HD>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c0, f0, P, Q);
        const T a1 = residual_at<T, HD>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c1, f1, P, Q);
        const T a2 = residual_at<T, HD>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c2, f2, P, Q);
        const T a3 = residual_at<T, HD>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c3, f3, P, Q);
        if (NORM) r2 = fmadd(a3, a3, fmadd(a2, a2, fmadd(a1, a1, a0 * a0)));
        return ((a0 + a1) + a2) + a3;
    };
    const T sum = B.D ? (B.par ? red4(std::true_type{}, std::true_type{})
                               : red4(std::true_type{}, std::false_type{}))
                      : (B.par ? red4(std::false_type{}, std::true_type{})
                               : red4(std::false_type{}, std::false_type{}));
    const long long cc = (long long)K * B.cQ + (long long)J * B.cP + I;
    B.fc[cfidx(B, I, J, K)] = sum * T(0.125);
    B.phic[cc] = T(0);
    return r2;
}

// After a red-black sweep every black cell satisfies its own equation (its
// residual is rounding-level), so right after smoothing the residual is
// carried by the red cells alone.  This variant restricts the residual of the
// 4 red children of each coarse cell (the black 4 count as zero): half the
// stencil work of k_resid_restrict, the same coarse right-hand side to
// rounding.  Valid only when the last operation on phi was a black pass.
// NORM: also each warp's sum of the squared red residuals into
// partials[t * kThreads / 32 + warp] (hence ||f - A phi||^2 of the smoothed
// iterate, summed per box in fixed order by the caller); no block barrier.
template <class T, bool FC, bool NORM = false>
__device__ __forceinline__ void restrict_red_tile(const BoxSet<T> &S,
                                                  const int *__restrict__ active, int t,
                                                  double *__restrict__ partials = nullptr)
{
    const int *ts = S.tstart[TK_COARSE];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;   // the whole CTA: its box is skipped
    const int nx = B.nx, ny = B.ny, nz = B.nz, P = B.P;
    const long long Q = B.Q;
    TilePos p = tile_pos<FC>(TK_COARSE, nx, ny, nz, t - ts[b]);
    const int I = p.x, J = p.y, K = p.z;
    if (NORM) {
        // the warp's sum in T (for FP32 no FP64 adds on the narrow pipe; an
        // exit test's sum needs no more), widened once
        T r2 = T(0);
        if (I < nx / 2 && J < ny / 2) r2 = restrict_red_cell<T, NORM>(B, I, J, K);
        for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
        const int tid = threadIdx.y * kTX + threadIdx.x;
        if ((tid & 31) == 0) partials[(long long)t * (kThreads / 32) + (tid >> 5)] = (double)r2;
        return;
    }
    if (I >= nx / 2 || J >= ny / 2) return;
    restrict_red_cell<T, NORM>(B, I, J, K);
}

template <class T, bool FC, bool NORM>
__global__ void __launch_bounds__(kThreads) k_resid_restrict_red(BoxSet<T> S,
                                                                 const int *__restrict__ active,
                                                                 double *__restrict__ partials)
{
    pdl_wait();
    restrict_red_tile<T, FC, NORM>(S, active, blockIdx.x, partials);
}

// --------------------------------------------------------- prolongation ----

// One thread per coarse cell: its correction is added to the 8 children (two
// rows of two planes, each child pair one vector store when nx allows).
template <class T, bool FC>
__device__ __forceinline__ void prolong_tile(const BoxSet<T> &S, const int *__restrict__ active,
                                             int t)
{
    const int *ts = S.tstart[TK_COARSE];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos<FC>(TK_COARSE, B.nx, B.ny, B.nz, t - ts[b]);
    const int I = p.x, J = p.y, K = p.z;
    if (I >= B.nx / 2 || J >= B.ny / 2) return;
    const T e = B.phic[(long long)K * B.cQ + (long long)J * B.cP + I];
    const long long o = (long long)(2 * K) * B.Q + (long long)(2 * J) * B.P + 2 * I;
    typedef typename Vec2<T>::type V2;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            V2 *q = reinterpret_cast<V2 *>(B.phi + o + c * B.Q + r * B.P);
            V2 v = *q;
            v.x += e;
            v.y += e;
            *q = v;
        }
}

template <class T, bool FC>
__global__ void __launch_bounds__(kThreads) k_prolong(BoxSet<T> S, const int *__restrict__ active)
{
    pdl_wait();
    prolong_tile<T, FC>(S, active, blockIdx.x);
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
    const long long cf = fidx(B, p.x, p.y, p.z);
    B.phi2[c] = B.D ? residual_at<T, true>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c, cf, B.P, B.Q)
                    : residual_at<T, false>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c, cf, B.P, B.Q);
}

// ------------------------------------------------------------- norms ----

// mode 0: residual of every cell; 1: f; 2: residual of the red cells only
// (right after a red-black sweep), one thread per red-black pair so that no
// lane idles.  Each thread adds a column of kColZ planes.
template <class T>
__global__ void __launch_bounds__(kThreads) k_norm_partials(BoxSet<T> S, const int *__restrict__ active,
                                                            int mode, double *__restrict__ partials)
{
    pdl_wait();
    const int kind = mode == 2 ? TK_PCOLZ : TK_COLZ;
    const int t = blockIdx.x;
    const int *ts = S.tstart[kind];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(kind, B.nx, B.ny, B.nz, t - ts[b]);
    double v = 0.0;
    const int ex = mode == 2 ? (B.nx + 1) / 2 : B.nx;
    auto column = [&](auto has_d) {
        constexpr bool HD = decltype(has_d)::value;
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
        for (int k = z0; k < z1; ++k) {
            const int x = mode == 2 ? 2 * p.x + ((p.y + k + B.par) & 1) : p.x;
            if (x >= B.nx) continue;
            const long long c = (long long)k * B.Q + (long long)p.y * B.P + x;
            const long long cf = fidx(B, x, p.y, k);
            const T r = mode == 1 ? B.f[cf]
                                  : residual_at<T, HD>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c, cf,
                                                       B.P, B.Q);
            v = fma((double)r, (double)r, v);
        }
    };
    if (p.x < ex && p.y < B.ny) {
        if (B.D) column(std::true_type{});
        else column(std::false_type{});
    }
    double s = block_sum(v);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[t] = s;
}

// Max norms for the solve's statistics (FP64 level 0): field 0 max |f|,
// field 1 max |f - A phi| with phi from phi2 for the boxes whose side flag is
// set.  Per TK_COLZ tile, then one CTA per box takes the max over its tiles.
__global__ void __launch_bounds__(kThreads) k_max_partials(BoxSet<double> S,
                                                           const int *__restrict__ side,
                                                           int field, double *__restrict__ partials)
{
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_COLZ];
    const int b = find_box(ts, S.nbox, t);
    const Box<double> &B = S.boxes[b];
    TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t - ts[b]);
    const double *phi = (side && side[B.box]) ? B.phi2 : B.phi;
    double v = 0.0;
    if (p.x < B.nx && p.y < B.ny) {
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
        for (int k = z0; k < z1; ++k) {
            const long long c = (long long)k * B.Q + (long long)p.y * B.P + p.x;
            const long long cf = fidx(B, p.x, p.y, k);
            const double r =
                field == 0 ? B.f[cf]
                           : residual_at<double, true>(phi, B.f, B.wx, B.wy, B.wz, B.D, c, cf,
                                                       B.P, B.Q);
            v = fmax(v, fabs(r));
        }
    }
    __shared__ double wmax[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int tid = threadIdx.y * kTX + threadIdx.x;
    if ((tid & 31) == 0) wmax[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) m = fmax(m, wmax[w]);
        partials[t] = m;
    }
}

__global__ void __launch_bounds__(1024) k_max_finish(BoxSet<double> S,
                                                     const double *__restrict__ partials,
                                                     double *__restrict__ out)
{
    __shared__ double wmax[32];
    const int b = blockIdx.x;
    const Box<double> &B = S.boxes[b];
    const int *ts = S.tstart[TK_COLZ];
    double m = 0.0;
    for (int q = ts[b] + (int)threadIdx.x; q < ts[b + 1]; q += 1024) m = fmax(m, partials[q]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < 32; ++w) r = fmax(r, wmax[w]);
        out[B.box] = r;
    }
}

// One CTA of 1024 threads per box: thread q adds partials q, q + 1024, ...
// in order, then a fixed shuffle tree and an ordered sum of the 32 warps.
template <class T>
__global__ void __launch_bounds__(1024) k_norm_finish(BoxSet<T> S, const int *__restrict__ active,
                                                      const double *__restrict__ partials,
                                                      double *__restrict__ out,
                                                      double *__restrict__ copy,
                                                      double *__restrict__ inv,
                                                      const double *__restrict__ mult,
                                                      const int *__restrict__ ts)
{
    pdl_wait();
    __shared__ double wsum[32];
    const int b = blockIdx.x;
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
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
        fs[q] = B.f[fidx(B, i, j, k)];
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
        const int i = 2 * p + ((j + k + color + B.par) & 1);
        if (i >= B.nx) continue;
        const long long c = (long long)k * B.Q + (long long)j * B.P + i;
        const long long cf =
            split_on(B) ? (long long)k * B.Q + (long long)j * B.P + (color ? (B.P >> 1) : 0) + p
                        : c;
        B.phi[c] = gs_value<T>(B.phi, B.f, B.invD, B.wx, B.wy, B.wz, c, cf, B.P, B.Q);
    }
}

// Periodic axes: fill the box's guard cells from its own opposite faces
// (records whose source is the box itself); the caller synchronises.
template <class T>
__device__ __forceinline__ void cta_exchange(const Box<T> &B, const ExchRec *rec, int nrec)
{
    for (int q = 0; q < nrec; ++q) {
        const ExchRec R = rec[q];
        const int n = R.ex * R.ey * R.ez;
        for (int e = threadIdx.x; e < n; e += CoarseThreads<T>::value) {
            const int a = e % R.ex, r = e / R.ex;
            const int bb = r % R.ey, c = r / R.ey;
            B.phi[(long long)(R.dk + c) * B.Q + (long long)(R.dj + bb) * B.P + R.di + a] =
                B.phi[(long long)(R.sk + c) * B.Q + (long long)(R.sj + bb) * B.P + R.si + a];
        }
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
        auto children = [&](auto has_d) {
            constexpr bool HD = decltype(has_d)::value;
            T sum = T(0);
            for (int c = 0; c < 2; ++c)
                for (int bb = 0; bb < 2; ++bb)
                    for (int a = 0; a < 2; ++a) {
                        const long long g = (long long)(2 * K + c) * B.Q +
                                            (long long)(2 * J + bb) * B.P + 2 * I + a;
                        sum += residual_at<T, HD>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, g,
                                                  fidx(B, 2 * I + a, 2 * J + bb, 2 * K + c),
                                                  B.P, B.Q);
                    }
            return sum;
        };
        const T sum = B.D ? children(std::true_type{}) : children(std::false_type{});
        const long long cc = (long long)K * B.cQ + (long long)J * B.cP + I;
        B.fc[cfidx(B, I, J, K)] = sum * T(0.125);
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
        fs[q] = B.f[fidx(B, i, j, k)];
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
                                                                  int nu1, int nu2, int post_first)
{
    pdl_wait();
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
    auto exch = [&](int l) {
        if (J.nrec[l] == 0) return;
        cta_exchange<T>(J.lv[l], J.rec[l], J.nrec[l]);
        __syncthreads();
    };
    for (int l = 0; l + 1 < nl; ++l) {
        for (int s = 0; s < nu1; ++s) {
            exch(l);
            cta_pass<T>(J.lv[l], 0);
            __syncthreads();
            exch(l);
            cta_pass<T>(J.lv[l], 1);
            __syncthreads();
        }
        exch(l);
        cta_resid_restrict<T>(J.lv[l]);
        __syncthreads();
    }
    cta_bottom<T>(J.lv[nl - 1], fs);
    __syncthreads();
    for (int l = nl - 2; l >= 0; --l) {
        cta_prolong<T>(J.lv[l]);
        __syncthreads();
        for (int s = 0; s < nu2; ++s) {
            exch(l);
            cta_pass<T>(J.lv[l], post_first);
            __syncthreads();
            exch(l);
            cta_pass<T>(J.lv[l], 1 - post_first);
            __syncthreads();
        }
    }
}

// ------------------------------------------------ mixed refinement step ----
//
// FP64 iterative refinement around FP32 V-cycles, in two passes per step:
//   k_refine_update:   x += c_e e, then e = 0   (in place, pointwise)
//   k_refine_residual: r = f - A64 x;  r32 = float(r) * float(1 / c_r);
//                      partial sums of r32^2 (FP32 per column, FP64 per CTA)
// so ||r|| = c_r * sqrt(sum r32^2).  Only the update, the residual and their
// conversions use the FP64 pipe (GB300 issues 2 FP64 FMA per SM per clock
// against 128 FP32): 11 FP64-pipe operations per cell.

__global__ void __launch_bounds__(kThreads) k_refine_update(BoxSet<double> S64, BoxSet<float> S32,
                                                            const int *__restrict__ active,
                                                            const double *__restrict__ c_e)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S64.tstart[TK_CELL];
    const int b = find_box(ts, S64.nbox, t);
    const Box<double> &B = S64.boxes[b];
    const Box<float> &E = S32.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const long long c = (long long)p.z * B.Q + (long long)p.y * B.P + p.x;
    const float e = E.phi[c];
    B.phi[c] = fma(c_e[B.box], (double)e, B.phi[c]);
    E.phi[c] = 0.f;   // the next step's FP32 cycles start from e = 0
}

// X_ZERO: x = 0 (a zero initial guess), so r = f exactly (every product in
// the FMA chain is a signed zero): f is read instead of the stencil formed,
// with the same roundings and sums after it.
template <bool X_ZERO>
__global__ void __launch_bounds__(kThreads) k_refine_residual(BoxSet<double> S64, BoxSet<float> S32,
                                                              const int *__restrict__ active,
                                                              const double *__restrict__ c_r_inv,
                                                              double *__restrict__ partials)
{
    pdl_wait();
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
        auto column = [&](auto has_d) {
            constexpr bool HD = decltype(has_d)::value;
            for (int k = z0; k < z1; ++k) {
                const long long c = (long long)k * B.Q + (long long)p.y * B.P + p.x;
                const long long cf = fidx(B, p.x, p.y, k);
                const double r = X_ZERO ? B.f[cf]
                                        : residual_at<double, HD>(B.phi, B.f, B.wx, B.wy, B.wz,
                                                                  B.D, c, cf, B.P, B.Q);
                const float r32 = (float)r * cri;
                E.f[c] = r32;
                acc = fmaf(r32, r32, acc);
            }
        };
        if (B.D) column(std::true_type{});
        else column(std::false_type{});
    }
    double s = block_sum((double)acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[t] = s;
}

// ----------------------------------------------- on-device convergence ----
//
// The same decision as the host loop, per active box, after each cycle:
// non-finite -> MG_ERR_NONFINITE; rel <= tol -> MG_OK; rel > 1e3 max(rel0,
// tol) -> MG_ERR_DIVERGED; stall_limit cycles in a row without a 10% gain
// over the best (V-cycles: 5; CG, whose residual is not monotone: no such
// rule), or max_cycles reached -> MG_ERR_NOT_CONVERGED.  A decided box is made
// inactive; the loop continues (graph condition 1) while any box is active.
// When the norm is taken at the start of the next cycle (look-ahead), the
// loop starts at step -1: the first call judges nothing (no cycle has run).
__global__ void __launch_bounds__(1024) k_judge(int nbox, const double *__restrict__ norm,
                                                const double *__restrict__ normf,
                                                int *__restrict__ active, JudgeState J,
                                                cudaGraphConditionalHandle handle, int use_handle)
{
    pdl_wait();
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const int c = *J.step + 1;
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
        if (!active[b]) continue;
        if (c == 0) {
            any = 1;
            continue;
        }
        const double rel = norm[b] / normf[b];
        if (c < MG_MAX_HIST) J.hist[(long long)b * MG_MAX_HIST + c] = rel;
        J.cycles[b] = c;
        int st = MG_ERR_NOT_CONVERGED;
        bool done = true;
        if (!isfinite(rel)) st = MG_ERR_NONFINITE;
        else if (rel <= *J.tol) st = MG_OK;
        else if (rel > 1e3 * fmax(J.rel0[b], *J.tol)) st = MG_ERR_DIVERGED;
        else {
            int stall = rel > 0.9 * J.best[b] ? J.stall[b] + 1 : 0;
            J.stall[b] = stall;
            J.best[b] = fmin(J.best[b], rel);
            done = (J.stall_limit > 0 && stall >= J.stall_limit) || c >= J.max_cycles;
        }
        J.status[b] = st;
        if (done) active[b] = 0;
        else any = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *J.step = c;
        if (use_handle) cudaGraphSetConditional(handle, any ? 1u : 0u);
    }
}

// ------------------------------------------------- packing and helpers ----

// The copies between the caller's packed arrays and the level layout, and
// the zeroing of a level's phi, take one thread per cell column of kColZ
// planes (TK_COLZ tiles): kColZ independent loads or stores in flight per
// thread instead of one per one-plane CTA.  partials (f only, or NULL): also
// the CTA's sum of f^2, as k_norm_partials in mode 1 forms it (the column's
// FMAs in plane order, then block_sum), so that ||f|| needs no pass of its own.
__global__ void __launch_bounds__(kThreads) k_pack(BoxSet<double> S, const long long *__restrict__ off,
                                                   const double *__restrict__ user, int to_f,
                                                   double *__restrict__ partials)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_COLZ];
    const int b = find_box(ts, S.nbox, t);
    const Box<double> &B = S.boxes[b];
    TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t - ts[b]);
    double v = 0.0;
    if (p.x < B.nx && p.y < B.ny) {
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
        const long long us = (long long)B.ny * B.nx;
        const double *src = user + off[B.box] + ((long long)z0 * B.ny + p.y) * B.nx + p.x;
#pragma unroll 4
        for (int k = z0; k < z1; ++k, src += us) {
            const double u = *src;
            if (to_f) {
                B.f[fidx(B, p.x, p.y, k)] = u;
                if (partials) v = fma(u, u, v);
            } else {
                B.phi[(long long)k * B.Q + (long long)p.y * B.P + p.x] = u;
            }
        }
    }
    if (partials) {   // uniform over the launch
        const double sum = block_sum(v);
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[t] = sum;
    }
}

__global__ void __launch_bounds__(kThreads) k_unpack(BoxSet<double> S, const long long *__restrict__ off,
                                                     double *__restrict__ user,
                                                     const int *__restrict__ side)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_COLZ];
    const int b = find_box(ts, S.nbox, t);
    const Box<double> &B = S.boxes[b];
    TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
    const long long us = (long long)B.ny * B.nx;
    double *dst = user + off[B.box] + ((long long)z0 * B.ny + p.y) * B.nx + p.x;
    const double *src = ((side && side[B.box]) ? B.phi2 : B.phi) + (long long)z0 * B.Q +
                        (long long)p.y * B.P + p.x;
#pragma unroll 4
    for (int k = z0; k < z1; ++k, dst += us, src += B.Q) *dst = *src;
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_zero(BoxSet<T> S, const int *__restrict__ active)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_COLZ];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
    T *dst = B.phi + (long long)z0 * B.Q + (long long)p.y * B.P + p.x;
#pragma unroll 4
    for (int k = z0; k < z1; ++k, dst += B.Q) *dst = T(0);
}

__global__ void k_scales(int nbox, const int *__restrict__ active, int init,
                         const double *__restrict__ norm, const double *__restrict__ normf,
                         double *__restrict__ se, double *__restrict__ sr, double *__restrict__ sr_inv)
{
    pdl_wait();
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

// First stage of the inner exit test's sums: chunk c of the set (chunk
// c - cstart[b] of box b, cstart the per-box chunk prefix) sums the per-warp
// partials of its kInnerChunk restriction tiles in fixed order.
__global__ void __launch_bounds__(256) k_inner_sum(BoxSet<float> S, const int *__restrict__ active32,
                                                   const int *__restrict__ cstart,
                                                   int chunk_tiles,
                                                   const double *__restrict__ partials,
                                                   double *__restrict__ chunks)
{
    pdl_wait();
    __shared__ double wsum[8];
    const int c = blockIdx.x;
    const int b = find_box(cstart, S.nbox, c);
    if (!active32[S.boxes[b].box]) return;   // the whole CTA
    const int *ts = S.tstart[TK_COARSE];
    constexpr int W = kThreads / 32;   // partial sums per tile of the restriction
    const int t0 = ts[b] + (c - cstart[b]) * chunk_tiles;
    const int t1 = min(t0 + chunk_tiles, ts[b + 1]);
    double v = 0.0;
    for (long long q = (long long)t0 * W + threadIdx.x; q < (long long)t1 * W; q += 256)
        v += partials[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += wsum[w];
        chunks[c] = tot;
    }
}

// Exit test of the inner FP32 cycles of a refinement step (mixed precision,
// adaptive inner cycles).  The step solves A e = r32 with r32 = r_k / se
// (||r_k|| = sr, so ||r32|| = sr / se); after its update x + se e the FP64
// residual is se times the inner residual r32 - A e, up to FP32 rounding.
// Per box still in the inner cycles: ||r32 - A e|| of the just smoothed
// iterate (the red-children restriction's sums, per box and in fixed order:
// its chunk sums) against max(tol ||f|| / 2, floor_rel sr) / se: at or below
// it the update is expected to meet tol, or the step has gained the factor
// floor_rel, and the box leaves the inner cycles of this step (active32 = 0).
// floor_rel: the most one step asks of FP32 arithmetic.  One CTA per box;
// coupled (the boxes of a level solved as one domain, whose norms and scales
// are the domain's): one CTA, one decision for every box.
__global__ void __launch_bounds__(1024) k_inner_judge(BoxSet<float> S, int *__restrict__ active32,
                                                      const int *__restrict__ cstart,
                                                      const double *__restrict__ chunks,
                                                      const double *__restrict__ se,
                                                      const double *__restrict__ sr,
                                                      const double *__restrict__ normf,
                                                      const double *__restrict__ tol,
                                                      double floor_rel, int coupled)
{
    pdl_wait();
    __shared__ double wsum[32];
    const int b = blockIdx.x;
    const int id = S.boxes[b].box;
    if (!active32[id]) return;   // the whole CTA
    const int lo = coupled ? cstart[0] : cstart[b], hi = coupled ? cstart[S.nbox] : cstart[b + 1];
    double v = 0.0;
    for (int q = lo + threadIdx.x; q < hi; q += 1024) v += chunks[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 32; ++w) tot += wsum[w];
        const double e = se[id];
        const double target =
            e > 0.0 ? fmax(0.5 * tol[0] * normf[id], floor_rel * sr[id]) / e : 0.0;
        if (!(sqrt(tot) > target)) {
            if (coupled)
                for (int q = 0; q < S.nbox; ++q) active32[S.boxes[q].box] = 0;
            else
                active32[id] = 0;
        }
    }
}

// Start of a refinement step's inner cycles: the inner flags are a copy of
// the step's; with a loop handle (inner cycles as a graph WHILE node) also
// the cycle counter to 0 and the loop condition to 1.  One CTA.
__global__ void __launch_bounds__(256) k_inner_begin(int nbox, const int *__restrict__ src,
                                                     int *__restrict__ dst, int *__restrict__ count,
                                                     cudaGraphConditionalHandle handle,
                                                     int use_handle)
{
    pdl_wait();
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) dst[b] = src[b];
    if (threadIdx.x == 0) {
        *count = 0;
        if (use_handle) cudaGraphSetConditional(handle, 1u);
    }
}

// End of one inner cycle in the WHILE form: the loop goes on while some box
// is still in the inner cycles and fewer than max_cycles have run (the
// counter bounds the loop whatever the flags say); count[1] sums the cycles
// of the whole solve.  One CTA.
__global__ void __launch_bounds__(256) k_inner_end(int nbox, const int *__restrict__ flags,
                                                   int *__restrict__ count, int max_cycles,
                                                   cudaGraphConditionalHandle handle)
{
    pdl_wait();
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < nbox; b += blockDim.x)
        if (flags[b]) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int c = count[0] + 1;
        count[0] = c;
        count[1] += 1;   // the solve's total, for the launch count
        cudaGraphSetConditional(handle, (any && c < max_cycles) ? 1u : 0u);
    }
}

cudaError_t launch_inner_begin(int nbox, const int *src, int *dst, int *count,
                               cudaGraphConditionalHandle handle, int use_handle, cudaStream_t st)
{
    return pdl_launch(k_inner_begin, dim3(1), dim3(256), 0, st, nbox, src, dst, count, handle,
                      use_handle);
}

cudaError_t launch_inner_end(int nbox, const int *flags, int *count, int max_cycles,
                             cudaGraphConditionalHandle handle, cudaStream_t st)
{
    return pdl_launch(k_inner_end, dim3(1), dim3(256), 0, st, nbox, flags, count, max_cycles,
                      handle);
}

// ------------------------------------------------------------- set-up ----
//
// Each set-up step is a per-position device function, called by a one-box
// kernel (the single-stage entry points) and by a set kernel that covers
// every box of a level in one launch (the solver).

// weight of a face between cells with coefficients a and b: the harmonic mean
// 2 a b / (a + b) times 1/h^2, given cb = (2 / h^2) b (the upper cell's
// factor, shared by the three faces below it), the quotient taken through
// rcp64 (within a few ulp of the correctly rounded quotient)
__device__ __forceinline__ double harmonic_w(double a, double b, double cb)
{
    return (a * cb) * rcp64(a + b);
}

// Wall w (0..5 = x-, x+, y-, y+, z-, z+) is Neumann when bit w of the mask is
// set: its faces carry no flux (weight 0); otherwise it is a Dirichlet wall
// h/2 from the cell centre (2 beta of the cell).
__device__ __forceinline__ double wall_beta(int bcm, int w, double b)
{
    return ((bcm >> w) & 1) ? 0.0 : 2.0 * b;
}

// Face weights at position (i, j, k) in [0, nx] x [0, ny] x [0, nz]: harmonic
// mean of the two cells' beta (a wall face: wall_beta) over h^2; with W32
// (mixed precision's finest level) also their FP32 roundings, the values
// the rounding step would write (a compile-time choice: a run-time test
// would cost the FP64-bound FP64 path its predicated conversions).
template <bool W32>
__device__ __forceinline__ void face_weights_at(int nx, int ny, int nz, int P, long long Q,
                                                double inv_h2, int bcm,
                                                const double *__restrict__ beta, double *wx,
                                                double *wy, double *wz, int i, int j, int k,
                                                float *wx32 = nullptr, float *wy32 = nullptr,
                                                float *wz32 = nullptr)
{
    auto bc = [&](int a, int bb, int c) { return beta[((long long)c * ny + bb) * nx + a]; };
    const long long q = (long long)k * Q + (long long)j * P + i;
    // cell (i, j, k) is the upper cell of all three faces at this position
    // (every inner face lies below a cell of the box)
    const double b = (i < nx && j < ny && k < nz) ? bc(i, j, k) : 0.0;
    const double cb = (2.0 * inv_h2) * b;
    if (j < ny && k < nz) {
        const double v = (i == 0) ? wall_beta(bcm, 0, bc(0, j, k)) * inv_h2
                       : (i == nx) ? wall_beta(bcm, 1, bc(nx - 1, j, k)) * inv_h2
                                   : harmonic_w(bc(i - 1, j, k), b, cb);
        wx[q] = v;
        if (W32) wx32[q] = f64_to_f32_rn(v);
    }
    if (i < nx && k < nz) {
        const double v = (j == 0) ? wall_beta(bcm, 2, bc(i, 0, k)) * inv_h2
                       : (j == ny) ? wall_beta(bcm, 3, bc(i, ny - 1, k)) * inv_h2
                                   : harmonic_w(bc(i, j - 1, k), b, cb);
        wy[q] = v;
        if (W32) wy32[q] = f64_to_f32_rn(v);
    }
    if (i < nx && j < ny) {
        const double v = (k == 0) ? wall_beta(bcm, 4, bc(i, j, 0)) * inv_h2
                       : (k == nz) ? wall_beta(bcm, 5, bc(i, j, nz - 1)) * inv_h2
                                   : harmonic_w(bc(i, j, k - 1), b, cb);
        wz[q] = v;
        if (W32) wz32[q] = f64_to_f32_rn(v);
    }
}

// Face weights of a coupled level's box from beta in the level layout (bl),
// whose guard cells hold the neighbouring box's beta across an interface or
// -1 on the union's boundary: an interface face takes the harmonic mean like
// any inner face (the neighbour computes the same value), a boundary face is
// a Dirichlet wall (2 beta).
__device__ __forceinline__ void face_weights_level_at(int nx, int ny, int nz, int P, long long Q,
                                                      double inv_h2, int bcm,
                                                      const double *__restrict__ bl, double *wx,
                                                      double *wy, double *wz, int i, int j, int k)
{
    const long long q = (long long)k * Q + (long long)j * P + i;
    // a below / left of the face, b = bl[q] above / right (the same cell for
    // all three faces); lo/hi: the walls on either side of axis d (their
    // Dirichlet or Neumann condition from bcm)
    const double b = bl[q];
    const double cb = (2.0 * inv_h2) * b;
    auto face = [&](double a, int d) {
        if (a < 0.0) return wall_beta(bcm, 2 * d, b) * inv_h2;
        if (b < 0.0) return wall_beta(bcm, 2 * d + 1, a) * inv_h2;
        return harmonic_w(a, b, cb);
    };
    if (j < ny && k < nz) wx[q] = face(bl[q - 1], 0);
    if (i < nx && k < nz) wy[q] = face(bl[q - P], 1);
    if (i < nx && j < ny) wz[q] = face(bl[q - Q], 2);
}

// Coarse position (I, J, K) in [0, cx] x [0, cy] x [0, cz]; coarse face
// beta = mean of the 4 fine faces, coarse h = 2h: w_c = (sum of 4 w) / 16.
template <class T>
__device__ __forceinline__ void coarsen_at(int nx, int ny, int nz, int P, long long Q,
                                           const T *__restrict__ wx, const T *__restrict__ wy,
                                           const T *__restrict__ wz, int cP, long long cQ,
                                           T *cwx, T *cwy, T *cwz, int I, int J, int K)
{
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    auto at = [&](int i, int j, int k) { return (long long)k * Q + (long long)j * P + i; };
    const long long cq = (long long)K * cQ + (long long)J * cP + I;
    const T q = T(0.0625);
    if (J < cy && K < cz)
        cwx[cq] = (wx[at(2 * I, 2 * J, 2 * K)] + wx[at(2 * I, 2 * J + 1, 2 * K)] +
                   wx[at(2 * I, 2 * J, 2 * K + 1)] + wx[at(2 * I, 2 * J + 1, 2 * K + 1)]) * q;
    if (I < cx && K < cz)
        cwy[cq] = (wy[at(2 * I, 2 * J, 2 * K)] + wy[at(2 * I + 1, 2 * J, 2 * K)] +
                   wy[at(2 * I, 2 * J, 2 * K + 1)] + wy[at(2 * I + 1, 2 * J, 2 * K + 1)]) * q;
    if (I < cx && J < cy)
        cwz[cq] = (wz[at(2 * I, 2 * J, 2 * K)] + wz[at(2 * I + 1, 2 * J, 2 * K)] +
                   wz[at(2 * I, 2 * J + 1, 2 * K)] + wz[at(2 * I + 1, 2 * J + 1, 2 * K)]) * q;
}

// ---- mixed precision's coarser FP32 levels, averaged in FP32
//
// Only the finest level's FP32 weights (the rounded FP64 ones) and the
// coarser FP32 levels are read by mixed precision's cycles: the coarser
// levels are averaged from the finer FP32 weights (coarsen_at<float>) and
// take their FP32 1/D from their own weights, with no FP64 coarse level.

// FP32 1/D of cell c from the level's FP32 weights.
__device__ __forceinline__ void inv_diag32_at(int P, long long Q, const float *__restrict__ wx,
                                              const float *__restrict__ wy,
                                              const float *__restrict__ wz, float *invD,
                                              long long c)
{
    invD[c] = 1.0f / (((wx[c] + wx[c + 1]) + (wy[c] + wy[c + P])) + (wz[c] + wz[c + Q]));
}

template <bool W32 = false>
__device__ __forceinline__ void inv_diag_at(int P, long long Q, const double *__restrict__ wx,
                                            const double *__restrict__ wy,
                                            const double *__restrict__ wz, double *invD,
                                            double *Dout, long long c, long long cf,
                                            float *invD32 = nullptr)
{
    const double D = ((wx[c] + wx[c + 1]) + (wy[c] + wy[c + P])) + (wz[c] + wz[c + Q]);
    if (invD) invD[cf] = rcp64(D);  // NULL: mixed precision, whose FP64 levels never smooth
    if (Dout) Dout[cf] = D;
    // mixed precision's finest level (no FP64 1/D): the FP32 1/D the
    // rounding step would write
    if (W32) invD32[c] = 1.0f / f64_to_f32_rn(D);
}

// Every stored weight (and the inverse diagonal) at position (i, j, k) in
// [0, nx] x [0, ny] x [0, nz], rounded to FP32 (the FP32 copies are in the
// natural layout; the FP64 invD and D are colour-split when rb).  Without an
// FP64 invD the FP32 one is the FP32 reciprocal of the rounded D.
__device__ __forceinline__ void round_at(int nx, int ny, int nz, int P, long long Q,
                                         const double *__restrict__ wx,
                                         const double *__restrict__ wy,
                                         const double *__restrict__ wz,
                                         const double *__restrict__ invD, float *wx32,
                                         float *wy32, float *wz32, float *invD32, int i, int j,
                                         int k, int rb = 0, int par = 0,
                                         const double *__restrict__ D = nullptr)
{
    const long long q = (long long)k * Q + (long long)j * P + i;
    if (j < ny && k < nz) wx32[q] = f64_to_f32_rn(wx[q]);
    if (i < nx && k < nz) wy32[q] = f64_to_f32_rn(wy[q]);
    if (i < nx && j < ny) wz32[q] = f64_to_f32_rn(wz[q]);
    if (i < nx && j < ny && k < nz) {
        const long long cf = rb ? split_at(i, j, k, par, P, Q) : q;
        invD32[q] = invD ? f64_to_f32_rn(invD[cf]) : 1.0f / f64_to_f32_rn(D[cf]);
    }
}

// The calling CTA assembles M = -A (symmetric positive definite) densely in
// `a`, inverts it by Gauss-Jordan elimination without pivoting (M is
// diagonally dominant, or symmetric positive definite after the shift below)
// and writes A^{-1} = -M^{-1} (FP64, and FP32 if inv32).  When every wall is
// Neumann (`singular`), M is only semi-definite with the constants as null
// space; c 1 1^T with c = trace(M) / n^2 is added, which makes it positive
// definite: applied to r it gives a solution of M x = r - mean(r) (the
// constant part of r, which no solution can match, is dropped), and the
// zero-mean one when r has zero mean.
// Storage of the symmetric matrix M being inverted.  Only entries (i, j)
// with i <= j are stored, written or read.  Full: row-major n x n (global
// scratch, any n; the lower triangle is left alone).  Packed: the upper
// triangle row by row, n (n + 1) / 2 entries (shared memory when it fits;
// row i holds (i, i..n-1) from i n - i (i - 1) / 2 on).
template <class R, bool PACKED>
struct SymStore {
    R *a;
    int n;
    __device__ __forceinline__ long long size() const
    {
        return PACKED ? (long long)n * (n + 1) / 2 : (long long)n * n;
    }
    // entry (i, i); entry (i, j), j >= i, is row(i)[j - i]
    __device__ __forceinline__ R *row(int i) const
    {
        return a + (PACKED ? (long long)i * n - (long long)i * (i - 1) / 2 : (long long)i * n + i);
    }
    __device__ __forceinline__ R &operator()(int i, int j) const { return row(i)[j - i]; }
};

// Packed FP64 / FP32 matrices up to this size are inverted in shared memory
// (n <= 225 in FP64, n <= 319 in FP32).
constexpr int kPackedBottomBytes = 200 * 1024;

// The upper triangle of the block of M = -A of one box, rows and columns
// from `at` on (the box's cells in C order): diagonal = sum of the six
// weights, -w to each later neighbour inside the box (the earlier ones are
// the mirrors).  Called by every thread of the CTA.
template <class S, class W>
__device__ __forceinline__ void assemble_box_block(int nx, int ny, int nz, int P, long long Q,
                                                   const W *__restrict__ wx,
                                                   const W *__restrict__ wy,
                                                   const W *__restrict__ wz, S a, int at)
{
    using R = typename std::remove_reference<decltype(*a.a)>::type;
    const int m = nx * ny * nz;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const int i = r % nx, j = (r / nx) % ny, k = r / (nx * ny);
        const long long c = (long long)k * Q + (long long)j * P + i;
        const W ww = wx[c], we = wx[c + 1], ws = wy[c], wn = wy[c + P], wd = wz[c],
                wu = wz[c + Q];
        R *row = a.row(at + r);
        row[0] = (R)(((ww + we) + (ws + wn)) + (wd + wu));
        if (i < nx - 1) row[1] = (R)-we;
        if (j < ny - 1) row[nx] = (R)-wn;
        if (k < nz - 1) row[nx * ny] = (R)-wu;
    }
}

template <class R, class S>
__device__ __forceinline__ void gauss_jordan_cta(S a, int n, bool singular, double *inv64,
                                                 float *inv32, R *col);

// The coarsest level's inverse in precision R (double: A^{-1} to inv64 and
// its rounding to inv32; float, when no FP64 inverse is wanted: inv32 only).
// a: the matrix storage (SymStore of R, n = the box's cells); col: 2n of R
// (shared memory).
template <class R, class S, class W>
__device__ __forceinline__ void bottom_inverse_cta(int nx, int ny, int nz, int P, long long Q,
                                                   const W *__restrict__ wx,
                                                   const W *__restrict__ wy,
                                                   const W *__restrict__ wz, bool singular,
                                                   S a, double *inv64, float *inv32, R *col)
{
    for (long long e = threadIdx.x; e < a.size(); e += blockDim.x) a.a[e] = R(0);
    __syncthreads();
    assemble_box_block(nx, ny, nz, P, Q, wx, wy, wz, a, 0);
    __syncthreads();
    gauss_jordan_cta(a, a.n, singular, inv64, inv32, col);
}

// In-place Gauss-Jordan inverse of M (symmetric positive definite; with
// `singular` first shifted by c 1 1^T as described above), written as
// A^{-1} = -M^{-1} to inv64 and/or inv32 (either may be NULL).  Pivots are
// taken in order, without exchanges (M is diagonally dominant or positive
// definite), and only the upper triangle is kept: after pivots 0..p an entry
// with exactly one index <= p is the negative of its mirror and every other
// entry equals its mirror, so the lower triangle follows from the upper one
// and each pivot costs n^2/2 updates instead of n^2 (the FP64 pipe of the
// single SM that inverts a box is the limit once the matrix sits in shared
// memory).  a: SymStore of R; col: 2n of R.
template <class R, class S>
__device__ __forceinline__ void gauss_jordan_cta(S a, int n, bool singular, double *inv64,
                                                 float *inv32, R *col)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    R *rowv = col + n;
    if (singular) {
        if (tid == 0) {
            R tr = R(0);
            for (int r = 0; r < n; ++r) tr += a(r, r);
            col[0] = tr / ((R)n * (R)n);
        }
        __syncthreads();
        const R shift = col[0];
        __syncthreads();
        for (long long e = tid; e < a.size(); e += nt) a.a[e] += shift;
        __syncthreads();
    }
    for (int p = 0; p < n; ++p) {
        // column p (the entries below the diagonal mirror those of row p)
        for (int i = tid; i < n; i += nt) col[i] = i <= p ? a(i, p) : a(p, i);
        __syncthreads();
        const R ip = R(1) / col[p];
        // new row p: a_pj / a_pp (a_pj for j < p is minus its stored mirror)
        for (int j = tid; j < n; j += nt)
            rowv[j] = j == p ? ip : (j > p ? a(p, j) : -a(j, p)) * ip;
        __syncthreads();
        for (int i = warp; i < n; i += nw) {
            const R ci = col[i];
            R *ar = a.row(i);
            for (int j = i + lane; j < n; j += 32) {
                if (i == p) ar[j - i] = rowv[j];             // row p (j >= p; j = p: 1 / a_pp)
                else if (j == p) ar[j - i] = -ci * ip;       // column p above the diagonal
                else ar[j - i] -= ci * rowv[j];
            }
        }
        __syncthreads();
    }
    for (long long e = tid; e < (long long)n * n; e += nt) {
        const int i = (int)(e / n), j = (int)(e % n);
        const double v = -(double)(i <= j ? a(i, j) : a(j, i));
        if (inv64) inv64[e] = v;
        if (inv32) inv32[e] = (float)v;
    }
}

// ---- one box (single-stage entry points): grid over positions

__global__ void k_face_weights(int nx, int ny, int nz, int P, long long Q, double inv_h2,
                               int bcm, const double *__restrict__ beta, double *__restrict__ wx,
                               double *__restrict__ wy, double *__restrict__ wz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i > nx || j > ny || k > nz) return;
    face_weights_at<false>(nx, ny, nz, P, Q, inv_h2, bcm, beta, wx, wy, wz, i, j, k);
}

__global__ void k_coarsen(int nx, int ny, int nz, int P, long long Q, const double *__restrict__ wx,
                          const double *__restrict__ wy, const double *__restrict__ wz, int cP,
                          long long cQ, double *__restrict__ cwx, double *__restrict__ cwy,
                          double *__restrict__ cwz)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z;
    if (I > nx / 2 || J > ny / 2 || K > nz / 2) return;
    coarsen_at(nx, ny, nz, P, Q, wx, wy, wz, cP, cQ, cwx, cwy, cwz, I, J, K);
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
    inv_diag_at(P, Q, wx, wy, wz, invD, Dout, c, c);
}

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
    round_at(nx, ny, nz, P, Q, wx, wy, wz, invD, wx32, wy32, wz32, invD32, i, j, k);
}

__global__ void __launch_bounds__(1024) k_bottom_inverse(int nx, int ny, int nz, int P, long long Q,
                                                         const double *__restrict__ wx,
                                                         const double *__restrict__ wy,
                                                         const double *__restrict__ wz,
                                                         int singular, double *__restrict__ a,
                                                         double *__restrict__ inv64,
                                                         float *__restrict__ inv32, int packed)
{
    __shared__ double col[2 * MG_BOTTOM_CELLS];
    extern __shared__ __align__(16) unsigned char bottom_packed[];
    const int n = nx * ny * nz;
    if (packed)
        bottom_inverse_cta<double>(nx, ny, nz, P, Q, wx, wy, wz, singular != 0,
                                   SymStore<double, true>{reinterpret_cast<double *>(bottom_packed), n},
                                   inv64, inv32, col);
    else
        bottom_inverse_cta<double>(nx, ny, nz, P, Q, wx, wy, wz, singular != 0,
                                   SymStore<double, false>{a, n}, inv64, inv32, col);
}

// ---- every box of a level in one launch (the solver's set-up)

__host__ __device__ constexpr int setup_kind(int step)
{
    return (step == 1 || step == 9) ? TK_CFACE
         : (step == 2 || step == 6 || step == 8) ? TK_CELL : TK_FACE;
}

// One set-up step at one position of box B (see k_setup for the steps).
template <int step>
__device__ __forceinline__ void setup_step(const SetupBox &B, const TilePos &p)
{
    if constexpr (step == 0)
        face_weights_at<false>(B.nx, B.ny, B.nz, B.P, B.Q, B.inv_h2, B.bc, B.beta, B.wx, B.wy,
                               B.wz, p.x, p.y, p.z);
    else if constexpr (step == 5)
        face_weights_at<true>(B.nx, B.ny, B.nz, B.P, B.Q, B.inv_h2, B.bc, B.beta, B.wx, B.wy,
                              B.wz, p.x, p.y, p.z, B.wx32, B.wy32, B.wz32);
    else if constexpr (step == 1)
        coarsen_at<double>(B.nx, B.ny, B.nz, B.P, B.Q, B.wx, B.wy, B.wz, B.cP, B.cQ, B.cwx,
                           B.cwy, B.cwz, p.x, p.y, p.z);
    else if constexpr (step == 2)
        inv_diag_at(B.P, B.Q, B.wx, B.wy, B.wz, B.invD, B.D,
                    (long long)p.z * B.Q + (long long)p.y * B.P + p.x,
                    B.rb ? split_at(p.x, p.y, p.z, B.par, B.P, B.Q)
                         : (long long)p.z * B.Q + (long long)p.y * B.P + p.x);
    else if constexpr (step == 6)
        inv_diag_at<true>(B.P, B.Q, B.wx, B.wy, B.wz, nullptr, B.D,
                          (long long)p.z * B.Q + (long long)p.y * B.P + p.x,
                          B.rb ? split_at(p.x, p.y, p.z, B.par, B.P, B.Q)
                               : (long long)p.z * B.Q + (long long)p.y * B.P + p.x,
                          B.invD32);
    else if constexpr (step == 4)
        face_weights_level_at(B.nx, B.ny, B.nz, B.P, B.Q, B.inv_h2, B.bc, B.betaL, B.wx, B.wy,
                              B.wz, p.x, p.y, p.z);
    else if constexpr (step == 8)
        inv_diag32_at(B.P, B.Q, B.wx32, B.wy32, B.wz32, B.invD32,
                      (long long)p.z * B.Q + (long long)p.y * B.P + p.x);
    else if constexpr (step == 9)
        coarsen_at<float>(B.nx, B.ny, B.nz, B.P, B.Q, B.wx32, B.wy32, B.wz32, B.cP, B.cQ,
                          B.cwx32, B.cwy32, B.cwz32, p.x, p.y, p.z);
    else
        round_at(B.nx, B.ny, B.nz, B.P, B.Q, B.wx, B.wy, B.wz, B.invD, B.wx32, B.wy32, B.wz32,
                 B.invD32, p.x, p.y, p.z, B.rb, B.par, B.D);
}

// step 0 faces (TK_FACE), 1 coarsen (TK_CFACE), 2 diagonal (TK_CELL),
// 3 FP32 copies (TK_FACE), 4 faces of a coupled level from betaL (TK_FACE),
// 5 faces with their FP32 copies (TK_FACE), 6 diagonal with the FP32 1/D
// (TK_CELL): 5 and 6 take the place of 0, 2 and 3 on mixed precision's
// finest level; 8 FP32 1/D (TK_CELL) and 9 FP32 coarsening (TK_CFACE) set
// up its coarser FP32 levels from the finer FP32 ones.  The step is a
// template argument: a run-time index into the set's tstart array
// (a kernel parameter) would make every thread copy the set to local memory.
template <int STEP>
__global__ void __launch_bounds__(kThreads) k_setup(SetupSet S, int t0)
{
    constexpr int kind = setup_kind(STEP);
    const int t = blockIdx.x + t0;
    const int *ts = S.tstart[kind];
    const int b = find_box(ts, S.nbox, t);
    const SetupBox &B = S.boxes[b];
    const TilePos p = tile_pos(kind, B.nx, B.ny, B.nz, t - ts[b]);
    int ex, ey, ez;
    tile_extent(kind, B.nx, B.ny, B.nz, ex, ey, ez);
    if (p.x >= ex || p.y >= ey) return;
    setup_step<STEP>(B, p);
}

// One CTA per box: the coarsest level's dense inverse, in FP64 when an FP64
// inverse is wanted, else (mixed precision, whose FP64 levels never solve)
// in FP32 straight away; a matrix whose packed upper triangle fits in the
// launch's dynamic shared memory (packed_bytes, at most kPackedBottomBytes)
// is inverted there, a larger one in the box's global scratch.
__global__ void __launch_bounds__(1024) k_setup_bottom(SetupSet S, int packed_bytes)
{
    __shared__ double col[2 * MG_BOTTOM_CELLS];
    extern __shared__ __align__(16) unsigned char bottom_packed[];
    const SetupBox &B = S.boxes[blockIdx.x];
    const bool singular = (B.bc & 63) == 63;
    const int n = B.nx * B.ny * B.nz;
    const long long tri = (long long)n * (n + 1) / 2;
    if (B.w32src) {
        // coarser FP32 levels averaged in FP32: assembled from their weights
        float *colf = reinterpret_cast<float *>(col);
        if (tri * (long long)sizeof(float) <= packed_bytes)
            bottom_inverse_cta<float>(
                B.nx, B.ny, B.nz, B.P, B.Q, B.wx32, B.wy32, B.wz32, singular,
                SymStore<float, true>{reinterpret_cast<float *>(bottom_packed), n}, nullptr,
                B.inv32, colf);
        else
            bottom_inverse_cta<float>(B.nx, B.ny, B.nz, B.P, B.Q, B.wx32, B.wy32, B.wz32,
                                      singular,
                                      SymStore<float, false>{reinterpret_cast<float *>(B.work), n},
                                      nullptr, B.inv32, colf);
    } else if (B.inv64) {
        if (tri * (long long)sizeof(double) <= packed_bytes)
            bottom_inverse_cta<double>(
                B.nx, B.ny, B.nz, B.P, B.Q, B.wx, B.wy, B.wz, singular,
                SymStore<double, true>{reinterpret_cast<double *>(bottom_packed), n}, B.inv64,
                B.inv32, col);
        else
            bottom_inverse_cta<double>(B.nx, B.ny, B.nz, B.P, B.Q, B.wx, B.wy, B.wz, singular,
                                       SymStore<double, false>{B.work, n}, B.inv64, B.inv32, col);
    } else {
        float *colf = reinterpret_cast<float *>(col);
        if (tri * (long long)sizeof(float) <= packed_bytes)
            bottom_inverse_cta<float>(
                B.nx, B.ny, B.nz, B.P, B.Q, B.wx, B.wy, B.wz, singular,
                SymStore<float, true>{reinterpret_cast<float *>(bottom_packed), n}, nullptr,
                B.inv32, colf);
        else
            bottom_inverse_cta<float>(B.nx, B.ny, B.nz, B.P, B.Q, B.wx, B.wy, B.wz, singular,
                                      SymStore<float, false>{reinterpret_cast<float *>(B.work), n},
                                      nullptr, B.inv32, colf);
    }
}

// ----------------------------------------------------- projection steps ----
//
// The velocity constraint around the solve (the equation of a MAESTRO step
// enforces it): f = div(u) - S from face velocities, and after the solve
// u -= beta_face grad(phi) on every face (phi = 0 outside, wall faces with
// doubled beta), so that div(u) = S.  beta_face / h = w h with the stored
// level weights w = beta_face / h^2.  Velocity and cell arrays are in their
// natural C layouts: u (nz, ny, nx+1), v (nz, ny+1, nx), w (nz+1, ny, nx).

__global__ void k_project_rhs(int nx, int ny, int nz, double inv_h, const double *__restrict__ u,
                              const double *__restrict__ v, const double *__restrict__ w,
                              const double *__restrict__ S, double *__restrict__ f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny || k >= nz) return;
    const long long ux = ((long long)k * ny + j) * (nx + 1) + i;
    const long long vy = ((long long)k * (ny + 1) + j) * nx + i;
    const long long wz = ((long long)k * ny + j) * nx + i;
    const long long c = wz;
    const double d = (u[ux + 1] - u[ux]) + (v[vy + nx] - v[vy]) + (w[wz + (long long)nx * ny] - w[wz]);
    f[c] = d * inv_h - (S ? S[c] : 0.0);
}

__global__ void k_project_correct(int nx, int ny, int nz, int P, long long Q, double h,
                                  const double *__restrict__ wx, const double *__restrict__ wy,
                                  const double *__restrict__ wzf, const double *__restrict__ phi,
                                  double *__restrict__ u, double *__restrict__ v,
                                  double *__restrict__ w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i > nx || j > ny || k > nz) return;
    auto ph = [&](int a, int b, int c) -> double {
        if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) return 0.0;
        return phi[((long long)c * ny + b) * nx + a];
    };
    const long long q = (long long)k * Q + (long long)j * P + i;
    if (j < ny && k < nz)
        u[((long long)k * ny + j) * (nx + 1) + i] -= wx[q] * h * (ph(i, j, k) - ph(i - 1, j, k));
    if (i < nx && k < nz)
        v[((long long)k * (ny + 1) + j) * nx + i] -= wy[q] * h * (ph(i, j, k) - ph(i, j - 1, k));
    if (i < nx && j < ny)
        w[((long long)k * ny + j) * nx + i] -= wzf[q] * h * (ph(i, j, k) - ph(i, j, k - 1));
}

// dbeta += chain of dL/dbeta_face through the harmonic mean (see mg.h); a
// Neumann wall face (bit w of bcm) has no coefficient and adds nothing.
// Arrays are contiguous (nz, ny, nx).
__global__ void k_beta_grad(int nx, int ny, int nz, double inv_h2, int bcm,
                            const double *__restrict__ beta, const double *__restrict__ phi,
                            const double *__restrict__ lam, double *__restrict__ dbeta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny || k >= nz) return;
    const long long sx = 1, sy = nx, sz = (long long)nx * ny;
    const long long c = k * sz + j * sy + i;
    const double bc = beta[c], pc = phi[c], lc = lam[c];
    double acc = 0.0;
    auto face = [&](bool inside, long long o, int w) {
        if (inside) {
            const double bo = beta[o];
            const double g = (lam[o] - lc) * (phi[o] - pc) * inv_h2;
            const double s = bc + bo;
            acc += g * (2.0 * bo * bo / (s * s));
        } else if (!((bcm >> w) & 1)) {
            acc += 2.0 * lc * pc * inv_h2;
        }
    };
    face(i > 0, c - sx, 0);
    face(i < nx - 1, c + sx, 1);
    face(j > 0, c - sy, 2);
    face(j < ny - 1, c + sy, 3);
    face(k > 0, c - sz, 4);
    face(k < nz - 1, c + sz, 5);
    dbeta[c] += acc;
}

// ------------------------------------------------------ wall values ----
//
// f_out = f - the lift of non-zero wall values, one thread per cell (only
// cells on the box surface change; the others are copied; f_out may be f).  vals packs one
// value per wall face, walls in the order x-, x+, y-, y+, z-, z+; an x wall
// is (nz, ny), a y wall (nz, nx), a z wall (ny, nx), C order.  A Dirichlet
// value g (phi on the wall) lifts w_wall g, with w_wall = 2 beta_c / h^2 the
// stored weight of the wall face; a Neumann value q (outward flux
// beta dphi/dn) lifts q / h.  Walls are taken in order, as in the oracle.
__global__ void k_bc_lift(int nx, int ny, int nz, int P, long long Q, double inv_h, int bcm,
                          const double *__restrict__ wx, const double *__restrict__ wy,
                          const double *__restrict__ wz, const double *__restrict__ vals,
                          const double *f, double *fout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny || k >= nz) return;
    const long long u = ((long long)k * ny + j) * nx + i;
    const long long c = (long long)k * Q + (long long)j * P + i;
    double v = f[u];
    const long long ax = (long long)ny * nz, ay = (long long)nx * nz, az = (long long)nx * ny;
    const long long o[6] = {0, ax, 2 * ax, 2 * ax + ay, 2 * ax + 2 * ay, 2 * ax + 2 * ay + az};
    auto term = [&](int w, double wall_w, long long at) {
        if ((bcm >> (6 + w / 2)) & 1) return;   // periodic axis: no wall
        const double g = vals[o[w] + at];
        v -= ((bcm >> w) & 1) ? g * inv_h : wall_w * g;
    };
    if (i == 0) term(0, wx[c], (long long)k * ny + j);
    if (i == nx - 1) term(1, wx[c + 1], (long long)k * ny + j);
    if (j == 0) term(2, wy[c], (long long)k * nx + i);
    if (j == ny - 1) term(3, wy[c + P], (long long)k * nx + i);
    if (k == 0) term(4, wz[c], (long long)j * nx + i);
    if (k == nz - 1) term(5, wz[c + Q], (long long)j * nx + i);
    fout[u] = v;
}

// ------------------------------------------------------------ means ----
//
// With every wall Neumann A is singular (constants): f loses its mean before
// the solve and phi after it.  Partial sums over TK_COLZ columns (field 0 =
// f, 1 = phi), then one CTA per box sums them in a fixed order and
// subtracts the mean from every cell.
__global__ void __launch_bounds__(kThreads) k_sum_partials(BoxSet<double> S, int field,
                                                           double *__restrict__ partials)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_COLZ];
    const int b = find_box(ts, S.nbox, t);
    const Box<double> &B = S.boxes[b];
    TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t - ts[b]);
    double v = 0.0;
    if (p.x < B.nx && p.y < B.ny) {
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
        for (int k = z0; k < z1; ++k)
            v += field ? B.phi[(long long)k * B.Q + (long long)p.y * B.P + p.x]
                       : B.f[fidx(B, p.x, p.y, k)];
    }
    double s = block_sum(v);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[t] = s;
}

__global__ void __launch_bounds__(1024) k_mean_finish(BoxSet<double> S,
                                                      const double *__restrict__ partials,
                                                      double *__restrict__ mean)
{
    pdl_wait();
    __shared__ double wsum[32];
    const int b = blockIdx.x;
    const Box<double> &B = S.boxes[b];
    const int *ts = S.tstart[TK_COLZ];
    double s = 0.0;
    for (int q = ts[b] + (int)threadIdx.x; q < ts[b + 1]; q += 1024) s += partials[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 32; ++w) tot += wsum[w];
        mean[B.box] = tot / ((double)B.nx * B.ny * B.nz);
    }
}

__global__ void __launch_bounds__(kThreads) k_sub_mean(BoxSet<double> S, int field,
                                                       const double *__restrict__ mean)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_CELL];
    const int b = find_box(ts, S.nbox, t);
    const Box<double> &B = S.boxes[b];
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    if (field) B.phi[(long long)p.z * B.Q + (long long)p.y * B.P + p.x] -= mean[B.box];
    else B.f[fidx(B, p.x, p.y, p.z)] -= mean[B.box];
}

// ------------------------------------------------- preconditioned CG ----
//
// Conjugate gradients on A x = f (A negative definite: the signs cancel in
// alpha and beta), preconditioned by one symmetric V-cycle z = V r.  Level-0
// FP64 arrays of every box: x in phi2, r in f, z in phi (the V-cycle's own
// solution), p and q in two extra arrays.  Per-box scalars in PcgScalars.

// PcgScalars (kernels.h): rz = <r, z> of the previous iteration (0 before the
// first), rzn = <r, z> of this one, pq = <p, A p>, beta, alpha; [nbox] each.

// A p at cell c (the operator; D stored on FP64 levels, element cf)
__device__ __forceinline__ double apply_at(const double *__restrict__ p,
                                           const Box<double> &B, long long c, long long cf)
{
    double s = fma(B.wx[c], p[c - 1], -B.D[cf] * p[c]);
    s = fma(B.wx[c + 1], p[c + 1], s);
    s = fma(B.wy[c], p[c - B.P], s);
    s = fma(B.wy[c + B.P], p[c + B.P], s);
    s = fma(B.wz[c], p[c - B.Q], s);
    return fma(B.wz[c + B.Q], p[c + B.Q], s);
}

// op 0: partials of <f, phi> (= <r, z>);
// op 1: p = z + beta p;
// op 2: q = A p, partials of <p, q> (a launch of its own: A p reads the
//       neighbours' p of op 1);
// op 3: x += alpha p, r -= alpha q, partials of <r, r>, phi = 0 (the next
//       V-cycle's zero start; z is dead once op 1 has used it);
// op 4 (start): x = phi (the initial guess), r = f - A x, p = 0, partials
//       of <r, r>;
// op 5: phi = x (before a restart from the true residual).
// Partials per TK_COLZ tile (a thread per column of kColZ planes).
__global__ void __launch_bounds__(kThreads) k_pcg(BoxSet<double> S, const int *__restrict__ active,
                                                  int op, double *const *__restrict__ pv,
                                                  double *const *__restrict__ qv, PcgScalars sc,
                                                  double *__restrict__ partials)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_COLZ];
    const int b = find_box(ts, S.nbox, t);
    const Box<double> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t - ts[b]);
    double *P = pv[B.box], *Qa = qv[B.box];
    double v = 0.0;
    if (p.x < B.nx && p.y < B.ny) {
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
        const double be = op == 1 ? sc.beta[B.box] : 0.0, al = op == 3 ? sc.alpha[B.box] : 0.0;
        for (int k = z0; k < z1; ++k) {
            const long long c = (long long)k * B.Q + (long long)p.y * B.P + p.x;
            const long long cf = fidx(B, p.x, p.y, k);
            if (op == 0) {
                v = fma(B.f[cf], B.phi[c], v);
            } else if (op == 1) {
                P[c] = fma(be, P[c], B.phi[c]);
            } else if (op == 2) {
                const double q = apply_at(P, B, c, cf);
                Qa[c] = q;
                v = fma(P[c], q, v);
            } else if (op == 3) {
                B.phi2[c] = fma(al, P[c], B.phi2[c]);
                const double r = fma(-al, Qa[c], B.f[cf]);
                B.f[cf] = r;
                B.phi[c] = 0.0;
                v = fma(r, r, v);
            } else if (op == 4) {
                B.phi2[c] = B.phi[c];
                const double r = residual_at<double, true>(B.phi, B.f, B.wx, B.wy, B.wz, B.D, c,
                                                           cf, B.P, B.Q);
                B.f[cf] = r;
                P[c] = 0.0;
                v = fma(r, r, v);
            } else {
                B.phi[c] = B.phi2[c];
            }
        }
    }
    if (op != 1 && op != 5) {
        const double sum = block_sum(v);
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[t] = sum;
    }
}

// Mixed-precision preconditioner (the FP32 V-cycle applied to the FP64 r):
// op 0: the FP32 right-hand side r / ||r|| and a zero FP32 start;
// op 1: z = ||r|| e, the FP32 solution scaled back into the FP64 phi.
// nrm: ||r|| per box (the last CG update's, or the start's).
__global__ void __launch_bounds__(kThreads) k_pcg_mixed(BoxSet<double> S64, BoxSet<float> S32,
                                                        const int *__restrict__ active, int op,
                                                        const double *__restrict__ nrm)
{
    pdl_wait();
    const int t = blockIdx.x;
    const int *ts = S64.tstart[TK_CELL];
    const int b = find_box(ts, S64.nbox, t);
    const Box<double> &B = S64.boxes[b];
    const Box<float> &E = S32.boxes[b];
    if (active && !active[B.box]) return;
    TilePos p = tile_pos(TK_CELL, B.nx, B.ny, B.nz, t - ts[b]);
    if (p.x >= B.nx || p.y >= B.ny) return;
    const long long c = (long long)p.z * B.Q + (long long)p.y * B.P + p.x;
    const double s = nrm[B.box];
    if (op == 0) {
        E.f[c] = s > 0.0 ? (float)(B.f[fidx(B, p.x, p.y, p.z)] / s) : 0.0f;
        E.phi[c] = 0.0f;
    } else {
        B.phi[c] = s * (double)E.phi[c];
    }
}

// Per-box scalars from finished sums.  step 0: rzn done -> beta = rzn / rz
// (0 on the first iteration), rz = rzn;  step 1: pq done -> alpha = rz / pq.
__global__ void k_pcg_scalars(int nbox, const int *__restrict__ active, int step, PcgScalars sc)
{
    pdl_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox || (active && !active[b])) return;
    if (step == 0) {
        const double rz = sc.rz[b], rzn = sc.rzn[b];
        sc.beta[b] = rz != 0.0 ? rzn / rz : 0.0;
        sc.rz[b] = rzn;
    } else {
        const double pq = sc.pq[b];
        sc.alpha[b] = pq != 0.0 ? sc.rz[b] / pq : 0.0;
    }
}

// One CTA per box: out[box] = sum of the box's partials (fixed order), or
// its square root.
__global__ void __launch_bounds__(1024) k_sum_finish(BoxSet<double> S, const int *__restrict__ active,
                                                     const double *__restrict__ partials,
                                                     double *__restrict__ out, int root)
{
    pdl_wait();
    __shared__ double wsum[32];
    const int b = blockIdx.x;
    const Box<double> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const int *ts = S.tstart[TK_COLZ];
    double s = 0.0;
    for (int q = ts[b] + (int)threadIdx.x; q < ts[b + 1]; q += 1024) s += partials[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 32; ++w) tot += wsum[w];
        out[B.box] = root ? sqrt(tot) : tot;
    }
}

// ---------------------------------------------------- coupled levels ----
//
// The boxes of a coupled level (one MultiFAB level, paper Sec. 2, solved as
// one domain) keep their arrays in the wide layout.  Before every kernel
// that reads a neighbour of a box's cell, the guard cells that face another
// box receive that box's current values (ghost exchange, one CTA per
// intersection patch); the other guard cells stay 0, the Dirichlet walls of
// the union.

template <class T>
__global__ void __launch_bounds__(kThreads) k_exchange(BoxSet<T> S, const int *__restrict__ active,
                                                       const ExchRec *__restrict__ rec, int second)
{
    pdl_wait();
    if (active && !active[0]) return;   // one decision for the whole level
    const ExchRec R = rec[blockIdx.x];
    const Box<T> &D = S.boxes[R.dst];
    const Box<T> &F = S.boxes[R.src];
    T *__restrict__ dphi = second ? D.phi2 : D.phi;          // second: the phi2 arrays
    const T *__restrict__ fphi = second ? F.phi2 : F.phi;
    const int n = R.ex * R.ey * R.ez;
    const int stride = kThreads * gridDim.y;  // a record's cells over gridDim.y CTAs
    for (int e = blockIdx.y * kThreads + threadIdx.y * kTX + threadIdx.x; e < n; e += stride) {
        const int a = e % R.ex, r = e / R.ex;
        const int bb = r % R.ey, c = r / R.ey;
        dphi[(long long)(R.dk + c) * D.Q + (long long)(R.dj + bb) * D.P + R.di + a] =
            fphi[(long long)(R.sk + c) * F.Q + (long long)(R.sj + bb) * F.P + R.si + a];
    }
}

// The guard cells of the six faces of every box (CTA (box, face)) = v.
template <class T>
__global__ void __launch_bounds__(kThreads) k_guard_fill(BoxSet<T> S, T v)
{
    const Box<T> &B = S.boxes[blockIdx.x];
    const int face = blockIdx.y;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const int ea = face < 2 ? ny : nx, eb = face < 4 ? nz : ny;
    for (int e = threadIdx.y * kTX + threadIdx.x; e < ea * eb; e += kThreads) {
        const int a = e % ea, b = e / ea;
        int i, j, k;
        if (face < 2) { i = face ? nx : -1; j = a; k = b; }
        else if (face < 4) { i = a; j = face == 3 ? ny : -1; k = b; }
        else { i = a; j = b; k = face == 5 ? nz : -1; }
        B.phi[(long long)k * B.Q + (long long)j * B.P + i] = v;
    }
}

// Dense inverse of the union of the boxes' coarsest levels (one CTA): each
// box's block as for a single box, plus -w between a box's cell and the cell
// of the neighbouring box (or, on a periodic axis, of the box itself) across
// every exchanged face (from the coarsest level's exchange records: guard
// cell of dst <-> cell of src), then Gauss-Jordan (with the constant shift
// when A is singular).  S: the coarsest level of every box, in union order.
__global__ void __launch_bounds__(1024) k_union_inverse(SetupSet S, UnionBottom U, double *a,
                                                        double *inv64, float *inv32)
{
    __shared__ double col[2 * MG_BOTTOM_CELLS];
    const int n = U.n;
    const SymStore<double, false> M{a, n};
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) a[e] = 0.0;
    __syncthreads();
    for (int b = 0; b < U.nbox; ++b) {
        const SetupBox &B = S.boxes[b];
        assemble_box_block(B.nx, B.ny, B.nz, B.P, B.Q, B.wx, B.wy, B.wz, M, U.off[b]);
    }
    __syncthreads();
    for (int q = 0; q < U.nrec; ++q) {
        const ExchRec R = U.rec[q];
        const SetupBox &D = S.boxes[R.dst];
        const SetupBox &F = S.boxes[R.src];
        const int m = R.ex * R.ey * R.ez;
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const int x = e % R.ex, r = e / R.ex;
            const int y = r % R.ey, z = r / R.ey;
            int gi = R.di + x, gj = R.dj + y, gk = R.dk + z;  // guard cell of dst
            const int si = R.si + x, sj = R.sj + y, sk = R.sk + z;
            // the dst cell next to the guard, and the weight of the face between
            int ci = min(max(gi, 0), D.nx - 1), cj = min(max(gj, 0), D.ny - 1),
                ck = min(max(gk, 0), D.nz - 1);
            const long long c = (long long)ck * D.Q + (long long)cj * D.P + ci;
            double w;
            if (gi < 0) w = D.wx[c];
            else if (gi >= D.nx) w = D.wx[c + 1];
            else if (gj < 0) w = D.wy[c];
            else if (gj >= D.ny) w = D.wy[c + D.P];
            else if (gk < 0) w = D.wz[c];
            else w = D.wz[c + D.Q];
            const int row = U.off[R.dst] + (ck * D.ny + cj) * D.nx + ci;
            const int cl = U.off[R.src] + (sk * F.ny + sj) * F.nx + si;
            // added, not set: across a periodic axis of 2 cells the same two
            // cells are also neighbours through the inner face
            a[(long long)row * n + cl] -= w;
        }
        __syncthreads();
    }
    gauss_jordan_cta(M, n, U.singular != 0, inv64, inv32, col);
}

// Coarsest solve of a coupled level: phi = Ainv f over the union, rows in
// chunks of 32 per CTA (grid y).  S: coarsest level of every box in union
// order.
template <class T>
__global__ void __launch_bounds__(kThreads) k_union_bottom(BoxSet<T> S, UnionBottom U,
                                                           const T *__restrict__ ainv,
                                                           const int *__restrict__ active)
{
    pdl_wait();
    __shared__ T fs[MG_BOTTOM_CELLS];
    if (active && !active[0]) return;
    const int n = U.n;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    auto locate = [&](int q, int &b, long long &c, long long &cf) {
        b = find_box(U.off, U.nbox, q);
        const Box<T> &B = S.boxes[b];
        const int r = q - U.off[b];
        const int i = r % B.nx, j = (r / B.nx) % B.ny, k = r / (B.nx * B.ny);
        c = (long long)k * B.Q + (long long)j * B.P + i;
        cf = fidx(B, i, j, k);
    };
    for (int q = tid; q < n; q += kThreads) {
        int b;
        long long c, cf;
        locate(q, b, c, cf);
        fs[q] = S.boxes[b].f[cf];
    }
    __syncthreads();
    const int lane = threadIdx.x, warp = threadIdx.y;
    for (int rr = 0; rr < 4; ++rr) {
        const int r = blockIdx.x * 32 + warp * 4 + rr;
        if (r >= n) break;
        const T *row = ainv + (long long)r * n;
        T acc = T(0);
        for (int q = lane; q < n; q += 32) acc = fmadd(row[q], fs[q], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            int b;
            long long c, cf;
            locate(r, b, c, cf);
            S.boxes[b].phi[c] = acc;
        }
    }
}

// A coupled level has one residual norm: norm[b] <- sqrt(sum over boxes of
// norm[b]^2) for every box (a fixed-order sum by one thread).
__global__ void k_norm_combine(int nbox, double *__restrict__ norm)
{
    pdl_wait();
    __shared__ double tot;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nbox; ++b) s += norm[b] * norm[b];
        tot = sqrt(s);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) norm[b] = tot;
}

// ------------------------------------ right-hand sides of one box ----
//
// A batch whose boxes are right-hand sides of one box (mg_solve_multi,
// mg_adjoint with several right-hand sides) has one set of weights, 1/D and
// D for all of them.  These pass variants take a tile of box 0's index
// space and update the same cells in every active right-hand side, so the
// six weights and 1/D of a cell are read once for all of them: an FP64 pass
// then moves 16 + 28 / nrhs bytes a cell and right-hand side (phi's sectors,
// half of f, half of phi written) instead of 44.  The arithmetic per cell is
// that of k_rbgs_pass / k_rbgs_pass_oop, in the same order.

template <class T>
__global__ void __launch_bounds__(kThreads) k_rbgs_pass_multi(BoxSet<T> S,
                                                              const int *__restrict__ active,
                                                              int color)
{
    pdl_wait();
    const Box<T> &B0 = S.boxes[0];
    const int P = B0.P;
    const long long Q = B0.Q;
    const TilePos p = tile_pos(TK_PAIR, B0.nx, B0.ny, B0.nz, blockIdx.x);
    const int j = p.y, k = p.z;
    const int i = 2 * p.x + ((j + k + color + B0.par) & 1);
    if (j >= B0.ny || i >= B0.nx) return;
    const long long c = (long long)k * Q + (long long)j * P + i;
    const long long cf =
        split_on(B0) ? (long long)k * Q + (long long)j * P + (color ? (P >> 1) : 0) + p.x : c;
    const T wxa = B0.wx[c], wxb = B0.wx[c + 1], wya = B0.wy[c], wyb = B0.wy[c + P],
            wza = B0.wz[c], wzb = B0.wz[c + Q], id = B0.invD[cf];
#pragma unroll 2
    for (int r = 0; r < S.nbox; ++r) {
        const Box<T> &B = S.boxes[r];
        if (active && !active[B.box]) continue;
        const T *__restrict__ ph = B.phi;
        T s = fmadd(wxa, ph[c - 1], -B.f[cf]);
        s = fmadd(wxb, ph[c + 1], s);
        s = fmadd(wya, ph[c - P], s);
        s = fmadd(wyb, ph[c + P], s);
        s = fmadd(wza, ph[c - Q], s);
        B.phi[c] = fmadd(wzb, ph[c + Q], s) * id;
    }
}

// One colour out of place (as k_rbgs_pass_oop) in every right-hand side.
template <class T>
__global__ void __launch_bounds__(kThreads) k_rbgs_pass_oop_multi(BoxSet<T> S,
                                                                  const int *__restrict__ active,
                                                                  int color, int from2)
{
    pdl_wait();
    const Box<T> &B0 = S.boxes[0];
    const int P = B0.P;
    const long long Q = B0.Q;
    const TilePos p = tile_pos(TK_PAIR, B0.nx, B0.ny, B0.nz, blockIdx.x);
    const int j = p.y, k = p.z, x0 = 2 * p.x;
    if (j >= B0.ny || x0 >= B0.nx) return;
    typedef typename Vec2<T>::type V2;
    const long long c0 = (long long)k * Q + (long long)j * P + x0;
    const int odd = (j + k + color + B0.par) & 1;
    const bool upd = x0 + odd < B0.nx;
    const long long c = c0 + odd;
    const long long cf =
        split_on(B0) ? (long long)k * Q + (long long)j * P + (color ? (P >> 1) : 0) + (x0 >> 1)
                     : c;
    T wxa = 0, wxb = 0, wya = 0, wyb = 0, wza = 0, wzb = 0, id = 0;
    if (upd) {
        wxa = B0.wx[c];
        wxb = B0.wx[c + 1];
        wya = B0.wy[c];
        wyb = B0.wy[c + P];
        wza = B0.wz[c];
        wzb = B0.wz[c + Q];
        id = B0.invD[cf];
    }
#pragma unroll 2
    for (int r = 0; r < S.nbox; ++r) {
        const Box<T> &B = S.boxes[r];
        if (active && !active[B.box]) continue;
        const T *__restrict__ src = from2 ? B.phi2 : B.phi;
        T *__restrict__ dst = from2 ? B.phi : B.phi2;
        V2 pair = *reinterpret_cast<const V2 *>(src + c0);
        if (upd) {
            T s = fmadd(wxa, src[c - 1], -B.f[cf]);
            s = fmadd(wxb, src[c + 1], s);
            s = fmadd(wya, src[c - P], s);
            s = fmadd(wyb, src[c + P], s);
            s = fmadd(wza, src[c - Q], s);
            s = fmadd(wzb, src[c + Q], s);
            const T nv = s * id;
            if (odd) pair.y = nv;
            else pair.x = nv;
        }
        *reinterpret_cast<V2 *>(dst + c0) = pair;
    }
}

// ------------------------------------------- persistent level sweeps ----
//
// The many boxes of a batch (the grids of one MultiFAB level, paper Sec. 2)
// walk a level's stages together.  Instead of one launch per stage, a level
// is smoothed by one launch going down (the pre-smoothing passes, then the
// residual and restriction) and one coming up (prolongation, then the
// post-smoothing passes).  The launch is persistent: its grid is at most the
// number of CTAs that can be resident at once (a cooperative launch, so the
// runtime refuses a grid that could not be), each CTA walks the tiles of
// every active box of a stage with a grid-sized stride, and a grid-wide
// barrier separates consecutive stages.  The barrier is bounded: a CTA that
// has polled it `polls` times without seeing it complete sets the error
// word and returns, so a failure (or a forced time-out) ends the launch with
// an error the host reports as MG_ERR_TIMEOUT, never a hang.

// The barrier (GridSync, kernels.h): one 32-bit word in device memory, zero
// when a solve starts.  Every CTA adds 1 except CTA 0, which adds
// 2^31 - (G - 1): when all G have arrived the word has grown by exactly
// 2^31, so its top bit has flipped and its low bits are back where they
// were -- the next barrier starts from there without a reset.
__device__ __forceinline__ bool grid_sync(const GridSync &g)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
        __threadfence();   // this CTA's stage results before its arrival
        const unsigned old = atomicAdd(g.word, add);
        const volatile unsigned *w = g.word;
        int ok = 1;
        long long i = 0;
        while (((old ^ *w) & 0x80000000u) == 0u) {
            if (i++ >= g.polls) {
                ok = 0;
                atomicExch(g.err, 1);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();   // the other CTAs' results after the barrier
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// One tile of an in-place single-colour pass (as k_rbgs_pass).
template <class T>
__device__ __forceinline__ void pass_tile(const BoxSet<T> &S, const int *__restrict__ active,
                                          int color, int t)
{
    const int *ts = S.tstart[TK_PAIR];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const int P = B.P;
    const long long Q = B.Q;
    const TilePos p = tile_pos(TK_PAIR, B.nx, B.ny, B.nz, t - ts[b]);
    const int j = p.y, k = p.z;
    const int i = 2 * p.x + ((j + k + color + B.par) & 1);
    if (j >= B.ny || i >= B.nx) return;
    const long long c = (long long)k * Q + (long long)j * P + i;
    const long long cf =
        split_on(B) ? (long long)k * Q + (long long)j * P + (color ? (P >> 1) : 0) + p.x : c;
    B.phi[c] = gs_value<T>(B.phi, B.f, B.invD, B.wx, B.wy, B.wz, c, cf, P, Q);
}

// One tile of the black pass out of place, phi2 -> phi (the rest of the
// finest level's first sweep after the look-ahead red pass).
template <class T>
__device__ __forceinline__ void pass_oop_tile(const BoxSet<T> &S, const int *__restrict__ active,
                                              int t)
{
    const int *ts = S.tstart[TK_PAIR];
    const int b = find_box(ts, S.nbox, t);
    const Box<T> &B = S.boxes[b];
    if (active && !active[B.box]) return;
    const TilePos p = tile_pos(TK_PAIR, B.nx, B.ny, B.nz, t - ts[b]);
    double unused = 0.0;
    if (p.y < B.ny && 2 * p.x < B.nx) oop_pair(B, 1, 1, p.y, p.z, 2 * p.x, false, unused);
}

// Work item q of a ghost exchange: record q % nrec, chunk q / nrec of
// `chunks` (as k_exchange with gridDim.y = chunks).
template <class T>
__device__ __forceinline__ void exchange_item(const BoxSet<T> &S, const ExchRec *__restrict__ rec,
                                              int nrec, int chunks, int q, int second)
{
    const ExchRec R = rec[q % nrec];
    const int chunk = q / nrec;
    const Box<T> &D = S.boxes[R.dst];
    const Box<T> &F = S.boxes[R.src];
    T *__restrict__ dphi = second ? D.phi2 : D.phi;
    const T *__restrict__ fphi = second ? F.phi2 : F.phi;
    const int n = R.ex * R.ey * R.ez;
    const int stride = kThreads * chunks;
    for (int e = chunk * kThreads + threadIdx.y * kTX + threadIdx.x; e < n; e += stride) {
        const int a = e % R.ex, r = e / R.ex;
        const int bb = r % R.ey, c = r / R.ey;
        dphi[(long long)(R.dk + c) * D.Q + (long long)(R.dj + bb) * D.P + R.di + a] =
            fphi[(long long)(R.sk + c) * F.Q + (long long)(R.sj + bb) * F.P + R.si + a];
    }
}

// A launch that finds the error word set (a barrier of an earlier launch in
// this solve gave up, leaving the barrier word mid-count) does nothing.
__device__ __forceinline__ bool grid_failed(const GridSync &g)
{
    return *reinterpret_cast<const volatile int *>(g.err) != 0;
}

template <class T>
__global__ void __launch_bounds__(kThreads, 3) k_level_down(BoxSet<T> S, const int *__restrict__ active,
                                                         LevelOps op, GridSync g)
{
    if (grid_failed(g)) return;
    auto each = [&](int n, auto &&work) {
        for (int t = blockIdx.x; t < n; t += gridDim.x) work(t);
    };
    auto exchange = [&](int second) -> bool {
        if (op.nrec == 0) return true;
        each(op.nrec * op.chunks,
             [&](int q) { exchange_item(S, op.rec, op.nrec, op.chunks, q, second); });
        return grid_sync(g);
    };
    const int npair = S.ntiles[TK_PAIR];
    int sweeps = op.nu;
    if (op.head_done) {
        if (!exchange(1)) return;
        each(npair, [&](int t) { pass_oop_tile(S, active, t); });
        if (!grid_sync(g)) return;
        --sweeps;
    }
    for (int sw = 0; sw < sweeps; ++sw)
        for (int color = 0; color < 2; ++color) {
            if (!exchange(0)) return;
            each(npair, [&](int t) { pass_tile(S, active, color, t); });
            if (!grid_sync(g)) return;
        }
    if (!exchange(0)) return;
    const int nc = S.ntiles[TK_COARSE];
    if (op.red && op.partials) {
        if (op.flat) each(nc, [&](int t) { restrict_red_tile<T, true, true>(S, active, t, op.partials); });
        else each(nc, [&](int t) { restrict_red_tile<T, false, true>(S, active, t, op.partials); });
    } else if (op.red) {
        if (op.flat) each(nc, [&](int t) { restrict_red_tile<T, true>(S, active, t); });
        else each(nc, [&](int t) { restrict_red_tile<T, false>(S, active, t); });
    } else {
        if (op.flat) each(nc, [&](int t) { restrict_tile<T, true>(S, active, t); });
        else each(nc, [&](int t) { restrict_tile<T, false>(S, active, t); });
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads, 4) k_level_up(BoxSet<T> S, const int *__restrict__ active,
                                                       LevelOps op, GridSync g)
{
    if (grid_failed(g)) return;
    auto each = [&](int n, auto &&work) {
        for (int t = blockIdx.x; t < n; t += gridDim.x) work(t);
    };
    const int nc = S.ntiles[TK_COARSE];
    if (op.flat) each(nc, [&](int t) { prolong_tile<T, true>(S, active, t); });
    else each(nc, [&](int t) { prolong_tile<T, false>(S, active, t); });
    const int npair = S.ntiles[TK_PAIR];
    for (int sw = 0; sw < op.nu; ++sw)
        for (int c = 0; c < 2; ++c) {
            if (!grid_sync(g)) return;
            if (op.nrec) {
                each(op.nrec * op.chunks,
                     [&](int q) { exchange_item(S, op.rec, op.nrec, op.chunks, q, 0); });
                if (!grid_sync(g)) return;
            }
            const int color = op.reverse ? 1 - c : c;
            each(npair, [&](int t) { pass_tile(S, active, color, t); });
        }
}

// ----------------------------------- coarsest level by conjugate gradients ----
//
// A box whose halving stops at a level too large for a dense inverse (more
// than MG_MAX_BOTTOM cells: a 33^3 box, or 100^3, whose coarsest level is
// 25^3) solves that level by conjugate gradients preconditioned with its
// diagonal, on M = -A (symmetric positive definite): x = phi, r = phi2, and
// two more level arrays p, q.  One persistent cooperative launch runs the
// whole iteration; each of its three stages per iteration ends at the
// bounded grid barrier of the persistent level sweeps, and every dot product
// is summed in a fixed order (per-CTA partial sums, then each CTA adds the
// partials 0 .. G-1), so every CTA takes the same decisions and the result
// is reproducible.  It stops when <r, D^-1 r> has fallen by tol^2, after
// maxit iterations, when 200 iterations in a row have not lowered it below
// its smallest value so far (rounding has stalled it), or if <p, M p> is
// not positive.

// (M v)_c = D_c v_c - sum_f w_f v_nbr: minus the operator, zero outside.
template <class T>
__device__ __forceinline__ T neg_apply(const Box<T> &B, const T *__restrict__ v, long long c,
                                       long long cf)
{
    const T a = B.wx[c], b = B.wx[c + 1], d = B.wy[c], e = B.wy[c + B.P], g = B.wz[c],
            h = B.wz[c + B.Q];
    const T D = B.D ? B.D[cf] : ((a + b) + (d + e)) + (g + h);
    T s = D * v[c];
    s = fmadd(-a, v[c - 1], s);
    s = fmadd(-b, v[c + 1], s);
    s = fmadd(-d, v[c - B.P], s);
    s = fmadd(-e, v[c + B.P], s);
    s = fmadd(-g, v[c - B.Q], s);
    return fmadd(-h, v[c + B.Q], s);
}

// Fixed-order sum of the G partials (every CTA gets the same bits).
__device__ __forceinline__ double sum_partials(const double *__restrict__ part, int G)
{
    __shared__ double tot;
    double v = 0.0;
    if (threadIdx.y == 0) {
        for (int i = threadIdx.x; i < G; i += kTX) v += part[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) tot = v;
    }
    __syncthreads();
    const double r = tot;
    __syncthreads();
    return r;
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_cg_bottom(BoxSet<T> S, const int *__restrict__ active,
                                                        T *p, T *q, double *part, GridSync g,
                                                        double tol, int maxit)
{
    const Box<T> &B = S.boxes[0];
    if ((active && !active[B.box]) || grid_failed(g)) return;
    const int nt = S.ntiles[TK_CELL], G = gridDim.x;
    double *pa = part, *pb = part + G;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    T *__restrict__ x = B.phi;
    T *__restrict__ r = B.phi2;
    // each stage walks the level's cells tile by tile
    auto cells = [&](auto &&body) {
        for (int t = blockIdx.x; t < nt; t += G) {
            const TilePos tp = tile_pos(TK_CELL, nx, ny, nz, t);
            if (tp.x < nx && tp.y < ny)
                body((long long)tp.z * B.Q + (long long)tp.y * B.P + tp.x, fidx(B, tp.x, tp.y, tp.z));
        }
    };
    auto put = [&](double *dst, double v) {
        const double bs = block_sum(v);
        if (threadIdx.x == 0 && threadIdx.y == 0) dst[blockIdx.x] = bs;
    };
    // x = 0, r = -f, p = D^-1 r, partial <r, D^-1 r>
    double acc = 0.0;
    cells([&](long long c, long long cf) {
        const T rv = -B.f[cf];
        const T zv = rv * B.invD[cf];
        x[c] = T(0);
        r[c] = rv;
        p[c] = zv;
        acc += (double)rv * (double)zv;
    });
    put(pb, acc);
    if (!grid_sync(g)) return;
    double rz = sum_partials(pb, G);
    const double rz0 = rz, stop = tol * tol * rz0;
    if (!(rz0 > 0.0)) return;   // f = 0 on this level: x = 0
    double best = rz0;
    int since = 0;
    for (int it = 0; it < maxit; ++it) {
        // q = M p, partial <p, q>
        acc = 0.0;
        cells([&](long long c, long long cf) {
            const T qv = neg_apply(B, p, c, cf);
            q[c] = qv;
            acc += (double)p[c] * (double)qv;
        });
        put(pa, acc);
        if (!grid_sync(g)) return;
        const double pq = sum_partials(pa, G);
        if (!(pq > 0.0)) return;
        const T alpha = (T)(rz / pq);
        // x += alpha p, r -= alpha q, partial <r, D^-1 r>
        acc = 0.0;
        cells([&](long long c, long long cf) {
            x[c] = fmadd(alpha, p[c], x[c]);
            const T rv = fmadd(-alpha, q[c], r[c]);
            r[c] = rv;
            acc += (double)rv * (double)(rv * B.invD[cf]);
        });
        put(pb, acc);
        if (!grid_sync(g)) return;
        const double rz1 = sum_partials(pb, G);
        if (rz1 <= stop) return;
        if (rz1 < best) {
            best = rz1;
            since = 0;
        } else if (++since >= 200) {
            return;
        }
        const T beta = (T)(rz1 / rz);
        rz = rz1;
        // p = D^-1 r + beta p
        cells([&](long long c, long long cf) { p[c] = fmadd(beta, p[c], r[c] * B.invD[cf]); });
        if (!grid_sync(g)) return;
    }
}

// ----------------------------------------------------------- launchers ----

static inline dim3 block2d() { return dim3(kTX, kTY); }

template <class T>
cudaError_t launch_rbgs_pass_oop(const BoxSet<T> &S, const int *active, int color, int from2,
                                 double *partials, cudaStream_t st)
{
    if (partials) {
        if (S.ntiles[TK_PCOLZ] == 0) return cudaSuccess;
        return pdl_launch(k_rbgs_pass_oop_norm<T>, dim3(S.ntiles[TK_PCOLZ]), block2d(), 0, st, S,
                          active, color, from2, partials);
    }
    if (S.ntiles[TK_PAIR] == 0) return cudaSuccess;
    return pdl_launch(k_rbgs_pass_oop<T>, dim3(S.ntiles[TK_PAIR]), block2d(), 0, st, S, active,
                      color, from2);
}

template <class T>
cudaError_t launch_rbgs_pass(const BoxSet<T> &S, const int *active, int color, cudaStream_t st)
{
    if (S.ntiles[TK_PAIR] == 0) return cudaSuccess;
    return pdl_launch(k_rbgs_pass<T>, dim3(S.ntiles[TK_PAIR]), block2d(), 0, st, S, active, color);
}

template <class T>
int sweep_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rbgs_sweep<T>, kSweepThreads, 0) !=
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
    return pdl_launch(k_rbgs_sweep<T>, dim3(S.ntiles[TK_SWEEP]), dim3(kTX, kSweepWarps), 0, st, S,
                      active, src_is_phi2);
}

template <class T>
cudaError_t launch_resid_restrict(const BoxSet<T> &S, const int *active, cudaStream_t st)
{
    if (S.ntiles[TK_COARSE] == 0) return cudaSuccess;
    if (S.flat & (1 << TK_COARSE))
        return pdl_launch(k_resid_restrict<T, true>, dim3(S.ntiles[TK_COARSE]), block2d(), 0, st,
                          S, active);
    return pdl_launch(k_resid_restrict<T, false>, dim3(S.ntiles[TK_COARSE]), block2d(), 0, st, S,
                      active);
}

template <class T>
cudaError_t launch_resid_restrict_red(const BoxSet<T> &S, const int *active, cudaStream_t st,
                                      double *partials)
{
    if (S.ntiles[TK_COARSE] == 0) return cudaSuccess;
    const dim3 g(S.ntiles[TK_COARSE]);
    const bool flat = S.flat & (1 << TK_COARSE);
    if (partials)
        return flat ? pdl_launch(k_resid_restrict_red<T, true, true>, g, block2d(), 0, st, S,
                                 active, partials)
                    : pdl_launch(k_resid_restrict_red<T, false, true>, g, block2d(), 0, st, S,
                                 active, partials);
    return flat ? pdl_launch(k_resid_restrict_red<T, true, false>, g, block2d(), 0, st, S, active,
                             partials)
                : pdl_launch(k_resid_restrict_red<T, false, false>, g, block2d(), 0, st, S, active,
                             partials);
}

cudaError_t launch_inner_judge(const BoxSet<float> &S, int *active32, const double *partials,
                               const int *cstart, int nchunks, int chunk_tiles, double *chunks,
                               const double *se, const double *sr, const double *normf,
                               const double *tol, double floor_rel, int coupled, cudaStream_t st)
{
    if (S.nbox == 0 || nchunks == 0) return cudaSuccess;
    cudaError_t e = pdl_launch(k_inner_sum, dim3(nchunks), dim3(256), 0, st, S, active32, cstart,
                               chunk_tiles, partials, chunks);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_inner_judge, dim3(coupled ? 1 : S.nbox), dim3(1024), 0, st, S, active32,
                      cstart, chunks, se, sr, normf, tol, floor_rel, coupled);
}

template <class T>
cudaError_t launch_prolong(const BoxSet<T> &S, const int *active, cudaStream_t st)
{
    if (S.ntiles[TK_COARSE] == 0) return cudaSuccess;
    if (S.flat & (1 << TK_COARSE))
        return pdl_launch(k_prolong<T, true>, dim3(S.ntiles[TK_COARSE]), block2d(), 0, st,
                          S, active);
    return pdl_launch(k_prolong<T, false>, dim3(S.ntiles[TK_COARSE]), block2d(), 0, st, S,
                      active);
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
    const int kind = mode == 2 ? TK_PCOLZ : TK_COLZ;
    if (S.ntiles[kind] == 0) return cudaSuccess;
    return pdl_launch(k_norm_partials<T>, dim3(S.ntiles[kind]), block2d(), 0, st, S, active, mode,
                      partials);
}

template <class T>
cudaError_t launch_norm_finish(const BoxSet<T> &S, const int *active, const double *partials,
                               double *out, double *copy, double *inv, cudaStream_t st,
                               const double *mult, int mode)
{
    if (S.nbox == 0) return cudaSuccess;
    // the partials' tile starts (the host picks the kind: a run-time index
    // into the kernel's parameter set would copy it to local memory)
    const int *ts = S.tstart[mode == 2 ? TK_PCOLZ : TK_COLZ];
    return pdl_launch(k_norm_finish<T>, dim3(S.nbox), dim3(1024), 0, st, S, active, partials, out,
                      copy, inv, mult, ts);
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
                                 int nu2, cudaStream_t st, int post_first)
{
    if (njobs == 0) return cudaSuccess;
    return pdl_launch(k_coarse_vcycle<T>, dim3(njobs), dim3(CoarseThreads<T>::value), 0, st, jobs,
                      active, nu1, nu2, post_first);
}

cudaError_t launch_refine_update(const BoxSet<double> &S64, const BoxSet<float> &S32,
                                 const int *active, const double *c_e, cudaStream_t st)
{
    if (S64.ntiles[TK_CELL] == 0) return cudaSuccess;
    return pdl_launch(k_refine_update, dim3(S64.ntiles[TK_CELL]), block2d(), 0, st, S64, S32,
                      active, c_e);
}

cudaError_t launch_refine_residual(const BoxSet<double> &S64, const BoxSet<float> &S32,
                                   const int *active, const double *c_r_inv, double *partials,
                                   cudaStream_t st, bool x_zero)
{
    if (S64.ntiles[TK_COLZ] == 0) return cudaSuccess;
    if (x_zero)
        return pdl_launch(k_refine_residual<true>, dim3(S64.ntiles[TK_COLZ]), block2d(), 0, st,
                          S64, S32, active, c_r_inv, partials);
    return pdl_launch(k_refine_residual<false>, dim3(S64.ntiles[TK_COLZ]), block2d(), 0, st, S64,
                      S32, active, c_r_inv, partials);
}

cudaError_t launch_judge(int nbox, const double *norm, const double *normf, int *active,
                         const JudgeState &J, cudaGraphConditionalHandle handle, int use_handle,
                         cudaStream_t st)
{
    const int threads = nbox < 1024 ? ((nbox + 31) / 32) * 32 : 1024;
    return pdl_launch(k_judge, dim3(1), dim3(threads), 0, st, nbox, norm, normf, active, J,
                      handle, use_handle);
}

cudaError_t launch_pack(const BoxSet<double> &S, const long long *off, const double *user,
                        int to_f, cudaStream_t st, double *partials)
{
    if (S.ntiles[TK_COLZ] == 0) return cudaSuccess;
    return pdl_launch(k_pack, dim3(S.ntiles[TK_COLZ]), block2d(), 0, st, S, off, user, to_f,
                      to_f ? partials : nullptr);
}

cudaError_t launch_unpack(const BoxSet<double> &S, const long long *off, double *user,
                          const int *side, cudaStream_t st)
{
    if (S.ntiles[TK_COLZ] == 0) return cudaSuccess;
    return pdl_launch(k_unpack, dim3(S.ntiles[TK_COLZ]), block2d(), 0, st, S, off, user, side);
}

template <class T>
cudaError_t launch_zero(const BoxSet<T> &S, const int *active, cudaStream_t st)
{
    if (S.ntiles[TK_COLZ] == 0) return cudaSuccess;
    return pdl_launch(k_zero<T>, dim3(S.ntiles[TK_COLZ]), block2d(), 0, st, S, active);
}

cudaError_t launch_scales(int nbox, const int *active, int init, const double *norm,
                          const double *normf, double *se, double *sr, double *sr_inv,
                          cudaStream_t st)
{
    return pdl_launch(k_scales, dim3((nbox + 127) / 128), dim3(128), 0, st, nbox, active, init,
                      norm, normf, se, sr, sr_inv);
}

static inline dim3 grid3(int ex, int ey, int ez)
{
    return dim3((ex + kTX - 1) / kTX, (ey + kTY - 1) / kTY, ez);
}

cudaError_t launch_face_weights(int nx, int ny, int nz, double inv_h2, int bcm, const double *beta,
                                double *wx, double *wy, double *wz, cudaStream_t st)
{
    k_face_weights<<<grid3(nx + 1, ny + 1, nz + 1), block2d(), 0, st>>>(
        nx, ny, nz, (int)pitch_row(nx), pitch_plane(nx, ny), inv_h2, bcm, beta, wx, wy, wz);
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

int packed_bottom_bytes(int n, bool fp64)
{
    const long long b = (long long)n * (n + 1) / 2 * (fp64 ? 8 : 4);
    return b <= kPackedBottomBytes ? (int)b : 0;
}

// the dense inverses' packed matrices: dynamic shared memory beyond 48 KB
static void bottom_smem_attributes()
{
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_bottom_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kPackedBottomBytes);
        cudaFuncSetAttribute(k_setup_bottom, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kPackedBottomBytes);
        cudaGetLastError();
    });
}

cudaError_t launch_bottom_inverse(int nx, int ny, int nz, const double *wx, const double *wy,
                                  const double *wz, int singular, double *work, double *inv64,
                                  float *inv32, cudaStream_t st)
{
    const int packed = packed_bottom_bytes(nx * ny * nz, true);
    bottom_smem_attributes();
    k_bottom_inverse<<<1, 1024, packed, st>>>(nx, ny, nz, (int)pitch_row(nx), pitch_plane(nx, ny),
                                              wx, wy, wz, singular, work, inv64, inv32,
                                              packed > 0 ? 1 : 0);
    return counted(cudaGetLastError());
}

cudaError_t launch_setup_tiles(const SetupSet &S, int step, int t0, int t1, cudaStream_t st)
{
    if (t1 <= t0) return cudaSuccess;
    const dim3 g(t1 - t0), b = block2d();
    switch (step) {
    case 0: k_setup<0><<<g, b, 0, st>>>(S, t0); break;
    case 1: k_setup<1><<<g, b, 0, st>>>(S, t0); break;
    case 2: k_setup<2><<<g, b, 0, st>>>(S, t0); break;
    case 3: k_setup<3><<<g, b, 0, st>>>(S, t0); break;
    case 4: k_setup<4><<<g, b, 0, st>>>(S, t0); break;
    case 5: k_setup<5><<<g, b, 0, st>>>(S, t0); break;
    case 6: k_setup<6><<<g, b, 0, st>>>(S, t0); break;
    case 8: k_setup<8><<<g, b, 0, st>>>(S, t0); break;
    case 9: k_setup<9><<<g, b, 0, st>>>(S, t0); break;
    default: return cudaErrorInvalidValue;
    }
    return counted(cudaGetLastError());
}

cudaError_t launch_setup(const SetupSet &S, int step, cudaStream_t st)
{
    if (step < 0 || step > 9 || step == 7) return cudaErrorInvalidValue;
    return launch_setup_tiles(S, step, 0, S.ntiles[setup_kind(step)], st);
}

cudaError_t launch_setup_bottom(const SetupSet &S, int packed_bytes, cudaStream_t st)
{
    if (S.nbox == 0) return cudaSuccess;
    bottom_smem_attributes();
    k_setup_bottom<<<S.nbox, 1024, packed_bytes, st>>>(S, packed_bytes);
    return counted(cudaGetLastError());
}

cudaError_t launch_project_rhs(int nx, int ny, int nz, double h, const double *u, const double *v,
                               const double *w, const double *S, double *f, cudaStream_t st)
{
    k_project_rhs<<<grid3(nx, ny, nz), block2d(), 0, st>>>(nx, ny, nz, 1.0 / h, u, v, w, S, f);
    return counted(cudaGetLastError());
}

cudaError_t launch_project_correct(int nx, int ny, int nz, double h, const double *wx,
                                   const double *wy, const double *wz, const double *phi,
                                   double *u, double *v, double *w, cudaStream_t st, bool wide)
{
    k_project_correct<<<grid3(nx + 1, ny + 1, nz + 1), block2d(), 0, st>>>(
        nx, ny, nz, (int)pitch_row(nx, wide), pitch_plane(nx, ny, wide), h, wx, wy, wz, phi, u,
        v, w);
    return counted(cudaGetLastError());
}

cudaError_t launch_beta_grad(int nx, int ny, int nz, double inv_h2, int bcm, const double *beta,
                             const double *phi, const double *lam, double *dbeta, cudaStream_t st)
{
    k_beta_grad<<<grid3(nx, ny, nz), block2d(), 0, st>>>(nx, ny, nz, inv_h2, bcm, beta, phi, lam,
                                                         dbeta);
    return counted(cudaGetLastError());
}

cudaError_t launch_bc_lift(int nx, int ny, int nz, double inv_h, int bcm, const double *wx,
                           const double *wy, const double *wz, const double *vals,
                           const double *f, double *fout, cudaStream_t st, bool wide)
{
    k_bc_lift<<<grid3(nx, ny, nz), block2d(), 0, st>>>(nx, ny, nz, (int)pitch_row(nx, wide),
                                                       pitch_plane(nx, ny, wide), inv_h, bcm, wx,
                                                       wy, wz, vals, f, fout);
    return counted(cudaGetLastError());
}

cudaError_t launch_remove_mean(const BoxSet<double> &S, int field, double *partials, double *mean,
                               cudaStream_t st)
{
    if (S.ntiles[TK_COLZ] == 0) return cudaSuccess;
    cudaError_t e = pdl_launch(k_sum_partials, dim3(S.ntiles[TK_COLZ]), block2d(), 0, st, S, field,
                               partials);
    if (e != cudaSuccess) return e;
    e = pdl_launch(k_mean_finish, dim3(S.nbox), dim3(1024), 0, st, S, partials, mean);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_sub_mean, dim3(S.ntiles[TK_CELL]), block2d(), 0, st, S, field, mean);
}

template <class T>
cudaError_t launch_exchange(const BoxSet<T> &S, const int *active, const ExchRec *rec, int nrec,
                            int max_cells, cudaStream_t st, int second)
{
    if (nrec == 0) return cudaSuccess;
    // about 4 cells per thread on the largest record (a 256^2 face: 64 CTAs)
    const int chunks = std::max(1, std::min(1024, (max_cells + 4 * kThreads - 1) / (4 * kThreads)));
    return pdl_launch(k_exchange<T>, dim3(nrec, chunks), block2d(), 0, st, S, active, rec, second);
}

template <class T>
cudaError_t launch_rbgs_pass_multi(const BoxSet<T> &S, const int *active, int color, int oop,
                                   int from2, cudaStream_t st)
{
    if (S.nbox == 0 || S.ntiles[TK_PAIR] == 0) return cudaSuccess;
    const int per = S.ntiles[TK_PAIR] / S.nbox;   // tiles of one right-hand side
    if (oop)
        return pdl_launch(k_rbgs_pass_oop_multi<T>, dim3(per), block2d(), 0, st, S, active, color,
                          from2);
    return pdl_launch(k_rbgs_pass_multi<T>, dim3(per), block2d(), 0, st, S, active, color);
}
template cudaError_t launch_rbgs_pass_multi<double>(const BoxSet<double> &, const int *, int, int,
                                                    int, cudaStream_t);
template cudaError_t launch_rbgs_pass_multi<float>(const BoxSet<float> &, const int *, int, int,
                                                   int, cudaStream_t);

template <class T>
int level_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_level_down<T>, kThreads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int m = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_level_up<T>, kThreads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, std::min(n, m));
}
template int level_ctas_per_sm<double>();
template int level_ctas_per_sm<float>();

template <class T>
cudaError_t launch_level(const BoxSet<T> &S, const int *active, int up, const LevelOps &op,
                         const GridSync &g, int grid, cudaStream_t st)
{
    if (S.nbox == 0 || grid < 1) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = block2d();
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident at once
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return counted(up ? cudaLaunchKernelEx(&cfg, k_level_up<T>, S, active, op, g)
                      : cudaLaunchKernelEx(&cfg, k_level_down<T>, S, active, op, g));
}
template cudaError_t launch_level<double>(const BoxSet<double> &, const int *, int,
                                          const LevelOps &, const GridSync &, int, cudaStream_t);
template cudaError_t launch_level<float>(const BoxSet<float> &, const int *, int,
                                         const LevelOps &, const GridSync &, int, cudaStream_t);

template <class T>
int cg_bottom_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cg_bottom<T>, kThreads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, n);
}
template int cg_bottom_ctas_per_sm<double>();
template int cg_bottom_ctas_per_sm<float>();

template <class T>
cudaError_t launch_cg_bottom(const BoxSet<T> &S, const int *active, T *p, T *q, double *part,
                             const GridSync &g, int grid, double tol, int maxit, cudaStream_t st)
{
    if (S.nbox == 0 || grid < 1) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = block2d();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return counted(cudaLaunchKernelEx(&cfg, k_cg_bottom<T>, S, active, p, q, part, g, tol, maxit));
}
template cudaError_t launch_cg_bottom<double>(const BoxSet<double> &, const int *, double *,
                                              double *, double *, const GridSync &, int, double,
                                              int, cudaStream_t);
template cudaError_t launch_cg_bottom<float>(const BoxSet<float> &, const int *, float *, float *,
                                             double *, const GridSync &, int, double, int,
                                             cudaStream_t);

template <class T>
cudaError_t launch_guard_fill(const BoxSet<T> &S, T v, cudaStream_t st)
{
    if (S.nbox == 0) return cudaSuccess;
    k_guard_fill<T><<<dim3(S.nbox, 6), block2d(), 0, st>>>(S, v);
    return counted(cudaGetLastError());
}

cudaError_t launch_union_inverse(const SetupSet &S, const UnionBottom &U, double *work,
                                 double *inv64, float *inv32, cudaStream_t st)
{
    k_union_inverse<<<1, 1024, 0, st>>>(S, U, work, inv64, inv32);
    return counted(cudaGetLastError());
}

template <class T>
cudaError_t launch_union_bottom(const BoxSet<T> &S, const UnionBottom &U, const T *ainv,
                                const int *active, cudaStream_t st)
{
    return pdl_launch(k_union_bottom<T>, dim3((U.n + 31) / 32), block2d(), 0, st, S, U, ainv,
                      active);
}

cudaError_t launch_norm_combine(int nbox, double *norm, cudaStream_t st)
{
    return pdl_launch(k_norm_combine, dim3(1), dim3(256), 0, st, nbox, norm);
}

cudaError_t launch_pcg(const BoxSet<double> &S, const int *active, int op, double *const *pv,
                       double *const *qv, const PcgScalars &sc, double *partials,
                       double *sum_out, cudaStream_t st)
{
    if (S.ntiles[TK_COLZ] == 0) return cudaSuccess;
    cudaError_t e =
        pdl_launch(k_pcg, dim3(S.ntiles[TK_COLZ]), block2d(), 0, st, S, active, op, pv, qv, sc,
                   partials);
    if (e != cudaSuccess || op == 1 || op == 5 || !sum_out) return e;
    return pdl_launch(k_sum_finish, dim3(S.nbox), dim3(1024), 0, st, S, active, partials, sum_out,
                      op >= 3);
}

cudaError_t launch_max_norm(const BoxSet<double> &S, const int *side, int field,
                            double *partials, double *out, cudaStream_t st)
{
    if (S.ntiles[TK_COLZ] == 0) return cudaSuccess;
    k_max_partials<<<S.ntiles[TK_COLZ], block2d(), 0, st>>>(S, side, field, partials);
    cudaError_t e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
    k_max_finish<<<S.nbox, 1024, 0, st>>>(S, partials, out);
    return counted(cudaGetLastError());
}

cudaError_t launch_pcg_mixed(const BoxSet<double> &S64, const BoxSet<float> &S32, const int *active,
                             int op, const double *nrm, cudaStream_t st)
{
    if (S64.ntiles[TK_CELL] == 0) return cudaSuccess;
    return pdl_launch(k_pcg_mixed, dim3(S64.ntiles[TK_CELL]), block2d(), 0, st, S64, S32, active,
                      op, nrm);
}

cudaError_t launch_pcg_scalars(int nbox, const int *active, int step, const PcgScalars &sc,
                               cudaStream_t st)
{
    return pdl_launch(k_pcg_scalars, dim3((nbox + 127) / 128), dim3(128), 0, st, nbox, active,
                      step, sc);
}

#define MG_INSTANTIATE(T)                                                                        \
    template cudaError_t launch_rbgs_pass<T>(const BoxSet<T> &, const int *, int, cudaStream_t);  \
    template cudaError_t launch_rbgs_pass_oop<T>(const BoxSet<T> &, const int *, int, int, double *, \
                                                 cudaStream_t);                                      \
    template cudaError_t launch_rbgs_sweep<T>(const BoxSet<T> &, const int *, int, cudaStream_t); \
    template cudaError_t launch_resid_restrict<T>(const BoxSet<T> &, const int *, cudaStream_t);  \
    template cudaError_t launch_resid_restrict_red<T>(const BoxSet<T> &, const int *,             \
                                                      cudaStream_t, double *);                    \
    template cudaError_t launch_prolong<T>(const BoxSet<T> &, const int *, cudaStream_t);         \
    template cudaError_t launch_residual_field<T>(const BoxSet<T> &, cudaStream_t);               \
    template cudaError_t launch_norm_partials<T>(const BoxSet<T> &, const int *, int, double *,   \
                                                 cudaStream_t);                                   \
    template cudaError_t launch_norm_finish<T>(const BoxSet<T> &, const int *, const double *,    \
                                               double *, double *, double *, cudaStream_t,        \
                                               const double *, int);                              \
    template cudaError_t launch_bottom<T>(const BoxSet<T> &, const int *, int, cudaStream_t);   \
    template cudaError_t launch_zero<T>(const BoxSet<T> &, const int *, cudaStream_t);          \
    template cudaError_t launch_coarse_vcycle<T>(const CoarseJob<T> *, int, const int *, int, int, \
                                                 cudaStream_t, int);                                \
    template cudaError_t launch_exchange<T>(const BoxSet<T> &, const int *, const ExchRec *, int,  \
                                            int, cudaStream_t, int);                                         \
    template cudaError_t launch_guard_fill<T>(const BoxSet<T> &, T, cudaStream_t);                 \
    template cudaError_t launch_union_bottom<T>(const BoxSet<T> &, const UnionBottom &, const T *, \
                                                const int *, cudaStream_t);

MG_INSTANTIATE(double)
MG_INSTANTIATE(float)

}  // namespace mg
