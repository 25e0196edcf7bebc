// sweep_tma.cu -- FP32 fused red-black sweep fed by the Tensor Memory
// Accelerator, warp-specialised (sm_103a).
//
// Same schedule and arithmetic as k_rbgs_sweep (kernels.cu), and bitwise the
// same result: a CTA owns a 64 x 8 tile and a chunk of planes, marches
// upward, computes the new red values of plane k (its tile plus a one-cell
// ring) and the new black values of plane k-1, out of place.  The roles are
// split over warps:
//   - warp 0, the producer: one thread issues, per plane, five tiled bulk
//     tensor copies (phi with a 2-cell halo, f and the three face-weight
//     arrays with a 1-cell halo, 15.5 KB) into a 6-stage shared-memory ring,
//     each stage guarded by a "full" mbarrier (the bytes landed) and an
//     "empty" one (every consumer warp has read it);
//   - warps 1..11, the consumers (8 row warps, 2 ring-row warps, 1
//     ring-column warp): they wait only on the full barriers, meet at one
//     named barrier per plane (between the red and the black updates), and
//     release a plane's stage when they have read it.
// Every operand address is a per-thread offset fixed at start plus a
// compile-time stage and region constant: the plane loop is unrolled by the
// number of stages, so a step's stage slots, ring slot and colour parity are
// constants and the consumers issue few instructions per cell.  A step holds
// three stages (planes k-1, k, k+1), so the other three are copies in
// flight: 106 KB of shared memory and 71 registers give 2 CTAs (24 warps)
// and six planes in flight per SM.  Measured at 512^3 (one launch, CUDA
// events): 636 us per sweep, 75% of HBM, against 677 us with 4 stages and 3
// CTAs per SM (one plane in flight per CTA), 980 us with 8 or 12 stages and
// one CTA per SM (too few warps to hide the update chain) and 798 us for
// the plain-load sweep.
// Waits are bounded: a wait that gives up sets the error word and the
// threads go on (no consumer may leave the loop while the others meet at
// the named barrier); the producer stops issuing, and before it exits it
// waits, with the default bound, for every copy it issued.
//
// TMA rules kept: every copy starts at x = x0 - 4 (x0 a multiple of 64), a
// multiple of 4 floats = 16 bytes; rows are P floats with P a multiple of 8;
// shared destinations are 128-byte aligned; only loads use out-of-range
// (negative) coordinates, which read zeros.
#include <cuda.h>

#include <mutex>

#include "kernels.h"

namespace mg {

namespace {

constexpr int kTileW = 72;                 // x0 - 4 .. x0 + 67
constexpr int kSrcRows = kSweepTY + 4;     // y0 - 2 .. y0 + 9
constexpr int kOpRows = kSweepTY + 2;      // y0 - 1 .. y0 + 8
constexpr int kWyRows = kSweepTY + 3;      // y0 - 1 .. y0 + 9 (faces)
constexpr int kConsumers = kSweepTY + 3;   // row warps, 2 ring-row warps, 1 ring-column warp
constexpr int kTmaThreads = 32 * (kConsumers + 1);

constexpr int pad128(int bytes) { return (bytes + 127) / 128 * 128; }
constexpr int kSrcBytes = kSrcRows * kTileW * 4;
constexpr int kOpBytes = kOpRows * kTileW * 4;
constexpr int kWyBytes = kWyRows * kTileW * 4;
constexpr int kSrcOff = 0;
constexpr int kFOff = kSrcOff + pad128(kSrcBytes);
constexpr int kWxOff = kFOff + pad128(kOpBytes);
constexpr int kWyOff = kWxOff + pad128(kOpBytes);
constexpr int kWzOff = kWyOff + pad128(kWyBytes);
constexpr int kStageBytes = kWzOff + pad128(kOpBytes);
constexpr unsigned kTxBytes = kSrcBytes + 3 * kOpBytes + kWyBytes;  // bytes landing per stage
// With the prolongation fused (the first post-smoothing sweep): the coarse
// correction under the phi tile, coarse columns x0/2 - 4 .. x0/2 + 35 and
// rows y0/2 - 1 .. y0/2 + 4 of coarse plane p/2, after the stage's regions
constexpr int kEcW = 40, kEcRows = kSweepTY / 2 + 2;
constexpr int kEcOff = kStageBytes;
constexpr int kEcBytes = kEcW * kEcRows * 4;
constexpr int kStageBytesP = kEcOff + pad128(kEcBytes);
constexpr int kRedSW = 2 * kTX + 2, kRedPlane = (kSweepTY + 2) * kRedSW;   // red ring, floats

// NS stages in the ring; the plane loop is unrolled by NS, so that every
// stage and red-ring slot is a compile-time constant.  The red ring needs at
// least 4 slots (planes k, k-1 and k-2 are read while the next step writes
// the fourth) and a slot count dividing the unroll.
__host__ __device__ constexpr int red_slots(int ns) { return ns % 4 == 0 ? 4 : ns; }
constexpr int smem_bytes(int ns, bool prol = false)
{
    return ns * (prol ? kStageBytesP : kStageBytes) + pad128(red_slots(ns) * kRedPlane * 4) + 128;
}

// the configuration the library launches: 6 stages, 2 CTAs (24 warps) per SM
constexpr int kStages = 6, kMinCtas = 2;

constexpr long long kWaitLimit = 1ll << 22;  // default try_wait polls before giving up

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void named_barrier(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of the barrier: at most `polls` polls;
// false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long polls)
{
    for (long long i = 0; i < polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, unsigned bar,
                                            int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<unsigned long long>(map))
                 : "memory");
}

}  // namespace

// Tensor maps of one box at one level: phi, phi2, f, wx, wy, wz and the
// coarse level's phi (the correction; absent where it is not encoded), each
// 128-byte aligned, as CUtensorMap is.
struct SweepMaps {
    CUtensorMap m[7];
};

namespace {

// Red update of one cell from its staged operands (the plain sweep's FMA
// order): s = -f + sum of w x neighbour, times the correctly rounded 1/D.
__device__ __forceinline__ float red_update(float sw, float se, float ss, float sn, float sd,
                                           float su, float wxa, float wxb, float wya, float wyb,
                                           float wza, float wzb, float f)
{
    float s = fmaf(wxa, sw, -f);
    s = fmaf(wxb, se, s);
    s = fmaf(wya, ss, s);
    s = fmaf(wyb, sn, s);
    s = fmaf(wza, sd, s);
    s = fmaf(wzb, su, s);
    return s * __frcp_rn(((wxa + wxb) + (wya + wyb)) + (wza + wzb));
}

// step(kb, J) for J = I .. U-1 while kb + J <= z1 (step 0 always runs).
template <int I, int U, class F>
__device__ __forceinline__ void unroll_steps(F &step, int kb, int z1)
{
    if constexpr (I < U) {
        if (I == 0 || kb + I <= z1) step(kb, std::integral_constant<int, I>{});
        unroll_steps<I + 1, U>(step, kb, z1);
    }
}

// PROL: the level's prolongation phi += e(parent) (the coarse correction,
// in the coarse level's phi) enters the sweep: each stage also holds the
// coarse tile under its plane, and a red update adds a neighbour's parent
// correction to the neighbour's staged value before using it, the FP32 sum
// the prolongation kernel would have stored.  A red update reads only black
// neighbours and a black update only the new red values, so the sweep's
// result is bitwise that of prolongation then sweep; the level's phi in
// memory stays unprolonged, which the out-of-place sweep never reads again.
template <int NS, int MINB, bool PROL>
__global__ void __launch_bounds__(kTmaThreads, MINB)
    k_rbgs_sweep_tma(BoxSet<float> S, const SweepMaps *__restrict__ maps,
                     const int *__restrict__ active, int src_is_phi2, int *__restrict__ err,
                     long long polls)
{
    constexpr int STG = (PROL ? kStageBytesP : kStageBytes) / 4;   // stage stride, floats
    constexpr int NR = red_slots(NS);
    constexpr int PHI = kSrcOff / 4, FF = kFOff / 4, WX = kWxOff / 4, WY = kWyOff / 4,
                  WZ = kWzOff / 4, EC = kEcOff / 4, TW = kTileW, SW = kRedSW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *const sm = reinterpret_cast<float *>(smem);
    float *const red = sm + NS * STG;
    __shared__ __align__(8) unsigned long long full[NS], empty[NS];

    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_SWEEP];
    const int b = find_box(ts, S.nbox, t);
    const Box<float> &B = S.boxes[b];
    if (active && !active[B.box]) return;  // uniform over the CTA
    const int nx = B.nx, ny = B.ny, nz = B.nz, P = B.P;
    const long long Q = B.Q;
    float *__restrict__ dst = src_is_phi2 ? B.phi : B.phi2;
    const SweepMaps &M = maps[b];
    const int zc = B.zc;
    // the tile of the plain sweep's index space (2D tiles of 32 pairs x 8 rows)
    int ex, ey, ez;
    tile_extent(TK_SWEEP, nx, ny, nz, ex, ey, ez, zc);
    const int ntx = (ex + kTX - 1) / kTX, nty = (ey + kSweepTY - 1) / kSweepTY;
    int loc = t - ts[b];
    const int tx = loc % ntx;
    loc /= ntx;
    const int ty = loc % nty;
    const int tz = loc / nty;
    const int x0 = tx * 2 * kTX, y0 = ty * kSweepTY;
    const int z0 = tz * zc, z1 = min(z0 + zc, nz);
    const int pfirst = z0 - 2, plast = z1 + 1;   // planes this CTA reads
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), kConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 0) {
        // producer: plane p goes to stage (p - pfirst) % NS; from plane
        // pfirst + NS on it waits until the consumers have released the stage
        if (lane == 0) {
            for (int i = 0; i < (PROL ? 7 : 6); ++i) tensormap_acquire(&M.m[i]);
            const CUtensorMap *msrc = &M.m[src_is_phi2 ? 1 : 0];
            int last = pfirst - 1;
            for (int p = pfirst; p <= plast; ++p) {
                const int i = p - pfirst, s = i % NS;
                if (i >= NS &&
                    !mbar_wait(smem_addr(&empty[s]), (unsigned)(((i / NS) - 1) & 1), polls)) {
                    atomicExch(err, 1);
                    break;
                }
                last = p;
                unsigned char *base = smem + s * (STG * 4);
                const unsigned bar = smem_addr(&full[s]);
                mbar_expect_tx(bar, kTxBytes + (PROL ? kEcBytes : 0));
                const int zt = p + 1;  // tensor z of logical plane p (guard plane first)
                tma_load_3d(smem_addr(base + kSrcOff), msrc, bar, x0 - 4, y0 - 2, zt);
                tma_load_3d(smem_addr(base + kFOff), &M.m[2], bar, x0 - 4, y0 - 1, zt);
                tma_load_3d(smem_addr(base + kWxOff), &M.m[3], bar, x0 - 4, y0 - 1, zt);
                tma_load_3d(smem_addr(base + kWyOff), &M.m[4], bar, x0 - 4, y0 - 1, zt);
                tma_load_3d(smem_addr(base + kWzOff), &M.m[5], bar, x0 - 4, y0 - 1, zt);
                // the coarse correction under plane p: coarse plane p >> 1
                // (planes -1, -2: the coarse guard plane, zero)
                if (PROL)
                    tma_load_3d(smem_addr(base + kEcOff), &M.m[6], bar, x0 / 2 - 4, y0 / 2 - 1,
                                (p >> 1) + 1);
            }
            // every copy issued has landed before this thread exits (the
            // earlier planes' stages were waited on before their reuse)
            for (int p = max(pfirst, last - NS + 1); p <= last; ++p)
                if (!mbar_wait(smem_addr(&full[(p - pfirst) % NS]),
                               (unsigned)(((p - pfirst) / NS) & 1), kWaitLimit))
                    atomicExch(err, 1);
        }
        return;
    }


    // consumers
    const int cw = warp - 1;           // 0..7 row warps, 8 / 9 ring rows, 10 ring column
    const bool own = cw < kSweepTY;
    const bool colw = cw == kSweepTY + 2;
    const int xa = x0 + 2 * lane;
    // this thread's red cell for the two colour parities q: x or y, the
    // staged-operand offsets (phi region, operand regions), the ring slot
    // position and validity
    int qy = 0;            // row warps: y + k decides q; ring column: x + y0 + k
    int phiC[2], opC[2], ringC[2];
    bool valid[2];
    bool ractive;
    // PROL: offsets in the coarse tile of the parents of the red cell's
    // west, east, south and north neighbours and of its own column (the
    // parent of its z neighbours, in their planes' tiles)
    int eW[2], eE[2], eS[2], eN[2], eC[2];
    auto ecoarse = [&](int x, int y) {
        return ((y >> 1) - (y0 >> 1) + 1) * kEcW + (x >> 1) - (x0 >> 1) + 4;
    };
    auto parents = [&](int q, int x, int y) {
        eW[q] = ecoarse(x - 1, y);
        eE[q] = ecoarse(x + 1, y);
        eS[q] = ecoarse(x, y - 1);
        eN[q] = ecoarse(x, y + 1);
        eC[q] = ecoarse(x, y);
    };
    if (!colw) {
        const int y = own ? y0 + cw : cw == kSweepTY ? y0 - 1 : y0 + kSweepTY;
        const int srow = own ? cw + 1 : cw == kSweepTY ? 0 : kSweepTY + 1;
        qy = y;
        for (int q = 0; q < 2; ++q) {
            const int x = xa + q;
            phiC[q] = (y - y0 + 2) * TW + (x - x0 + 4);
            opC[q] = (y - y0 + 1) * TW + (x - x0 + 4);
            ringC[q] = srow * SW + x - x0 + 1;
            valid[q] = y >= 0 && y < ny && x < nx;
            parents(q, x, y);
        }
        ractive = true;
    } else {
        const int xc = lane < kSweepTY / 2 ? x0 - 1 : x0 + 2 * kTX;
        qy = xc + y0;
        for (int q = 0; q < 2; ++q) {
            const int yy = y0 + 2 * (lane % (kSweepTY / 2)) + q;
            phiC[q] = (yy - y0 + 2) * TW + (xc - x0 + 4);
            opC[q] = (yy - y0 + 1) * TW + (xc - x0 + 4);
            ringC[q] = (yy - y0 + 1) * SW + xc - x0 + 1;
            valid[q] = lane < kSweepTY && xc >= 0 && xc < nx && yy < ny;
            parents(q, xc, yy);
        }
        ractive = lane < kSweepTY;
    }
    // row warps: the pair (xa, xa + 1) of row yo
    const int yo = y0 + cw;
    const bool orow = own && yo < ny;
    const int pairC = (cw + 1) * SW + 2 * lane + 1;   // ring position of xa
    const int bopC = (cw + 1) * TW + 2 * lane + 4;    // operand position of xa
    const bool fullp = xa + 1 < nx, halfp = xa < nx;
    float *gdst = dst + (long long)(z0 - 2) * Q + (long long)yo * P + xa;   // plane kb - 1

    auto step = [&](int kb, auto J) {
        constexpr int j = decltype(J)::value;
        // plane k = kb + j: stages of planes k-1, k, k+1, ring slots of k, k-1, k-2
        constexpr int sM = j % NS, s0 = (j + 1) % NS, sP = (j + 2) % NS;
        constexpr int r0 = j % NR, rm = (j + NR - 1) % NR, rmm = (j + NR - 2) % NR;
        const int k = kb + j;
        if (!mbar_wait(smem_addr(&full[sP]), (unsigned)(((k + 1 - pfirst) / NS) & 1),
                       polls) &&
            lane == 0)
            atomicExch(err, 1);
        const float *SM_ = sm + sM * STG, *S0 = sm + s0 * STG, *SP = sm + sP * STG;
        float *R0 = red + r0 * kRedPlane;
        // (1) red values of plane k: own columns, and the ring inside the chunk
        if (ractive && (own || (k >= z0 && k < z1))) {
            const int q = (qy + k) & 1;
            const int c = q ? phiC[1] : phiC[0];
            const int o = q ? opC[1] : opC[0];
            const bool v = (q ? valid[1] : valid[0]) && k >= 0 && k < nz;
            float nw = S0[PHI + c - 1], ne = S0[PHI + c + 1], ns = S0[PHI + c - TW],
                  nn = S0[PHI + c + TW], nd = SM_[PHI + c], nu = SP[PHI + c];
            if (PROL) {   // the neighbours as the prolongation leaves them
                nw += S0[EC + (q ? eW[1] : eW[0])];
                ne += S0[EC + (q ? eE[1] : eE[0])];
                ns += S0[EC + (q ? eS[1] : eS[0])];
                nn += S0[EC + (q ? eN[1] : eN[0])];
                nd += SM_[EC + (q ? eC[1] : eC[0])];
                nu += SP[EC + (q ? eC[1] : eC[0])];
            }
            const float val = red_update(nw, ne, ns, nn, nd, nu, S0[WX + o], S0[WX + o + 1],
                                         S0[WY + o], S0[WY + o + TW], S0[WZ + o], SP[WZ + o],
                                         S0[FF + o]);
            R0[q ? ringC[1] : ringC[0]] = v ? val : 0.f;
        }
        named_barrier(1, 32 * kConsumers);
        // (2) black values of plane k-1 and the pair store (row warps)
        const int km = k - 1;
        if (orow && km >= z0 && km < z1) {
            const float *Rm = red + rm * kRedPlane, *Rmm = red + rmm * kRedPlane;
            const int pm = (yo + km) & 1;   // red parity at plane k-1
            const int xb = xa + (pm ^ 1);
            const int lb = pairC + (pm ^ 1), ob = bopC + (pm ^ 1);
            const float rv = Rm[pairC + pm];
            float bv = 0.f;
            if (xb < nx) {
                const float wxa = SM_[WX + ob], wxb = SM_[WX + ob + 1];
                const float wya = SM_[WY + ob], wyb = SM_[WY + ob + TW];
                const float wza = SM_[WZ + ob], wzb = S0[WZ + ob];
                float s = fmaf(wxa, Rm[lb - 1], -SM_[FF + ob]);
                s = fmaf(wxb, Rm[lb + 1], s);
                s = fmaf(wya, Rm[lb - SW], s);
                s = fmaf(wyb, Rm[lb + SW], s);
                s = fmaf(wza, Rmm[lb], s);
                s = fmaf(wzb, R0[lb], s);
                bv = s * __frcp_rn(((wxa + wxb) + (wya + wyb)) + (wza + wzb));
            }
            const float va = pm ? bv : rv, vb = pm ? rv : bv;
            float *g = gdst + (long long)j * Q;
            if (fullp) {
                float2 v2;
                v2.x = va;
                v2.y = vb;
                *reinterpret_cast<float2 *>(g) = v2;
            } else if (halfp) {
                g[0] = va;
            }
        }
        // (3) plane k-1 is read: release its stage
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[sM]));
    };
    // the first step also needs planes pfirst and pfirst + 1
    if (!(mbar_wait(smem_addr(&full[0]), 0u, polls) &&
          mbar_wait(smem_addr(&full[1]), 0u, polls)) &&
        lane == 0)
        atomicExch(err, 1);
    for (int kb = z0 - 1; kb <= z1; kb += NS, gdst += NS * Q)
        unroll_steps<0, NS>(step, kb, z1);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

}  // namespace

// Encode the maps of a box level (arrays given by their allocation base =
// logical (0, 0, -1)): phi, phi2, f, wx, wy, wz, and with phic_base the
// coarse level's phi (cx x cy x cz cells) for the fused prolongation.
// Returns false if the driver cannot (or a box does not fit).
bool encode_sweep_maps(SweepMaps *out, int nx, int ny, int nz, const float *phi_base,
                       const float *phi2_base, const float *f_base, const float *wx_base,
                       const float *wy_base, const float *wz_base, const float *phic_base,
                       int cx, int cy, int cz)
{
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    if (!sweep_tma_fits(nx, ny)) return false;
    const cuuint32_t ones[3] = {1, 1, 1};
    auto enc = [&](CUtensorMap *m, const float *base, int mx, int my, int mz,
                   const cuuint32_t *box) {
        const long long P = pitch_row(mx), Q = pitch_plane(mx, my);
        const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)(my + 1), (cuuint64_t)(mz + 2)};
        const cuuint64_t strides[2] = {(cuuint64_t)P * 4, (cuuint64_t)Q * 4};
        return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims,
                  strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const cuuint32_t box_src[3] = {kTileW, kSrcRows, 1};
    const cuuint32_t box_op[3] = {kTileW, kOpRows, 1};
    const cuuint32_t box_wy[3] = {kTileW, kWyRows, 1};
    const float *base[6] = {phi_base, phi2_base, f_base, wx_base, wy_base, wz_base};
    const cuuint32_t *box[6] = {box_src, box_src, box_op, box_op, box_wy, box_op};
    for (int i = 0; i < 6; ++i)
        if (!enc(&out->m[i], base[i], nx, ny, nz, box[i])) return false;
    memset(&out->m[6], 0, sizeof(CUtensorMap));
    if (phic_base) {
        if (!sweep_tma_prol_fits(nx, ny, cx, cy)) return false;
        const cuuint32_t box_ec[3] = {kEcW, kEcRows, 1};
        if (!enc(&out->m[6], phic_base, cx, cy, cz, box_ec)) return false;
    }
    return true;
}

// The fused prolongation reads a 40 x 6 coarse tile: the coarse rows and
// planes hold it, and the level is twice the coarse one in x and y.
bool sweep_tma_prol_fits(int nx, int ny, int cx, int cy)
{
    return nx == 2 * cx && ny == 2 * cy && pitch_row(cx) >= kEcW && cy + 1 >= kEcRows;
}

size_t sweep_maps_size() { return sizeof(SweepMaps); }

// The ring's dynamic shared memory, and the largest shared-memory carveout so
// that two CTAs fit on an SM.  Function attributes are per device: they
// are set once on each device, the first time a launch or an occupancy
// query runs with that device current.
template <int NS, int MINB, bool PROL>
static void set_smem_attributes()
{
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static bool done[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        dev = -1;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && done[dev]) return;
    cudaFuncSetAttribute(k_rbgs_sweep_tma<NS, MINB, PROL>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(NS, PROL));
    cudaFuncSetAttribute(k_rbgs_sweep_tma<NS, MINB, PROL>,
                         cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (dev >= 0) done[dev] = true;
}

// Levels whose rows and planes hold a whole copy box (72 x 12).
bool sweep_tma_fits(int nx, int ny) { return pitch_row(nx) >= kTileW && ny + 1 >= kSrcRows; }

int sweep_tma_ctas_per_sm()
{
    int n = 0;
    set_smem_attributes<kStages, kMinCtas, false>();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rbgs_sweep_tma<kStages, kMinCtas, false>,
                                                      kTmaThreads,
                                                      smem_bytes(kStages)) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

long long sweep_wait_polls(int wait_limit)
{
    return wait_limit == 0 ? kWaitLimit : wait_limit < 0 ? 0 : (long long)wait_limit;
}

cudaError_t launch_rbgs_sweep_tma(const BoxSet<float> &S, const SweepMaps *maps, const int *active,
                                  int src_is_phi2, int *err, cudaStream_t st, long long wait_polls,
                                  bool prolong)
{
    if (S.ntiles[TK_SWEEP] == 0) return cudaSuccess;
    if (prolong) {
        set_smem_attributes<kStages, kMinCtas, true>();
        k_rbgs_sweep_tma<kStages, kMinCtas, true>
            <<<S.ntiles[TK_SWEEP], kTmaThreads, smem_bytes(kStages, true), st>>>(
                S, maps, active, src_is_phi2, err, wait_polls);
    } else {
        set_smem_attributes<kStages, kMinCtas, false>();
        k_rbgs_sweep_tma<kStages, kMinCtas, false>
            <<<S.ntiles[TK_SWEEP], kTmaThreads, smem_bytes(kStages), st>>>(
                S, maps, active, src_is_phi2, err, wait_polls);
    }
    return cudaGetLastError();
}

}  // namespace mg
