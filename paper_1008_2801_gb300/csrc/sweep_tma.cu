// sweep_tma.cu -- FP32 fused red-black sweep fed by the Tensor Memory
// Accelerator (sm_103a).
//
// Same schedule and arithmetic as k_rbgs_sweep (kernels.cu): a CTA owns a
// 64 x 8 tile and a chunk of planes, marches upward, computes the new red
// values of plane k (its tile plus a one-cell ring) and the new black values
// of plane k-1, out of place.  Here every operand comes from shared memory:
// one thread issues, per plane, five tiled bulk tensor copies (phi with a
// 2-cell halo, f and the three face-weight arrays with a 1-cell halo) into a
// 4-stage ring, two planes ahead of the plane being computed, and an
// mbarrier per stage counts the bytes in.  Like the plain sweep it computes
// 1/D from the six weights, so a stage is 15.1 KB and three CTAs (68 KB of
// shared memory each) fit on an SM.  Waits are bounded: a wait that
// gives up sets the error word and the CTA stops (after waiting, again
// bounded, for its copies in flight), so a failure is reported, never hung.
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
constexpr int kStages = 4;

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
constexpr int kRedBytes = 3 * (kSweepTY + 2) * (2 * kTX + 2) * 4;
constexpr int kSmemBytes = kStages * kStageBytes + pad128(kRedBytes) + 128;

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

// Tensor maps of one box at one level: phi, phi2, f, wx, wy, wz.
struct alignas(64) SweepMaps {
    CUtensorMap m[6];
};

namespace {

__global__ void __launch_bounds__(kTX * kSweepTY, 3)
    k_rbgs_sweep_tma(BoxSet<float> S, const SweepMaps *__restrict__ maps,
                     const int *__restrict__ active, int src_is_phi2, int *__restrict__ err,
                     long long polls)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float(*red)[kSweepTY + 2][2 * kTX + 2] =
        reinterpret_cast<float(*)[kSweepTY + 2][2 * kTX + 2]>(smem + kStages * kStageBytes);
    __shared__ __align__(8) unsigned long long bars[kStages];

    const int t = blockIdx.x;
    const int *ts = S.tstart[TK_SWEEP];
    const int b = find_box(ts, S.nbox, t);
    const Box<float> &B = S.boxes[b];
    if (active && !active[B.box]) return;  // uniform over the CTA
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    float *__restrict__ dst = src_is_phi2 ? B.phi : B.phi2;
    const int P = B.P;
    const long long Q = B.Q;
    const SweepMaps &M = maps[b];
    const CUtensorMap *msrc = &M.m[src_is_phi2 ? 1 : 0];

    const int zc = B.zc;
    const TilePos tp = tile_pos(TK_SWEEP, nx, ny, nz, t - ts[b], zc);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int x0 = 2 * (tp.x - tx);
    const int y0 = tp.y - ty;
    const int xa = x0 + 2 * tx;
    const int y = y0 + ty;
    const int z0 = tp.z * zc;
    const int z1 = min(z0 + zc, nz);
    const bool rowin = y < ny;
    const int pfirst = z0 - 2, plast = z1 + 1;   // planes this CTA reads

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int i = 0; i < 6; ++i) tensormap_acquire(&M.m[i]);
    }
    __syncthreads();

    // plane p -> stage and phase
    auto stage_of = [&](int p) { return (p - pfirst) & (kStages - 1); };
    auto phase_of = [&](int p) { return (unsigned)(((p - pfirst) / kStages) & 1); };
    auto issue = [&](int p) {  // thread 0: the six tiles of plane p
        const int s = stage_of(p);
        const unsigned bar = smem_addr(&bars[s]);
        unsigned char *base = smem + s * kStageBytes;
        mbar_expect_tx(bar, kTxBytes);
        const int zt = p + 1;  // tensor z of logical plane p (guard plane first)
        tma_load_3d(smem_addr(base + kSrcOff), msrc, bar, x0 - 4, y0 - 2, zt);
        tma_load_3d(smem_addr(base + kFOff), &M.m[2], bar, x0 - 4, y0 - 1, zt);
        tma_load_3d(smem_addr(base + kWxOff), &M.m[3], bar, x0 - 4, y0 - 1, zt);
        tma_load_3d(smem_addr(base + kWyOff), &M.m[4], bar, x0 - 4, y0 - 1, zt);
        tma_load_3d(smem_addr(base + kWzOff), &M.m[5], bar, x0 - 4, y0 - 1, zt);
    };
    if (tid == 0)
        for (int p = pfirst; p < pfirst + kStages && p <= plast; ++p) issue(p);

    auto srcv = [&](int p, int xx, int yy) {
        const float *a = reinterpret_cast<const float *>(smem + stage_of(p) * kStageBytes + kSrcOff);
        return a[(yy - (y0 - 2)) * kTileW + (xx - (x0 - 4))];
    };
    auto opv = [&](int p, int off, int xx, int yy) {
        const float *a = reinterpret_cast<const float *>(smem + stage_of(p) * kStageBytes + off);
        return a[(yy - (y0 - 1)) * kTileW + (xx - (x0 - 4))];
    };
    // red value of cell (xx, yy) at plane k from the staged operands
    auto red_at = [&](int k, int xx, int yy) {
        float s = fmaf(opv(k, kWxOff, xx, yy), srcv(k, xx - 1, yy), -opv(k, kFOff, xx, yy));
        s = fmaf(opv(k, kWxOff, xx + 1, yy), srcv(k, xx + 1, yy), s);
        s = fmaf(opv(k, kWyOff, xx, yy), srcv(k, xx, yy - 1), s);
        s = fmaf(opv(k, kWyOff, xx, yy + 1), srcv(k, xx, yy + 1), s);
        s = fmaf(opv(k, kWzOff, xx, yy), srcv(k - 1, xx, yy), s);
        s = fmaf(opv(k + 1, kWzOff, xx, yy), srcv(k + 1, xx, yy), s);
        // 1/D from the six weights, as the plain sweep computes it
        const float d = ((opv(k, kWxOff, xx, yy) + opv(k, kWxOff, xx + 1, yy)) +
                         (opv(k, kWyOff, xx, yy) + opv(k, kWyOff, xx, yy + 1))) +
                        (opv(k, kWzOff, xx, yy) + opv(k + 1, kWzOff, xx, yy));
        return s * __frcp_rn(d);
    };

    const bool ring_row = ty < 2;
    const bool ring_col = ty == 2 && tx < kSweepTY;
    const int ring_y = ty == 0 ? y0 - 1 : y0 + kSweepTY;
    const int ring_x = tx < kSweepTY / 2 ? x0 - 1 : x0 + 2 * kTX;
    const int ring_m = tx % (kSweepTY / 2);

    // planes pfirst and pfirst + 1 must be present before the first step.
    // Every wait outcome is agreed by the whole CTA (__syncthreads_and), so a
    // give-up takes every thread out of the loop together.
    bool ok = true;
    for (int p = pfirst; p <= pfirst + 1 && ok; ++p)
        ok = __syncthreads_and(mbar_wait(smem_addr(&bars[stage_of(p)]), phase_of(p), polls));

    int k = z0 - 1;
    for (; k <= z1 && ok; ++k) {
        if (!__syncthreads_and(
                mbar_wait(smem_addr(&bars[stage_of(k + 1)]), phase_of(k + 1), polls))) {
            ok = false;
            break;
        }
        const int s0 = (k - z0 + 3) % 3;
        // (1) red values of plane k: own column and ring
        {
            const int xr = xa + ((y + k) & 1);
            float v = 0.f;
            if (k >= 0 && k < nz && rowin && xr < nx) v = red_at(k, xr, y);
            red[s0][ty + 1][xr - x0 + 1] = v;
        }
        if ((ring_row || ring_col) && k >= z0 && k < z1) {
            int xx, yy;
            bool in;
            if (ring_row) {
                yy = ring_y;
                xx = x0 + 2 * tx + ((yy + k) & 1);
                in = yy >= 0 && yy < ny && xx < nx;
            } else {
                xx = ring_x;
                yy = y0 + 2 * ring_m + ((xx + y0 + k) & 1);
                in = xx >= 0 && xx < nx && yy < ny;
            }
            red[s0][yy - y0 + 1][xx - x0 + 1] = in ? red_at(k, xx, yy) : 0.f;
        }
        __syncthreads();
        // (2) black values of plane k-1 and the pair store
        const int km = k - 1;
        if (km >= z0 && km < z1 && rowin) {
            const int sm = (km - z0 + 3) % 3;
            const int smm = (km - 1 - z0 + 3) % 3;
            const int parm = (y + km) & 1;
            const int xb = xa + (parm ^ 1);
            const int lb = xb - x0 + 1;
            const float rv = red[sm][ty + 1][xa + parm - x0 + 1];
            float bv = 0.f;
            if (xb < nx) {
                float s = fmaf(opv(km, kWxOff, xb, y), red[sm][ty + 1][lb - 1],
                               -opv(km, kFOff, xb, y));
                s = fmaf(opv(km, kWxOff, xb + 1, y), red[sm][ty + 1][lb + 1], s);
                s = fmaf(opv(km, kWyOff, xb, y), red[sm][ty][lb], s);
                s = fmaf(opv(km, kWyOff, xb, y + 1), red[sm][ty + 2][lb], s);
                s = fmaf(opv(km, kWzOff, xb, y), red[smm][ty + 1][lb], s);
                s = fmaf(opv(k, kWzOff, xb, y), red[s0][ty + 1][lb], s);
                const float d = ((opv(km, kWxOff, xb, y) + opv(km, kWxOff, xb + 1, y)) +
                                 (opv(km, kWyOff, xb, y) + opv(km, kWyOff, xb, y + 1))) +
                                (opv(km, kWzOff, xb, y) + opv(k, kWzOff, xb, y));
                bv = s * __frcp_rn(d);
            }
            const long long c0 = (long long)km * Q + (long long)y * P + xa;
            const float va = parm ? bv : rv;
            const float vb = parm ? rv : bv;
            if (xa + 1 < nx) {
                float2 v2;
                v2.x = va;
                v2.y = vb;
                *reinterpret_cast<float2 *>(dst + c0) = v2;
            } else if (xa < nx) {
                dst[c0] = va;
            }
        }
        __syncthreads();
        // plane k-1 is consumed: its stage takes plane k+3
        if (tid == 0 && k + 3 <= plast && k - 1 >= pfirst) issue(k + 3);
    }
    if (!ok) {
        // report, then wait (with the default bound, whatever `polls` was)
        // for every copy this CTA issued: planes pfirst .. k + 2 (the loop
        // stopped at step k, whose copies up to plane k + 2 were issued; at
        // most the first kStages planes if it stopped before its first step)
        if (tid == 0) atomicExch(err, 1);
        __syncthreads();
        if (tid == 0) {
            const int last = min(plast, k + 2);
            for (int p = pfirst; p <= last; ++p)
                mbar_wait(smem_addr(&bars[stage_of(p)]), phase_of(p), kWaitLimit);
        }
        __syncthreads();
    }
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

// Encode the six maps of a box level (arrays given by their allocation
// base = logical (0, 0, -1)).  Returns false if the driver cannot.
bool encode_sweep_maps(SweepMaps *out, int nx, int ny, int nz, const float *phi_base,
                       const float *phi2_base, const float *f_base, const float *wx_base,
                       const float *wy_base, const float *wz_base)
{
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    const long long P = pitch_row(nx), Q = pitch_plane(nx, ny);
    if (!sweep_tma_fits(nx, ny)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)(ny + 1), (cuuint64_t)(nz + 2)};
    const cuuint64_t strides[2] = {(cuuint64_t)P * 4, (cuuint64_t)Q * 4};
    const cuuint32_t ones[3] = {1, 1, 1};
    const cuuint32_t box_src[3] = {kTileW, kSrcRows, 1};
    const cuuint32_t box_op[3] = {kTileW, kOpRows, 1};
    const cuuint32_t box_wy[3] = {kTileW, kWyRows, 1};
    const float *base[6] = {phi_base, phi2_base, f_base, wx_base, wy_base, wz_base};
    const cuuint32_t *box[6] = {box_src, box_src, box_op, box_op, box_wy, box_op};
    for (int i = 0; i < 6; ++i) {
        CUresult r = fn(&out->m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                        const_cast<float *>(base[i]), dims, strides, box[i], ones,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

size_t sweep_maps_size() { return sizeof(SweepMaps); }

// The ring's dynamic shared memory, and the largest shared-memory carveout so
// that three CTAs fit on an SM.  Function attributes are per device: they
// are set once on each device, the first time a launch or an occupancy
// query runs with that device current.
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
    cudaFuncSetAttribute(k_rbgs_sweep_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmemBytes);
    cudaFuncSetAttribute(k_rbgs_sweep_tma, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (dev >= 0) done[dev] = true;
}

// Levels whose rows and planes hold a whole copy box (72 x 12).
bool sweep_tma_fits(int nx, int ny) { return pitch_row(nx) >= kTileW && ny + 1 >= kSrcRows; }

int sweep_tma_ctas_per_sm()
{
    int n = 0;
    set_smem_attributes();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rbgs_sweep_tma, kTX * kSweepTY,
                                                      kSmemBytes) != cudaSuccess) {
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
                                  int src_is_phi2, int *err, cudaStream_t st, long long wait_polls)
{
    if (S.ntiles[TK_SWEEP] == 0) return cudaSuccess;
    set_smem_attributes();
    k_rbgs_sweep_tma<<<S.ntiles[TK_SWEEP], dim3(kTX, kSweepTY), kSmemBytes, st>>>(
        S, maps, active, src_is_phi2, err, wait_polls);
    return cudaGetLastError();
}

}  // namespace mg
