// norm_noalloc.cu -- residual norm that allocates nothing (mg_ops.h,
// mg_op_residual_norm_noalloc).
//
// Some callers cannot allocate device memory: a host application whose
// device memory all belongs to its own pool allocator (no cudaMalloc may run
// beside it), or a time-critical loop that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree.  mg_op_residual_norm needs a
// caller-provided scratch array for its per-tile partial sums; this variant
// keeps those partial sums in a file-scope device array instead, so the
// caller passes only inputs and the output.
//
// The array is a fixed, modest size (kNoallocTiles doubles = 512 KiB on
// every GPU that loads the library, held until the process exits).  All
// calls share it and each call overwrites exactly the slots it reads, so no
// clearing is needed; two calls whose kernels overlap on the GPU (different
// streams, or host threads) race on it and must be ordered by the caller.
//
// Host code may not use the array's name as a device address (in host code
// it is only a stand-in symbol): the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made while it is current.  That first call therefore does a runtime
// query; make it before any stream capture that should contain the call.
// The cached address belongs to the device's primary context as it was at
// that first call: after cudaDeviceReset (or any other teardown of that
// context) the module is loaded afresh and the address may change, so the
// entry point must not be used across a device reset in one process.
#include <mutex>

#include "common.cuh"
#include "mg_ops.h"
#include "solver.h"

namespace {

using namespace mg;

constexpr int kNoallocTiles = 65536;   // partial sums: 512 KiB of doubles
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocTiles];

std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device.
int scratch_address(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(MG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(MG_ERR_UNSUPPORTED, "device %d beyond the %d devices supported", dev,
                         kMaxDevices);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            return set_error(MG_ERR_CUDA, "cudaGetSymbolAddress(norm scratch): %s",
                             cudaGetErrorString(e));
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return MG_OK;
}

// f - A phi at cell c (the operator of mg.h; D summed when not stored).
template <class T>
__device__ __forceinline__ T resid(const Box<T> &B, long long c)
{
    const T a = B.wx[c], b = B.wx[c + 1], d = B.wy[c], e = B.wy[c + B.P], g = B.wz[c],
            h = B.wz[c + B.Q];
    T s = a * B.phi[c - 1];
    s = fma(b, B.phi[c + 1], s);
    s = fma(d, B.phi[c - B.P], s);
    s = fma(e, B.phi[c + B.P], s);
    s = fma(g, B.phi[c - B.Q], s);
    s = fma(h, B.phi[c + B.Q], s);
    const T D = B.D ? B.D[c] : ((a + b) + (d + e)) + (g + h);
    return B.f[c] - fma(-D, B.phi[c], s);
}

// One CTA per column tile (32 x 8 columns, 16 planes): fixed-order sum of r^2.
template <class T>
__global__ void __launch_bounds__(kThreads) k_noalloc_partials(Box<T> B, double *__restrict__ part)
{
    const int t = blockIdx.x;
    const TilePos p = tile_pos(TK_COLZ, B.nx, B.ny, B.nz, t);
    double v = 0.0;
    if (p.x < B.nx && p.y < B.ny) {
        const int z0 = p.z * kColZ, z1 = min(z0 + kColZ, B.nz);
        for (int k = z0; k < z1; ++k) {
            const long long c = (long long)k * B.Q + (long long)p.y * B.P + p.x;
            const double r = (double)resid<T>(B, c);
            v = fma(r, r, v);
        }
    }
    const double s = block_sum(v);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[t] = s;
}

__global__ void __launch_bounds__(1024) k_noalloc_finish(const double *__restrict__ part, int n,
                                                         double *__restrict__ out)
{
    __shared__ double w[32];
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += 1024) s += part[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < 32; ++i) tot += w[i];
        *out = sqrt(tot);
    }
}

template <class T>
int run(const int n[3], const void *wx, const void *wy, const void *wz, const void *D,
        const void *f, const void *phi, double *out, cudaStream_t st)
{
    const long long Q = pitch_plane(n[0], n[1]);
    Box<T> B{};
    B.nx = n[0];
    B.ny = n[1];
    B.nz = n[2];
    B.P = (int)pitch_row(n[0]);
    B.Q = Q;
    B.wx = static_cast<const T *>(wx) + Q;
    B.wy = static_cast<const T *>(wy) + Q;
    B.wz = static_cast<const T *>(wz) + Q;
    B.D = D ? static_cast<const T *>(D) + Q : nullptr;
    B.f = const_cast<T *>(static_cast<const T *>(f)) + Q;
    B.phi = const_cast<T *>(static_cast<const T *>(phi)) + Q;
    const long long tiles = tiles_of(TK_COLZ, n[0], n[1], n[2]);
    if (tiles > kNoallocTiles)
        return set_error(MG_ERR_INVALID_ARG,
                         "mg_op_residual_norm_noalloc: %lld column tiles exceed the static "
                         "scratch of %d (32 x 8 columns of 16 planes each; at most %d)",
                         tiles, kNoallocTiles, kNoallocTiles);
    double *part = nullptr;
    int rc = scratch_address(&part);
    if (rc != MG_OK) return rc;
    k_noalloc_partials<T><<<(unsigned)tiles, dim3(kTX, kTY), 0, st>>>(B, part);
    k_noalloc_finish<<<1, 1024, 0, st>>>(part, (int)tiles, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(MG_ERR_CUDA, "mg_op_residual_norm_noalloc launch: %s",
                         cudaGetErrorString(e));
    return MG_OK;
}

}  // namespace

extern "C" int mg_op_residual_norm_noalloc(int prec, const int n[3], const void *wx,
                                           const void *wy, const void *wz, const void *D,
                                           const void *f, const void *phi, double *out,
                                           void *stream)
{
    if (!n || n[0] < 1 || n[1] < 1 || n[2] < 1 || !wx || !wy || !wz || !f || !phi || !out)
        return set_error(MG_ERR_INVALID_ARG, "mg_op_residual_norm_noalloc: bad argument");
    if (prec == MG_OPS_F64)
        return run<double>(n, wx, wy, wz, D, f, phi, out, (cudaStream_t)stream);
    if (prec == MG_OPS_F32)
        return run<float>(n, wx, wy, wz, D, f, phi, out, (cudaStream_t)stream);
    return set_error(MG_ERR_INVALID_ARG, "prec must be MG_OPS_F64 or MG_OPS_F32");
}
