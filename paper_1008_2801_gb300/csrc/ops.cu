// ops.cu -- single-stage entry points (mg_ops.h): one box, caller-owned
// arrays in the level layout, one kernel (or a short fixed sequence) each.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "mg_ops.h"
#include "solver.h"

using namespace mg;

namespace {

#define CKO(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_error(MG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

bool bad_dims(const int n[3]) { return !n || n[0] < 1 || n[1] < 1 || n[2] < 1; }
bool all_even(const int n[3]) { return n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0; }

template <class T>
T *logical(const void *base, const int n[3])
{
    return base ? const_cast<T *>(static_cast<const T *>(base)) + pitch_plane(n[0], n[1]) : nullptr;
}

// Device descriptor block of a one-box set, freed in stream order.
template <class T>
struct OneBox {
    Box<T> box;
    int ts[TK_NKIND][2];
};

template <class T>
struct TempSet {
    BoxSet<T> S{};
    void *mem = nullptr;
    cudaStream_t st = nullptr;
    int make(const Box<T> &B, cudaStream_t stream)
    {
        st = stream;
        OneBox<T> h;
        memset(&h, 0, sizeof h);
        h.box = B;
        S.nbox = 1;
        for (int k = 0; k < TK_NKIND; ++k) {
            h.ts[k][0] = 0;
            h.ts[k][1] = tiles_of(k, B.nx, B.ny, B.nz, B.zc);
            S.ntiles[k] = h.ts[k][1];
            int ex, ey, ez;
            tile_extent(k, B.nx, B.ny, B.nz, ex, ey, ez, B.zc);
            if (tile_flat(k, ex)) S.flat |= 1 << k;
        }
        CKO(cudaMallocAsync(&mem, sizeof h, st));
        CKO(cudaMemcpyAsync(mem, &h, sizeof h, cudaMemcpyHostToDevice, st));
        OneBox<T> *d = static_cast<OneBox<T> *>(mem);
        S.boxes = &d->box;
        for (int k = 0; k < TK_NKIND; ++k) S.tstart[k] = d->ts[k];
        return MG_OK;
    }
    ~TempSet()
    {
        if (mem) cudaFreeAsync(mem, st);
    }
};

template <class T>
Box<T> level_box(const int n[3], const void *wx, const void *wy, const void *wz, const void *invD,
                 const void *f, const void *phi, const void *phi2)
{
    Box<T> B{};
    B.nx = n[0];
    B.ny = n[1];
    B.nz = n[2];
    B.P = (int)pitch_row(n[0]);
    B.Q = pitch_plane(n[0], n[1]);
    B.wx = logical<T>(wx, n);
    B.wy = logical<T>(wy, n);
    B.wz = logical<T>(wz, n);
    B.invD = logical<T>(invD, n);
    B.f = logical<T>(f, n);
    B.phi = logical<T>(phi, n);
    B.phi2 = logical<T>(phi2, n);
    B.zc = kSweepZ;
    return B;
}

template <class T, class F>
int with_set(const Box<T> &B, cudaStream_t st, F launch)
{
    cudaGetLastError();  // drop a stale non-sticky error of an earlier call
    TempSet<T> ts;
    int rc = ts.make(B, st);
    if (rc != MG_OK) return rc;
    CKO(launch(ts.S));
    return MG_OK;
}

}  // namespace

extern "C" {

int mg_layout(const int n[3], long long *P, long long *Q, long long *elems)
{
    if (bad_dims(n)) return set_error(MG_ERR_INVALID_ARG, "bad dims");
    if (P) *P = pitch_row(n[0]);
    if (Q) *Q = pitch_plane(n[0], n[1]);
    if (elems) *elems = level_elems(n[0], n[1], n[2]);
    return MG_OK;
}

int mg_op_face_weights(const int n[3], double h, int bc, const double *beta, double *wx,
                       double *wy, double *wz, void *stream)
{
    if (bad_dims(n) || !(h > 0.0) || bc < 0 || bc > 63 || !beta || !wx || !wy || !wz)
        return set_error(MG_ERR_INVALID_ARG, "bad argument");
    CKO(launch_face_weights(n[0], n[1], n[2], 1.0 / (h * h), bc, beta, logical<double>(wx, n),
                            logical<double>(wy, n), logical<double>(wz, n), (cudaStream_t)stream));
    return MG_OK;
}

int mg_op_coarsen_weights(const int n[3], const double *wx, const double *wy, const double *wz,
                          double *cwx, double *cwy, double *cwz, void *stream)
{
    if (bad_dims(n) || !all_even(n) || !wx || !wy || !wz || !cwx || !cwy || !cwz)
        return set_error(MG_ERR_INVALID_ARG, "bad argument (fine dims must be even)");
    const int c[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    CKO(launch_coarsen(n[0], n[1], n[2], logical<double>(wx, n), logical<double>(wy, n),
                       logical<double>(wz, n), logical<double>(cwx, c), logical<double>(cwy, c),
                       logical<double>(cwz, c), (cudaStream_t)stream));
    return MG_OK;
}

int mg_op_inv_diag(const int n[3], const double *wx, const double *wy, const double *wz,
                   double *invD, double *D, void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !invD)
        return set_error(MG_ERR_INVALID_ARG, "bad argument");
    CKO(launch_inv_diag(n[0], n[1], n[2], logical<double>(wx, n), logical<double>(wy, n),
                        logical<double>(wz, n), logical<double>(invD, n), logical<double>(D, n),
                        (cudaStream_t)stream));
    return MG_OK;
}

int mg_op_round_f32(const int n[3], const double *wx, const double *wy, const double *wz,
                    const double *invD, float *wx32, float *wy32, float *wz32, float *invD32,
                    void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !invD || !wx32 || !wy32 || !wz32 || !invD32)
        return set_error(MG_ERR_INVALID_ARG, "bad argument");
    CKO(launch_round_f32(n[0], n[1], n[2], logical<double>(wx, n), logical<double>(wy, n),
                         logical<double>(wz, n), logical<double>(invD, n), logical<float>(wx32, n),
                         logical<float>(wy32, n), logical<float>(wz32, n),
                         logical<float>(invD32, n), (cudaStream_t)stream));
    return MG_OK;
}

#define DISPATCH(prec, BODY)                                                          \
    do {                                                                              \
        if ((prec) == MG_OPS_F64) {                                                   \
            typedef double T;                                                         \
            BODY;                                                                     \
        } else if ((prec) == MG_OPS_F32) {                                            \
            typedef float T;                                                          \
            BODY;                                                                     \
        } else {                                                                      \
            return set_error(MG_ERR_INVALID_ARG, "prec must be MG_OPS_F64 or _F32"); \
        }                                                                             \
    } while (0)

int mg_op_rbgs_pass(int prec, const int n[3], const void *wx, const void *wy, const void *wz,
                    const void *invD, const void *f, void *phi, int color, void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !invD || !f || !phi || (color != 0 && color != 1))
        return set_error(MG_ERR_INVALID_ARG, "bad argument");
    DISPATCH(prec, {
        Box<T> B = level_box<T>(n, wx, wy, wz, invD, f, phi, nullptr);
        return with_set(B, (cudaStream_t)stream, [&](const BoxSet<T> &S) {
            return launch_rbgs_pass(S, nullptr, color, (cudaStream_t)stream);
        });
    });
}

int mg_op_rbgs_sweep(int prec, const int n[3], const void *wx, const void *wy, const void *wz,
                     const void *f, const void *phi_in, void *phi_out, int zc, void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !f || !phi_in || !phi_out ||
        phi_in == phi_out)
        return set_error(MG_ERR_INVALID_ARG, "bad argument (phi_in and phi_out must differ)");
    if (level_elems(n[0], n[1], n[2]) > kSweepMaxElems)
        return set_error(MG_ERR_UNSUPPORTED, "fused sweep: level of 2^31 elements or more");
    DISPATCH(prec, {
        Box<T> B = level_box<T>(n, wx, wy, wz, nullptr, f, phi_in, phi_out);
        B.zc = zc > 0 ? zc : kSweepZ;
        return with_set(B, (cudaStream_t)stream, [&](const BoxSet<T> &S) {
            return launch_rbgs_sweep(S, nullptr, 0, (cudaStream_t)stream);
        });
    });
}

// The TMA sweep through a one-box set; phic (or null): the coarse level's
// phi, for the fused prolongation.
static int sweep_tma_op(const int n[3], const float *wx, const float *wy, const float *wz,
                        const float *f, const float *phic, const float *phi_in, float *phi_out,
                        int zc, void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !f || !phi_in || !phi_out ||
        phi_in == phi_out || (phic && !all_even(n)))
        return set_error(MG_ERR_INVALID_ARG,
                         "bad argument (phi_in and phi_out must differ; with phic n even)");
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    const int c[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    Box<float> B = level_box<float>(n, wx, wy, wz, nullptr, f, phi_in, phi_out);
    B.zc = zc > 0 ? zc : kSweepZ;
    if (phic) {
        B.phic = logical<float>(phic, c);
        B.cP = (int)pitch_row(c[0]);
        B.cQ = pitch_plane(c[0], c[1]);
    }
    std::vector<char> host(sweep_maps_size() + 128);   // tensor maps are 128-byte aligned
    SweepMaps *m = reinterpret_cast<SweepMaps *>(round_up((long long)(uintptr_t)host.data(), 128));
    if (!sweep_tma_fits(n[0], n[1]))
        return set_error(MG_ERR_UNSUPPORTED, "level too small for the TMA sweep (nx >= 64, ny >= 11)");
    if (phic && !sweep_tma_prol_fits(n[0], n[1], c[0], c[1]))
        return set_error(MG_ERR_UNSUPPORTED, "coarse level too small for its copy box");
    if (!encode_sweep_maps(m, n[0], n[1], n[2], phi_in, phi_out, f, wx, wy, wz, phic, c[0], c[1],
                           c[2]))
        return set_error(MG_ERR_UNSUPPORTED, "tensor maps cannot be encoded on this driver");
    TempSet<float> ts;
    int rc = ts.make(B, st);
    if (rc != MG_OK) return rc;
    char *dev = nullptr;
    CKO(cudaMallocAsync(&dev, sweep_maps_size() + 64, st));
    int *err = reinterpret_cast<int *>(dev + sweep_maps_size());
    CKO(cudaMemcpyAsync(dev, m, sweep_maps_size(), cudaMemcpyHostToDevice, st));
    CKO(cudaMemsetAsync(err, 0, sizeof(int), st));
    CKO(launch_rbgs_sweep_tma(ts.S, reinterpret_cast<const SweepMaps *>(dev), nullptr, 0, err, st,
                              sweep_wait_polls(0), phic != nullptr));
    int herr = 0;
    CKO(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKO(cudaStreamSynchronize(st));
    CKO(cudaFreeAsync(dev, st));
    if (herr) return set_error(MG_ERR_TIMEOUT, "a tile-copy wait gave up");
    return MG_OK;
}

int mg_op_rbgs_sweep_tma(const int n[3], const float *wx, const float *wy, const float *wz,
                         const float *f, const float *phi_in, float *phi_out, int zc,
                         void *stream)
{
    return sweep_tma_op(n, wx, wy, wz, f, nullptr, phi_in, phi_out, zc, stream);
}

int mg_op_rbgs_sweep_tma_prolong(const int n[3], const float *wx, const float *wy,
                                 const float *wz, const float *f, const float *phic,
                                 const float *phi_in, float *phi_out, int zc, void *stream)
{
    if (!phic) return set_error(MG_ERR_INVALID_ARG, "bad argument (phic)");
    return sweep_tma_op(n, wx, wy, wz, f, phic, phi_in, phi_out, zc, stream);
}

int mg_op_residual(int prec, const int n[3], const void *wx, const void *wy, const void *wz,
                   const void *D, const void *f, const void *phi, void *r, void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !f || !phi || !r)
        return set_error(MG_ERR_INVALID_ARG, "bad argument");
    DISPATCH(prec, {
        Box<T> B = level_box<T>(n, wx, wy, wz, nullptr, f, phi, r);
        B.D = logical<T>(D, n);
        return with_set(B, (cudaStream_t)stream, [&](const BoxSet<T> &S) {
            return launch_residual_field(S, (cudaStream_t)stream);
        });
    });
}

int mg_op_residual_restrict(int prec, const int n[3], const void *wx, const void *wy,
                            const void *wz, const void *D, const void *f, const void *phi,
                            void *fc, void *phic, void *stream)
{
    if (bad_dims(n) || !all_even(n) || !wx || !wy || !wz || !f || !phi || !fc || !phic)
        return set_error(MG_ERR_INVALID_ARG, "bad argument (fine dims must be even)");
    const int c[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    DISPATCH(prec, {
        Box<T> B = level_box<T>(n, wx, wy, wz, nullptr, f, phi, nullptr);
        B.D = logical<T>(D, n);
        B.fc = logical<T>(fc, c);
        B.phic = logical<T>(phic, c);
        B.cP = (int)pitch_row(c[0]);
        B.cQ = pitch_plane(c[0], c[1]);
        return with_set(B, (cudaStream_t)stream, [&](const BoxSet<T> &S) {
            return launch_resid_restrict(S, nullptr, (cudaStream_t)stream);
        });
    });
}

int mg_op_residual_restrict_red(int prec, const int n[3], const void *wx, const void *wy,
                                const void *wz, const void *D, const void *f, const void *phi,
                                void *fc, void *phic, void *stream)
{
    if (bad_dims(n) || !all_even(n) || !wx || !wy || !wz || !f || !phi || !fc || !phic)
        return set_error(MG_ERR_INVALID_ARG, "bad argument (fine dims must be even)");
    const int c[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    DISPATCH(prec, {
        Box<T> B = level_box<T>(n, wx, wy, wz, nullptr, f, phi, nullptr);
        B.D = logical<T>(D, n);
        B.fc = logical<T>(fc, c);
        B.phic = logical<T>(phic, c);
        B.cP = (int)pitch_row(c[0]);
        B.cQ = pitch_plane(c[0], c[1]);
        return with_set(B, (cudaStream_t)stream, [&](const BoxSet<T> &S) {
            return launch_resid_restrict_red(S, nullptr, (cudaStream_t)stream);
        });
    });
}

int mg_op_prolong_add(int prec, const int n[3], const void *phic, void *phi, void *stream)
{
    if (bad_dims(n) || !all_even(n) || !phic || !phi)
        return set_error(MG_ERR_INVALID_ARG, "bad argument (fine dims must be even)");
    const int c[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    DISPATCH(prec, {
        Box<T> B = level_box<T>(n, nullptr, nullptr, nullptr, nullptr, nullptr, phi, nullptr);
        B.phic = logical<T>(phic, c);
        B.cP = (int)pitch_row(c[0]);
        B.cQ = pitch_plane(c[0], c[1]);
        return with_set(B, (cudaStream_t)stream, [&](const BoxSet<T> &S) {
            return launch_prolong(S, nullptr, (cudaStream_t)stream);
        });
    });
}

int mg_op_bottom_inverse(const int n[3], int singular, const double *wx, const double *wy,
                         const double *wz, double *work, double *Ainv, void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !work || !Ainv ||
        (long long)n[0] * n[1] * n[2] > MG_MAX_BOTTOM)
        return set_error(MG_ERR_INVALID_ARG, "bad argument (at most MG_MAX_BOTTOM cells)");
    CKO(launch_bottom_inverse(n[0], n[1], n[2], logical<double>(wx, n), logical<double>(wy, n),
                              logical<double>(wz, n), singular ? 1 : 0, work, Ainv, nullptr,
                              (cudaStream_t)stream));
    return MG_OK;
}

int mg_op_bottom_solve(int prec, const int n[3], const void *Ainv, const void *f, void *phi,
                       void *stream)
{
    if (bad_dims(n) || !Ainv || !f || !phi || (long long)n[0] * n[1] * n[2] > MG_MAX_BOTTOM)
        return set_error(MG_ERR_INVALID_ARG, "bad argument (at most MG_MAX_BOTTOM cells)");
    DISPATCH(prec, {
        Box<T> B = level_box<T>(n, nullptr, nullptr, nullptr, nullptr, f, phi, nullptr);
        B.ainv = static_cast<const T *>(Ainv);
        const int cells = n[0] * n[1] * n[2];
        return with_set(B, (cudaStream_t)stream, [&](const BoxSet<T> &S) {
            return launch_bottom(S, nullptr, cells, (cudaStream_t)stream);
        });
    });
}

long long mg_op_norm_scratch(const int n[3])
{
    if (bad_dims(n)) return 0;
    return tiles_of(TK_CELL, n[0], n[1], n[2]);
}

int mg_op_residual_norm(int prec, const int n[3], const void *wx, const void *wy, const void *wz,
                        const void *D, const void *f, const void *phi, double *partials,
                        double *out, void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !f || !phi || !partials || !out)
        return set_error(MG_ERR_INVALID_ARG, "bad argument");
    DISPATCH(prec, {
        Box<T> B = level_box<T>(n, wx, wy, wz, nullptr, f, phi, nullptr);
        B.D = logical<T>(D, n);
        return with_set(B, (cudaStream_t)stream, [&](const BoxSet<T> &S) {
            cudaError_t e = launch_norm_partials(S, nullptr, 0, partials, (cudaStream_t)stream);
            if (e != cudaSuccess) return e;
            return launch_norm_finish(S, nullptr, partials, out, nullptr, nullptr,
                                      (cudaStream_t)stream);
        });
    });
}

int mg_op_refine(const int n[3], const double *wx, const double *wy, const double *wz,
                 const double *D, const double *f, double *x, float *e, float *r32,
                 const double *c_e, const double *c_r, double *partials, double *out,
                 void *stream)
{
    if (bad_dims(n) || !wx || !wy || !wz || !f || !x || !e || !r32 || !c_e || !c_r ||
        !partials || !out)
        return set_error(MG_ERR_INVALID_ARG, "bad argument");
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    Box<double> B = level_box<double>(n, wx, wy, wz, nullptr, f, x, nullptr);
    B.D = logical<double>(D, n);
    Box<float> E = level_box<float>(n, nullptr, nullptr, nullptr, nullptr, r32, e, nullptr);
    TempSet<double> s64;
    TempSet<float> s32;
    int rc = s64.make(B, st);
    if (rc != MG_OK) return rc;
    rc = s32.make(E, st);
    if (rc != MG_OK) return rc;
    double *sc = nullptr;  // se, sr, sr_inv
    CKO(cudaMallocAsync(&sc, 3 * sizeof(double), st));
    CKO(launch_scales(1, nullptr, 1, nullptr, c_r, sc, sc + 1, sc + 2, st));
    CKO(launch_refine_update(s64.S, s32.S, nullptr, c_e, st));
    CKO(launch_refine_residual(s64.S, s32.S, nullptr, sc + 2, partials, st));
    CKO(launch_norm_finish(s64.S, nullptr, partials, out, nullptr, nullptr, st, sc + 1));
    CKO(cudaFreeAsync(sc, st));
    return MG_OK;
}

int mg_op_beta_grad(const int n[3], double h, int bc, const double *beta, const double *phi,
                    const double *lambda, double *dbeta, void *stream)
{
    if (bad_dims(n) || !(h > 0.0) || bc < 0 || bc > 63 || !beta || !phi || !lambda || !dbeta)
        return set_error(MG_ERR_INVALID_ARG, "bad argument");
    CKO(launch_beta_grad(n[0], n[1], n[2], 1.0 / (h * h), bc, beta, phi, lambda, dbeta,
                         (cudaStream_t)stream));
    return MG_OK;
}

}  // extern "C"
