// solver.cu -- hierarchy set-up, V-cycle driver and the mg.h C ABI.
//
// The solve is the variable-coefficient Poisson equation of the paper's
// Sec. 1 (one per MAESTRO time step).  One Solver holds any number of
// independent boxes (the grids of a MultiFAB level, paper Sec. 2); mg_ctx is
// the one-box case.  Every V-cycle stage is one kernel launch over the tiles
// of all boxes still active at that level, and the whole cycle (plus the
// fine-level residual norm) is captured once as a CUDA graph and replayed.
#include "solver.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

namespace mg {

static thread_local char g_err[1024] = "";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return set_error(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,        \
                             "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,         \
                             __LINE__);                                                         \
    } while (0)

#define CKS(expr)                    \
    do {                             \
        int s_ = (expr);             \
        if (s_ != MG_OK) return s_;  \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Severity order used to report the worst status of several solves.
static int severity(int s)
{
    switch (s) {
    case MG_OK: return 0;
    case MG_ERR_NOT_CONVERGED: return 1;
    case MG_ERR_DIVERGED: return 2;
    case MG_ERR_NONFINITE: return 3;
    default: return 4;
    }
}
static int worse(int a, int b) { return severity(b) > severity(a) ? b : a; }

// Halve every dimension while all are even and at least 4.
static std::vector<std::array<int, 3>> level_dims(int nx, int ny, int nz)
{
    std::vector<std::array<int, 3>> d;
    d.push_back({nx, ny, nz});
    while (d.size() < 32 && nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 && nx >= 4 && ny >= 4 &&
           nz >= 4) {
        nx /= 2;
        ny /= 2;
        nz /= 2;
        d.push_back({nx, ny, nz});
    }
    return d;
}

// ------------------------------------------------------------ building ----

// Bump allocator over a byte arena (dry run computes the size).
struct Bump {
    char *base = nullptr;
    size_t used = 0;
    template <class T>
    T *take(size_t count)
    {
        used = (size_t)round_up((long long)used, 256);
        T *p = base ? reinterpret_cast<T *>(base + used) : nullptr;
        used += count * sizeof(T);
        return p;
    }
};

template <class T>
static void carve(Solver *s, Hier<T> &H, Bump &bump, bool full)
{
    H.lv.assign(s->nbox, {});
    H.ainv.assign(s->nbox, nullptr);
    for (int b = 0; b < s->nbox; ++b) {
        H.lv[b].resize(s->nlev[b]);
        for (int l = 0; l < s->nlev[b]; ++l) {
            const auto &d = s->dims[b][l];
            const long long E = level_elems(d[0], d[1], d[2]);
            const long long Q = pitch_plane(d[0], d[1]);
            auto arr = [&]() {
                T *p = bump.take<T>((size_t)E);
                return p ? p + Q : nullptr;
            };
            LevelBufs<T> &L = H.lv[b][l];
            L.wx = arr();
            L.wy = arr();
            L.wz = arr();
            L.invD = arr();
            if (sizeof(T) == sizeof(double)) L.D = arr();
            if (full || l == 0) {
                L.phi = arr();
                L.phi2 = arr();
                L.f = arr();
            }
        }
        const auto &db = s->dims[b][s->nlev[b] - 1];
        const size_t nb = (size_t)db[0] * db[1] * db[2];
        H.ainv[b] = bump.take<T>(nb * nb);
    }
}

template <class T>
static Box<T> make_box(const Solver *s, const Hier<T> &H, int b, int l)
{
    Box<T> B{};
    const LevelBufs<T> &L = H.lv[b][l];
    const auto &d = s->dims[b][l];
    B.phi = L.phi;
    B.phi2 = L.phi2;
    B.f = L.f;
    B.wx = L.wx;
    B.wy = L.wy;
    B.wz = L.wz;
    B.invD = L.invD;
    B.D = L.D;
    B.nx = d[0];
    B.ny = d[1];
    B.nz = d[2];
    B.P = (int)pitch_row(d[0]);
    B.Q = pitch_plane(d[0], d[1]);
    if (l + 1 < s->nlev[b]) {
        const LevelBufs<T> &C = H.lv[b][l + 1];
        const auto &c = s->dims[b][l + 1];
        B.phic = C.phi;
        B.fc = C.f;
        B.cP = (int)pitch_row(c[0]);
        B.cQ = pitch_plane(c[0], c[1]);
    }
    if (l == s->nlev[b] - 1) B.ainv = H.ainv[b];
    B.box = b;
    B.zc = kSweepZ;
    return B;
}

// Host image of the descriptor arena; sets are patched to device addresses
// after upload.
struct DescBlob {
    std::vector<char> bytes;
    size_t put(const void *p, size_t n)
    {
        size_t o = (size_t)round_up((long long)bytes.size(), 64);
        bytes.resize(o + n);
        if (n) memcpy(bytes.data() + o, p, n);
        return o;
    }
};

template <class T>
struct SetPlan {
    BoxSet<T> *target;
    size_t boxes_off;
    size_t ts_off[TK_NKIND];
};

template <class T>
static SetPlan<T> plan_set(DescBlob &blob, BoxSet<T> *target, const std::vector<Box<T>> &boxes)
{
    SetPlan<T> p{};
    p.target = target;
    *target = BoxSet<T>{};
    target->nbox = (int)boxes.size();
    p.boxes_off = blob.put(boxes.data(), boxes.size() * sizeof(Box<T>));
    for (int k = 0; k < TK_NKIND; ++k) {
        std::vector<int> ts(boxes.size() + 1, 0);
        for (size_t i = 0; i < boxes.size(); ++i)
            ts[i + 1] = ts[i] + tiles_of(k, boxes[i].nx, boxes[i].ny, boxes[i].nz,
                                         boxes[i].zc > 0 ? boxes[i].zc : kSweepZ);
        target->ntiles[k] = ts.back();
        p.ts_off[k] = blob.put(ts.data(), ts.size() * sizeof(int));
    }
    return p;
}

template <class T>
static void patch_set(const SetPlan<T> &p, char *dev)
{
    p.target->boxes = reinterpret_cast<const Box<T> *>(dev + p.boxes_off);
    for (int k = 0; k < TK_NKIND; ++k)
        p.target->tstart[k] = reinterpret_cast<const int *>(dev + p.ts_off[k]);
}

// Planes per CTA of the fused sweep for a set of boxes: the grid should fill
// whole waves of resident CTAs (a second, nearly empty wave doubles the time
// of a z-marching kernel), while short chunks pay one extra red half-plane
// per chunk boundary.  Returns the chunk length and its score (fraction of
// useful work, 1 = perfect).
template <class T>
static int choose_zc(const std::vector<Box<T>> &boxes, long long slots, double *score)
{
    int maxnz = 1;
    for (const auto &B : boxes) maxnz = std::max(maxnz, B.nz);
    int best = std::min(kSweepZ, maxnz);
    double best_s = -1.0;
    for (int Z = 2; Z <= maxnz; ++Z) {
        long long ctas = 0;
        for (const auto &B : boxes) ctas += tiles_of(TK_SWEEP, B.nx, B.ny, B.nz, Z);
        const long long waves = (ctas + slots - 1) / slots;
        const double fill = (double)ctas / (double)(waves * slots);
        const double sc = fill * (double)Z / (Z + 1.0);
        if (sc > best_s + 1e-9) {
            best_s = sc;
            best = Z;
        }
    }
    *score = best_s;
    return best;
}

// Cell limit of the levels run by the one-CTA coarse kernel.
template <class T>
static long long coarse_limit(const mg_opts &o)
{
    if (o.coarse_cells < 0) return -1;
    if (o.coarse_cells > 0) return o.coarse_cells;
    return sizeof(T) == sizeof(double) ? 1024 : 4096;
}

template <class T>
static void plan_hier(const Solver *s, Hier<T> &H, DescBlob &blob, std::vector<SetPlan<T>> &plans,
                      size_t *jobs_off)
{
    H.smooth.assign(std::max(s->maxlev - 1, 0), BoxSet<T>{});
    std::vector<Box<T>> fine, bottom;
    std::vector<CoarseJob<T>> jobs;
    const long long lim = coarse_limit<T>(s->opts);
    H.lc.assign(s->nbox, 0);
    for (int b = 0; b < s->nbox; ++b) {
        fine.push_back(make_box(s, H, b, 0));
        bottom.push_back(make_box(s, H, b, s->nlev[b] - 1));
        // first level small enough for the coarse kernel (the coarsest level
        // always is: it is solved there when the kernel is off)
        int lc = s->nlev[b] - 1;
        if (lim > 0) {
            for (int l = 0; l < s->nlev[b]; ++l) {
                const auto &d = s->dims[b][l];
                if ((long long)d[0] * d[1] * d[2] <= lim && s->nlev[b] - l <= kMaxCoarse) {
                    lc = l;
                    break;
                }
            }
        }
        H.lc[b] = lc;
        CoarseJob<T> J;
        memset(&J, 0, sizeof J);
        J.nlev = s->nlev[b] - lc;
        J.box = b;
        for (int l = lc; l < s->nlev[b]; ++l) J.lv[l - lc] = make_box(s, H, b, l);
        jobs.push_back(J);
    }
    plans.push_back(plan_set(blob, &H.fine, fine));
    plans.push_back(plan_set(blob, &H.bottom, bottom));
    H.fused.assign(H.smooth.size(), 0);
    const long long slots = (long long)s->sms * sweep_ctas_per_sm<T>();
    for (int l = 0; l + 1 < s->maxlev; ++l) {
        std::vector<Box<T>> set;
        for (int b = 0; b < s->nbox; ++b)
            if (l < H.lc[b]) set.push_back(make_box(s, H, b, l));
        if (!set.empty()) {
            double score = 0.0;
            const int zc = choose_zc(set, slots, &score);
            for (auto &B : set) B.zc = zc;
            // fused sweeps when the grid can keep the GPU busy
            const bool ok = score >= 0.7;
            H.fused[l] = s->opts.smoother == 2 || (s->opts.smoother == 0 && ok);
        }
        plans.push_back(plan_set(blob, &H.smooth[l], set));
    }
    H.njobs = (int)jobs.size();
    *jobs_off = blob.put(jobs.data(), jobs.size() * sizeof(CoarseJob<T>));
}

static int validate_opts(const mg_opts *o)
{
    if (o->precision != MG_FP64 && o->precision != MG_MIXED)
        return set_error(MG_ERR_INVALID_ARG, "precision must be MG_FP64 or MG_MIXED");
    if (o->nu1 < 0 || o->nu1 > 8 || o->nu2 < 0 || o->nu2 > 8 || o->nu1 + o->nu2 < 1)
        return set_error(MG_ERR_INVALID_ARG, "nu1, nu2 must be in 0..8 with nu1 + nu2 >= 1");
    if (o->max_cycles < 1 || o->max_cycles > 100000)
        return set_error(MG_ERR_INVALID_ARG, "max_cycles must be in 1..100000");
    if (o->smoother < 0 || o->smoother > 2)
        return set_error(MG_ERR_INVALID_ARG, "smoother must be 0, 1 or 2");
    return MG_OK;
}

int solver_create(Solver **out, int nbox, const int (*n)[3], const double *dx, int bc,
                  const mg_opts *opts)
{
    if (!out) return set_error(MG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nbox < 1 || !n || !dx) return set_error(MG_ERR_INVALID_ARG, "need nbox >= 1, n, dx");
    if (bc != MG_BC_DIRICHLET0)
        return set_error(MG_ERR_UNSUPPORTED, "only MG_BC_DIRICHLET0 is implemented");
    mg_opts o;
    mg_default_opts(&o);
    if (opts) o = *opts;
    CKS(validate_opts(&o));

    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    Solver *s = new Solver();
    s->dev = dev;
    s->sms = sms;
    s->nbox = nbox;
    s->opts = o;
    s->has32 = o.precision == MG_MIXED;
    s->off.assign(nbox + 1, 0);
    for (int b = 0; b < nbox; ++b) {
        const int nx = n[b][0], ny = n[b][1], nz = n[b][2];
        if (nx < 1 || ny < 1 || nz < 1 || !(dx[b] > 0.0) || !std::isfinite(dx[b])) {
            delete s;
            return set_error(MG_ERR_INVALID_ARG, "box %d: need n >= 1 and finite dx > 0", b);
        }
        if ((long long)nx * ny * nz > (1LL << 33)) {
            delete s;
            return set_error(MG_ERR_UNSUPPORTED, "box %d: more than 2^33 cells", b);
        }
        s->n.push_back({nx, ny, nz});
        s->dx.push_back(dx[b]);
        s->dims.push_back(level_dims(nx, ny, nz));
        s->nlev.push_back((int)s->dims.back().size());
        s->maxlev = std::max(s->maxlev, s->nlev.back());
        const auto &db = s->dims.back().back();
        const int cells = db[0] * db[1] * db[2];
        if (cells > MG_MAX_BOTTOM) {
            delete s;
            return set_error(MG_ERR_UNSUPPORTED,
                             "box %d: coarsest level %dx%dx%d has %d cells (> %d); the dims "
                             "must halve down to a small level",
                             b, db[0], db[1], db[2], cells, MG_MAX_BOTTOM);
        }
        s->max_bottom = std::max(s->max_bottom, cells);
        s->off[b + 1] = s->off[b] + (long long)nx * ny * nz;
    }
    s->total = s->off[nbox];

    // level arrays: dry run for the size, then carve the zero-filled arena
    Bump bump;
    carve(s, s->h64, bump, true);
    if (s->has32) carve(s, s->h32, bump, true);
    size_t work_elems = 0, ntiles0 = 0;
    for (int b = 0; b < nbox; ++b) {
        const auto &db = s->dims[b].back();
        const size_t nb = (size_t)db[0] * db[1] * db[2];
        work_elems = std::max(work_elems, nb * nb);
        ntiles0 += (size_t)tiles_of(TK_CELL, s->n[b][0], s->n[b][1], s->n[b][2]);
    }
    bump.take<double>(s->total);      // beta copy
    bump.take<double>(work_elems);    // inverse scratch
    bump.take<double>(ntiles0);       // partials
    for (int i = 0; i < 6; ++i) bump.take<double>(nbox);
    bump.take<int>(nbox);
    const size_t bytes = bump.used;
    cudaError_t e = cudaMalloc(&s->arena, bytes);
    if (e != cudaSuccess) {
        delete s;
        return set_error(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                         "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    e = cudaMemset(s->arena, 0, bytes);
    if (e != cudaSuccess) {
        solver_destroy(s);
        return set_error(MG_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
    }
    Bump real;
    real.base = s->arena;
    carve(s, s->h64, real, true);
    if (s->has32) carve(s, s->h32, real, true);
    s->beta = real.take<double>(s->total);
    s->work = real.take<double>(work_elems);
    s->partials = real.take<double>(ntiles0);
    s->dnorm = real.take<double>(nbox);
    s->dnormf = real.take<double>(nbox);
    s->dinv = real.take<double>(nbox);
    s->se = real.take<double>(nbox);
    s->sr = real.take<double>(nbox);
    s->sr_inv = real.take<double>(nbox);
    s->active = real.take<int>(nbox);

    // launch-set descriptors (+ packed offsets and side flags)
    DescBlob blob;
    std::vector<SetPlan<double>> p64;
    std::vector<SetPlan<float>> p32;
    size_t jobs64 = 0, jobs32 = 0;
    plan_hier(s, s->h64, blob, p64, &jobs64);
    if (s->has32) plan_hier(s, s->h32, blob, p32, &jobs32);
    const size_t off_at = blob.put(s->off.data(), s->off.size() * sizeof(long long));
    std::vector<int> zeros(nbox, 0);
    const size_t side_at = blob.put(zeros.data(), zeros.size() * sizeof(int));
    e = cudaMalloc(&s->desc, blob.bytes.size());
    if (e != cudaSuccess) {
        solver_destroy(s);
        return set_error(MG_ERR_OOM, "cudaMalloc(descriptors): %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(s->desc, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        solver_destroy(s);
        return set_error(MG_ERR_CUDA, "descriptor upload: %s", cudaGetErrorString(e));
    }
    for (auto &p : p64) patch_set(p, s->desc);
    for (auto &p : p32) patch_set(p, s->desc);
    s->h64.jobs = reinterpret_cast<const CoarseJob<double> *>(s->desc + jobs64);
    if (s->has32) s->h32.jobs = reinterpret_cast<const CoarseJob<float> *>(s->desc + jobs32);
    s->doff = reinterpret_cast<const long long *>(s->desc + off_at);
    s->dside = reinterpret_cast<int *>(s->desc + side_at);

    if (cudaMallocHost(&s->hnorm, sizeof(double) * 2 * nbox) != cudaSuccess ||
        cudaMallocHost(&s->hactive, sizeof(int) * nbox) != cudaSuccess ||
        cudaMallocHost(&s->hside, sizeof(int) * nbox) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&s->ev_setup0) != cudaSuccess ||
        cudaEventCreate(&s->ev_setup1) != cudaSuccess) {
        solver_destroy(s);
        return set_error(MG_ERR_CUDA, "host buffers / stream / events: %s",
                         cudaGetErrorString(cudaGetLastError()));
    }
    *out = s;
    return MG_OK;
}

void solver_destroy(Solver *s)
{
    if (!s) return;
    DeviceGuard g(s->dev);
    for (auto *v : {&s->slots64, &s->slots32, &s->direct})
        for (auto &sl : *v) {
            cudaEventDestroy(sl.b);
            cudaEventDestroy(sl.e);
        }
    for (auto e : s->ev_free) cudaEventDestroy(e);
    if (s->h64.graph) cudaGraphExecDestroy(s->h64.graph);
    if (s->h32.graph) cudaGraphExecDestroy(s->h32.graph);
    if (s->arena) cudaFree(s->arena);
    if (s->desc) cudaFree(s->desc);
    if (s->stage_a) cudaFree(s->stage_a);
    if (s->hnorm) cudaFreeHost(s->hnorm);
    if (s->hactive) cudaFreeHost(s->hactive);
    if (s->hside) cudaFreeHost(s->hside);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->ev_setup0) cudaEventDestroy(s->ev_setup0);
    if (s->ev_setup1) cudaEventDestroy(s->ev_setup1);
    delete s;
}

// ------------------------------------------------------------- pointers ----

static bool is_device_ptr(const void *p, int dev, bool *wrong_dev)
{
    cudaPointerAttributes a{};
    *wrong_dev = false;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) {
        *wrong_dev = a.device != dev;
        return true;
    }
    return a.type == cudaMemoryTypeManaged;
}

static int ensure_stage(Solver *s)
{
    if (s->stage_a) return MG_OK;
    CK(cudaMalloc(&s->stage_a, sizeof(double) * 3 * (size_t)s->total));
    s->stage_b = s->stage_a + s->total;
    s->stage_c = s->stage_b + s->total;
    return MG_OK;
}

static double *stage_buf(Solver *s, int which)
{
    return which == 0 ? s->stage_a : which == 1 ? s->stage_b : s->stage_c;
}

// Device view of a packed caller array: the pointer itself, or staging
// buffer `which` (0..2) holding a copy (copy_in: host -> stage on the stream).
static int device_view(Solver *s, const double *p, int which, bool copy_in, cudaStream_t st,
                       const double **dv, bool *staged)
{
    bool wrong = false;
    if (is_device_ptr(p, s->dev, &wrong)) {
        if (wrong) return set_error(MG_ERR_INVALID_ARG, "device pointer on another device");
        *dv = p;
        *staged = false;
        return MG_OK;
    }
    CKS(ensure_stage(s));
    double *stage = stage_buf(s, which);
    if (copy_in)
        CK(cudaMemcpyAsync(stage, p, sizeof(double) * s->total, cudaMemcpyHostToDevice, st));
    *dv = stage;
    *staged = true;
    return MG_OK;
}

// --------------------------------------------------------------- set-up ----

int solver_set_beta(Solver *s, const double *beta, cudaStream_t st)
{
    if (!s || !beta) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(s->dev);
    cudaGetLastError();  // drop a stale non-sticky error of an earlier call
    CK(cudaEventRecord(s->ev_setup0, st));
    const long long k0 = launch_counter();
    CK(cudaMemcpyAsync(s->beta, beta, sizeof(double) * s->total, cudaMemcpyDefault, st));
    for (int b = 0; b < s->nbox; ++b) {
        auto &L = s->h64.lv[b];
        const auto &d0 = s->dims[b][0];
        CK(launch_face_weights(d0[0], d0[1], d0[2], 1.0 / (s->dx[b] * s->dx[b]), s->beta + s->off[b],
                               L[0].wx, L[0].wy, L[0].wz, st));
        for (int l = 1; l < s->nlev[b]; ++l) {
            const auto &d = s->dims[b][l - 1];
            CK(launch_coarsen(d[0], d[1], d[2], L[l - 1].wx, L[l - 1].wy, L[l - 1].wz, L[l].wx,
                              L[l].wy, L[l].wz, st));
        }
        for (int l = 0; l < s->nlev[b]; ++l) {
            const auto &d = s->dims[b][l];
            CK(launch_inv_diag(d[0], d[1], d[2], L[l].wx, L[l].wy, L[l].wz, L[l].invD, L[l].D, st));
            if (s->has32) {
                auto &M = s->h32.lv[b][l];
                CK(launch_round_f32(d[0], d[1], d[2], L[l].wx, L[l].wy, L[l].wz, L[l].invD,
                                    const_cast<float *>(M.wx), const_cast<float *>(M.wy),
                                    const_cast<float *>(M.wz), const_cast<float *>(M.invD), st));
            }
        }
        const int lb = s->nlev[b] - 1;
        const auto &db = s->dims[b][lb];
        CK(launch_bottom_inverse(db[0], db[1], db[2], L[lb].wx, L[lb].wy, L[lb].wz, s->work,
                                 s->h64.ainv[b], s->has32 ? s->h32.ainv[b] : nullptr, st));
    }
    CK(cudaEventRecord(s->ev_setup1, st));
    s->kernels += launch_counter() - k0;
    s->beta_set = true;
    s->setup_pending = true;
    return MG_OK;
}

// ------------------------------------------------------------ profiling ----

static cudaEvent_t take_event(Solver *s)
{
    if (!s->ev_free.empty()) {
        cudaEvent_t e = s->ev_free.back();
        s->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static cudaError_t record(Solver *s, cudaEvent_t ev, cudaStream_t st)
{
    return s->capturing ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                        : cudaEventRecord(ev, st);
}

// Open a timed stretch of stage class `kind`; returns its slot or -1.
static int prof_begin(Solver *s, int kind, cudaStream_t st)
{
    if (!s->prof || !s->rec) return -1;
    ProfSlot sl{kind, take_event(s), take_event(s)};
    if (record(s, sl.b, st) != cudaSuccess) return -1;
    s->rec->push_back(sl);
    return (int)s->rec->size() - 1;
}

static void prof_end(Solver *s, int slot, cudaStream_t st)
{
    if (slot < 0 || !s->rec) return;
    record(s, (*s->rec)[slot].e, st);
}

// Add the times of all slots that ran since the last call (stream synced).
static void prof_collect(Solver *s)
{
    auto add = [&](const std::vector<ProfSlot> &v) {
        for (const auto &sl : v) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, sl.b, sl.e) == cudaSuccess) {
                s->prof_ms[sl.kind] += ms;
                s->prof_n[sl.kind] += 1;
            }
        }
    };
    for (auto *v : s->pending) add(*v);
    s->pending.clear();
    add(s->direct);
    for (auto &sl : s->direct) {
        s->ev_free.push_back(sl.b);
        s->ev_free.push_back(sl.e);
    }
    s->direct.clear();
    cudaGetLastError();
}

// ------------------------------------------------------------ the cycle ----

template <class T>
static cudaError_t smooth(Solver *s, const BoxSet<T> &S, int nu, bool fine, bool fused,
                          cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    int left = nu;
    if (fused) {
        for (; left >= 2; left -= 2) {
            for (int src = 0; src < 2; ++src) {
                int sl = fine ? prof_begin(s, MG_PROF_SWEEP, st) : -1;
                if ((e = launch_rbgs_sweep(S, s->active, src, st)) != cudaSuccess) return e;
                prof_end(s, sl, st);
            }
        }
    }
    for (; left > 0; --left) {
        for (int color = 0; color < 2; ++color) {
            int sl = fine ? prof_begin(s, MG_PROF_PASS, st) : -1;
            if ((e = launch_rbgs_pass(S, s->active, color, st)) != cudaSuccess) return e;
            prof_end(s, sl, st);
        }
    }
    return e;
}

template <class T>
static cudaError_t enqueue_vcycle(Solver *s, const Hier<T> &H, cudaStream_t st)
{
    cudaError_t e;
    const int nl = (int)H.smooth.size();
    int coarse = -1;
    for (int l = 0; l < nl; ++l) {
        const BoxSet<T> &S = H.smooth[l];
        if (S.nbox == 0) continue;
        if ((e = smooth(s, S, s->opts.nu1, l == 0, H.fused[l] != 0, st)) != cudaSuccess) return e;
        int sl = l == 0 ? prof_begin(s, MG_PROF_RESTRICT, st) : -1;
        if ((e = launch_resid_restrict(S, s->active, st)) != cudaSuccess) return e;
        prof_end(s, sl, st);
        if (l == 0) coarse = prof_begin(s, MG_PROF_COARSE, st);
    }
    if (nl == 0 || H.smooth[0].nbox == 0) coarse = prof_begin(s, MG_PROF_COARSE, st);
    if ((e = launch_coarse_vcycle(H.jobs, H.njobs, s->active, s->opts.nu1, s->opts.nu2, st)) !=
        cudaSuccess)
        return e;
    for (int l = nl - 1; l >= 0; --l) {
        const BoxSet<T> &S = H.smooth[l];
        if (S.nbox == 0) continue;
        if (l == 0) {
            prof_end(s, coarse, st);
            coarse = -1;
        }
        int sl = l == 0 ? prof_begin(s, MG_PROF_PROLONG, st) : -1;
        if ((e = launch_prolong(S, s->active, st)) != cudaSuccess) return e;
        prof_end(s, sl, st);
        if ((e = smooth(s, S, s->opts.nu2, l == 0, H.fused[l] != 0, st)) != cudaSuccess) return e;
    }
    prof_end(s, coarse, st);
    return cudaSuccess;
}

// FP64: V-cycle followed by the fine residual norm into dnorm.
static cudaError_t enqueue_step64(Solver *s, cudaStream_t st)
{
    cudaError_t e = enqueue_vcycle(s, s->h64, st);
    if (e != cudaSuccess) return e;
    int sl = prof_begin(s, MG_PROF_NORM, st);
    if ((e = launch_norm_partials(s->h64.fine, s->active, 0, s->partials, st)) != cudaSuccess)
        return e;
    e = launch_norm_finish(s->h64.fine, s->active, s->partials, s->dnorm, nullptr, nullptr, st);
    prof_end(s, sl, st);
    return e;
}

// Mixed: zero the FP32 correction, FP32 V-cycle on r32.
static cudaError_t enqueue_step32(Solver *s, cudaStream_t st)
{
    cudaError_t e = launch_zero(s->h32.fine, s->active, st);
    if (e != cudaSuccess) return e;
    return enqueue_vcycle(s, s->h32, st);
}

template <class F>
static int run_step(Solver *s, cudaGraphExec_t *graph, std::vector<ProfSlot> *slots,
                    long long *graph_kernels, F enqueue, cudaStream_t st)
{
    if (!s->opts.use_graph) {
        s->rec = &s->direct;
        cudaError_t e = enqueue(s, st);
        s->rec = nullptr;
        CK(e);
        return MG_OK;
    }
    if (*graph && s->graph_prof != s->prof) {
        // re-capture with (or without) the event nodes
        cudaGraphExecDestroy(s->h64.graph);
        s->h64.graph = nullptr;
        if (s->h32.graph) cudaGraphExecDestroy(s->h32.graph);
        s->h32.graph = nullptr;
        for (auto *v : {&s->slots64, &s->slots32}) {
            for (auto &sl : *v) {
                s->ev_free.push_back(sl.b);
                s->ev_free.push_back(sl.e);
            }
            v->clear();
        }
    }
    if (!*graph) {
        cudaGraph_t gr = nullptr;
        s->graph_prof = s->prof;
        CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
        const long long k0 = launch_counter();
        s->rec = slots;
        s->capturing = true;
        cudaError_t e = enqueue(s, s->cap);
        s->capturing = false;
        s->rec = nullptr;
        *graph_kernels = launch_counter() - k0;
        s->cap_kernels += *graph_kernels;
        cudaError_t e2 = cudaStreamEndCapture(s->cap, &gr);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            return set_error(MG_ERR_CUDA, "V-cycle capture: %s",
                             cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(graph, gr, 0);
        cudaGraphDestroy(gr);
        CK(e);
    }
    CK(cudaGraphLaunch(*graph, st));
    s->kernels += *graph_kernels;
    if (s->prof) s->pending.push_back(slots);
    return MG_OK;
}

#define RUN64(s, st) run_step(s, &(s)->h64.graph, &(s)->slots64, &(s)->graph_kernels64, enqueue_step64, st)
#define RUN32(s, st) run_step(s, &(s)->h32.graph, &(s)->slots32, &(s)->graph_kernels32, enqueue_step32, st)

// Per-box bookkeeping of the convergence loop.
struct BoxState {
    int status = MG_ERR_NOT_CONVERGED;
    bool done = false;
    double nf = 0.0, rel0 = 0.0, best = 0.0;
    int stall = 0, cycles = 0;
    double hist[MG_MAX_HIST];
    int nh = 0;
};

// Judge box b after a cycle with relative residual rel; returns true if done.
static bool judge(BoxState &B, double rel, double tol, int cycle, int max_cycles)
{
    if (B.nh < MG_MAX_HIST) B.hist[B.nh++] = rel;
    B.cycles = cycle;
    if (!std::isfinite(rel)) { B.status = MG_ERR_NONFINITE; return true; }
    if (rel <= tol) { B.status = MG_OK; return true; }
    if (rel > 1e3 * std::max(B.rel0, tol)) { B.status = MG_ERR_DIVERGED; return true; }
    if (rel > 0.9 * B.best) ++B.stall;
    else B.stall = 0;
    B.best = std::min(B.best, rel);
    if (B.stall >= 5 || cycle >= max_cycles) { B.status = MG_ERR_NOT_CONVERGED; return true; }
    return false;
}

static int upload_active(Solver *s, const std::vector<BoxState> &bs, cudaStream_t st)
{
    for (int b = 0; b < s->nbox; ++b) s->hactive[b] = bs[b].done ? 0 : 1;
    CK(cudaMemcpyAsync(s->active, s->hactive, sizeof(int) * s->nbox, cudaMemcpyHostToDevice, st));
    return MG_OK;
}

static int read_norms(Solver *s, const double *dev, double *host, cudaStream_t st)
{
    CK(cudaMemcpyAsync(host, dev, sizeof(double) * s->nbox, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return MG_OK;
}

int solver_solve(Solver *s, const double *f, double *phi, double tol, mg_stats *st,
                 cudaStream_t stream, bool zero_guess)
{
    if (!s || !f || !phi) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    if (!(tol > 0.0)) return set_error(MG_ERR_INVALID_ARG, "tol must be > 0");
    if (!s->beta_set) return set_error(MG_ERR_INVALID_ARG, "mg_set_beta was not called");
    DeviceGuard g(s->dev);
    cudaGetLastError();  // drop a stale non-sticky error of an earlier call
    const auto t0 = std::chrono::steady_clock::now();
    const long long k0 = launch_counter(), c0 = s->cap_kernels;
    const int nbox = s->nbox;
    const bool mixed = s->has32;
    Hier<double> &H = s->h64;

    // inputs into the level layout
    const double *fd = nullptr, *pd = nullptr;
    bool fst = false, pst = false;
    CKS(device_view(s, f, 0, true, stream, &fd, &fst));
    CK(launch_pack(H.fine, s->doff, fd, 1, stream));
    for (int b = 0; b < nbox; ++b) s->hactive[b] = 1;
    CK(cudaMemcpyAsync(s->active, s->hactive, sizeof(int) * nbox, cudaMemcpyHostToDevice, stream));
    if (zero_guess) {
        CK(launch_zero(H.fine, nullptr, stream));
    } else {
        CKS(device_view(s, phi, 1, true, stream, &pd, &pst));
        CK(launch_pack(H.fine, s->doff, pd, 0, stream));
    }
    // ||f|| and the starting residual
    CK(launch_norm_partials(H.fine, nullptr, 1, s->partials, stream));
    CK(launch_norm_finish(H.fine, nullptr, s->partials, s->dnormf, nullptr, nullptr, stream));
    CK(launch_norm_partials(H.fine, nullptr, 0, s->partials, stream));
    CK(launch_norm_finish(H.fine, nullptr, s->partials, s->dnorm, nullptr, nullptr, stream));
    CK(cudaMemcpyAsync(s->hnorm, s->dnormf, sizeof(double) * nbox, cudaMemcpyDeviceToHost, stream));
    CKS(read_norms(s, s->dnorm, s->hnorm + nbox, stream));

    std::vector<BoxState> bs(nbox);
    std::vector<int> side(nbox, 0);
    bool any = false;
    for (int b = 0; b < nbox; ++b) {
        BoxState &B = bs[b];
        B.nf = s->hnorm[b];
        const double r0 = s->hnorm[nbox + b];
        if (!std::isfinite(B.nf) || !std::isfinite(r0)) {
            B.status = MG_ERR_NONFINITE;
            B.done = true;
            continue;
        }
        if (B.nf == 0.0) {
            B.status = MG_OK;
            B.done = true;
            B.rel0 = 0.0;
            B.hist[B.nh++] = 0.0;
            continue;
        }
        B.rel0 = B.best = r0 / B.nf;
        B.hist[B.nh++] = B.rel0;
        if (B.rel0 <= tol) {
            B.status = MG_OK;
            B.done = true;
        } else {
            any = true;
        }
    }
    // zero right-hand side: the solution is zero
    for (int b = 0; b < nbox; ++b) s->hactive[b] = bs[b].nf == 0.0 ? 1 : 0;
    CK(cudaMemcpyAsync(s->active, s->hactive, sizeof(int) * nbox, cudaMemcpyHostToDevice, stream));
    CK(launch_zero(H.fine, s->active, stream));
    CKS(upload_active(s, bs, stream));

    if (!mixed) {
        for (int c = 1; any; ++c) {
            CKS(RUN64(s, stream));
            CKS(read_norms(s, s->dnorm, s->hnorm, stream));
            if (s->prof) prof_collect(s);
            bool changed = false;
            any = false;
            for (int b = 0; b < nbox; ++b) {
                if (bs[b].done) continue;
                if (judge(bs[b], s->hnorm[b] / bs[b].nf, tol, c, s->opts.max_cycles)) {
                    bs[b].done = true;
                    changed = true;
                } else {
                    any = true;
                }
            }
            if (changed && any) CKS(upload_active(s, bs, stream));
        }
    } else {
        // FP64 iterative refinement around FP32 V-cycles: step k forms
        // x_k = x_{k-1} + se e (e from the last FP32 cycle; nothing at k = 0),
        // the FP64 residual r_k = f - A x_k, r32 = r_k / sr for the next
        // cycle and ||r_k|| = sr ||r32||.
        CK(launch_zero(s->h32.fine, nullptr, stream));
        CK(launch_scales(nbox, s->active, 1, s->dnorm, s->dnormf, s->se, s->sr, s->sr_inv, stream));
        for (int k = 0; any; ++k) {
            s->rec = &s->direct;
            const int sl = prof_begin(s, MG_PROF_REFINE, stream);
            if (k > 0) CK(launch_refine_update(H.fine, s->h32.fine, s->active, s->se, stream));
            CK(launch_refine_residual(H.fine, s->h32.fine, s->active, s->sr_inv, s->partials,
                                      stream));
            CK(launch_norm_finish(H.fine, s->active, s->partials, s->dnorm, nullptr, nullptr,
                                  stream, s->sr));
            prof_end(s, sl, stream);
            s->rec = nullptr;
            CK(launch_scales(nbox, s->active, 0, s->dnorm, s->dnormf, s->se, s->sr, s->sr_inv,
                             stream));
            CKS(read_norms(s, s->dnorm, s->hnorm, stream));
            if (s->prof) prof_collect(s);
            bool changed = false;
            any = false;
            for (int b = 0; b < nbox; ++b) {
                if (bs[b].done) continue;
                // step 0 only forms the starting residual
                if (k == 0) {
                    any = true;
                    continue;
                }
                if (judge(bs[b], s->hnorm[b] / bs[b].nf, tol, k, s->opts.max_cycles)) {
                    bs[b].done = true;
                    changed = true;
                } else {
                    any = true;
                }
            }
            if (!any) break;
            if (changed) CKS(upload_active(s, bs, stream));
            CKS(RUN32(s, stream));
        }
    }

    // solution out
    for (int b = 0; b < nbox; ++b) s->hside[b] = side[b];
    CK(cudaMemcpyAsync(s->dside, s->hside, sizeof(int) * nbox, cudaMemcpyHostToDevice, stream));
    bool wrong = false;
    if (is_device_ptr(phi, s->dev, &wrong)) {
        if (wrong) return set_error(MG_ERR_INVALID_ARG, "phi on another device");
        CK(launch_unpack(H.fine, s->doff, phi, s->dside, stream));
    } else {
        CKS(ensure_stage(s));
        CK(launch_unpack(H.fine, s->doff, s->stage_b, s->dside, stream));
        CK(cudaMemcpyAsync(phi, s->stage_b, sizeof(double) * s->total, cudaMemcpyDeviceToHost,
                           stream));
    }
    CK(cudaStreamSynchronize(stream));
    (void)fst;
    (void)pst;
    s->kernels += (launch_counter() - k0) - (s->cap_kernels - c0);

    if (s->setup_pending) {
        cudaEventElapsedTime(&s->t_setup_ms, s->ev_setup0, s->ev_setup1);
        s->setup_pending = false;
    }
    const float ms =
        std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    int worst = MG_OK;
    for (int b = 0; b < nbox; ++b) {
        worst = worse(worst, bs[b].status);
        if (st) {
            mg_stats &o = st[b];
            memset(&o, 0, sizeof o);
            o.cycles = bs[b].cycles;
            o.status = bs[b].status;
            o.norm_f = bs[b].nf;
            o.rel_resid0 = bs[b].rel0;
            o.rel_resid = bs[b].nh ? bs[b].hist[bs[b].nh - 1] : 0.0;
            for (int i = 0; i < bs[b].nh; ++i) o.hist[i] = bs[b].hist[i];
            o.t_setup_ms = s->t_setup_ms;
            o.t_solve_ms = ms;
        }
    }
    if (worst != MG_OK)
        set_error(worst, "solve finished with status %d (%s)", worst, mg_error_string(worst));
    return worst;
}

// --------------------------------------------------------------- adjoint ----

int solver_adjoint(Solver *s, int nrhs, const double *phi, const double *g, double *dLdf,
                   double *dLdbeta, double tol, mg_stats *st, cudaStream_t stream)
{
    if (!s || !phi || !g || !dLdf || !dLdbeta || nrhs < 1)
        return set_error(MG_ERR_INVALID_ARG, "NULL argument or nrhs < 1");
    DeviceGuard gd(s->dev);
    cudaGetLastError();  // drop a stale non-sticky error of an earlier call
    int worst = MG_OK;
    const double *dbd = nullptr;
    bool dbst = false;
    CKS(device_view(s, dLdbeta, 2, true, stream, &dbd, &dbst));
    double *db = const_cast<double *>(dbd);
    for (int r = 0; r < nrhs; ++r) {
        const size_t o = (size_t)r * s->total;
        int rc = solver_solve(s, g + o, dLdf + o, tol, st ? st + (size_t)r * s->nbox : nullptr,
                              stream, true);
        if (rc != MG_OK && rc != MG_ERR_NOT_CONVERGED && rc != MG_ERR_DIVERGED) return rc;
        worst = worse(worst, rc);
        // lambda sits in the level-0 phi arrays; phi of this right-hand side
        CKS(ensure_stage(s));
        CK(launch_unpack(s->h64.fine, s->doff, s->stage_b, s->dside, stream));
        s->kernels += 1;
        const double *pd = nullptr;
        bool pst = false;
        CKS(device_view(s, phi + o, 0, true, stream, &pd, &pst));
        for (int b = 0; b < s->nbox; ++b) {
            const auto &d = s->n[b];
            s->kernels += 1;
            CK(launch_beta_grad(d[0], d[1], d[2], 1.0 / (s->dx[b] * s->dx[b]), s->beta + s->off[b],
                                pd + s->off[b], s->stage_b + s->off[b], db + s->off[b], stream));
        }
    }
    if (dbst)
        CK(cudaMemcpyAsync(dLdbeta, db, sizeof(double) * s->total, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (worst != MG_OK) set_error(worst, "adjoint solve status %d", worst);
    return worst;
}

}  // namespace mg

// ================================================================ C ABI ====

using namespace mg;

struct mg_ctx {
    Solver *s;
};
struct mg_batch {
    Solver *s;
};

extern "C" {

void mg_default_opts(mg_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = MG_FP64;
    o->nu1 = 2;
    o->nu2 = 2;
    o->max_cycles = 100;
    o->use_graph = 1;
    o->smoother = 0;
}

int mg_create(mg_ctx **out, const int n[3], double dx, int bc, const mg_opts *opts)
{
    if (!out || !n) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    int nn[1][3] = {{n[0], n[1], n[2]}};
    Solver *s = nullptr;
    int rc = solver_create(&s, 1, nn, &dx, bc, opts);
    if (rc != MG_OK) return rc;
    *out = new mg_ctx{s};
    return MG_OK;
}

int mg_set_beta(mg_ctx *ctx, const double *beta, void *stream)
{
    if (!ctx) return set_error(MG_ERR_INVALID_ARG, "NULL context");
    return solver_set_beta(ctx->s, beta, (cudaStream_t)stream);
}

int mg_solve(mg_ctx *ctx, const double *f, double *phi, double tol, mg_stats *st, void *stream)
{
    if (!ctx) return set_error(MG_ERR_INVALID_ARG, "NULL context");
    return solver_solve(ctx->s, f, phi, tol, st, (cudaStream_t)stream, false);
}

int mg_solve_multi(mg_ctx *ctx, int nrhs, const double *f, double *phi, double tol, mg_stats *st,
                   void *stream)
{
    if (!ctx || nrhs < 1 || !f || !phi)
        return set_error(MG_ERR_INVALID_ARG, "NULL argument or nrhs < 1");
    int worst = MG_OK;
    const size_t n = (size_t)ctx->s->total;
    for (int r = 0; r < nrhs; ++r) {
        int rc = solver_solve(ctx->s, f + r * n, phi + r * n, tol, st ? st + r : nullptr,
                              (cudaStream_t)stream, false);
        if (rc != MG_OK && rc != MG_ERR_NOT_CONVERGED && rc != MG_ERR_DIVERGED &&
            rc != MG_ERR_NONFINITE)
            return rc;
        worst = worse(worst, rc);
    }
    return worst;
}

int mg_adjoint(mg_ctx *ctx, int nrhs, const double *phi, const double *g, double *dLdf,
               double *dLdbeta, double tol, mg_stats *st, void *stream)
{
    if (!ctx) return set_error(MG_ERR_INVALID_ARG, "NULL context");
    return solver_adjoint(ctx->s, nrhs, phi, g, dLdf, dLdbeta, tol, st, (cudaStream_t)stream);
}

int mg_levels(const mg_ctx *ctx, int *nlev, int *dims)
{
    if (!ctx || !nlev) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    const Solver *s = ctx->s;
    *nlev = s->nlev[0];
    if (dims)
        for (int l = 0; l < s->nlev[0]; ++l)
            for (int d = 0; d < 3; ++d) dims[3 * l + d] = s->dims[0][l][d];
    return MG_OK;
}

void mg_destroy(mg_ctx *ctx)
{
    if (!ctx) return;
    solver_destroy(ctx->s);
    delete ctx;
}

int mg_batch_create(mg_batch **out, int nbox, const int (*n)[3], const double *dx, int bc,
                    const mg_opts *opts)
{
    if (!out) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    Solver *s = nullptr;
    int rc = solver_create(&s, nbox, n, dx, bc, opts);
    if (rc != MG_OK) return rc;
    *out = new mg_batch{s};
    return MG_OK;
}

int mg_batch_set_beta(mg_batch *b, const double *beta, void *stream)
{
    if (!b) return set_error(MG_ERR_INVALID_ARG, "NULL batch");
    return solver_set_beta(b->s, beta, (cudaStream_t)stream);
}

int mg_solve_batched(mg_batch *b, const double *f, double *phi, double tol, mg_stats *st,
                     void *stream)
{
    if (!b) return set_error(MG_ERR_INVALID_ARG, "NULL batch");
    return solver_solve(b->s, f, phi, tol, st, (cudaStream_t)stream, false);
}

void mg_batch_destroy(mg_batch *b)
{
    if (!b) return;
    solver_destroy(b->s);
    delete b;
}

static int profile_enable(Solver *s, int on)
{
    s->prof = on != 0;
    return MG_OK;
}

static int profile_read(Solver *s, mg_profile *out, int reset)
{
    if (!out) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    memset(out, 0, sizeof *out);
    for (int k = 0; k < MG_PROF_NKIND; ++k) {
        out->ms[k] = s->prof_ms[k];
        out->launches[k] = s->prof_n[k];
        out->cells[k] = k == MG_PROF_COARSE ? 0 : s->total;
    }
    out->kernels = s->kernels;
    if (reset) {
        memset(s->prof_ms, 0, sizeof s->prof_ms);
        memset(s->prof_n, 0, sizeof s->prof_n);
        s->kernels = 0;
    }
    return MG_OK;
}

int mg_profile_enable(mg_ctx *ctx, int on)
{
    if (!ctx) return set_error(MG_ERR_INVALID_ARG, "NULL context");
    return profile_enable(ctx->s, on);
}

int mg_profile_read(mg_ctx *ctx, mg_profile *out, int reset)
{
    if (!ctx) return set_error(MG_ERR_INVALID_ARG, "NULL context");
    return profile_read(ctx->s, out, reset);
}

int mg_batch_profile_enable(mg_batch *b, int on)
{
    if (!b) return set_error(MG_ERR_INVALID_ARG, "NULL batch");
    return profile_enable(b->s, on);
}

int mg_batch_profile_read(mg_batch *b, mg_profile *out, int reset)
{
    if (!b) return set_error(MG_ERR_INVALID_ARG, "NULL batch");
    return profile_read(b->s, out, reset);
}

const char *mg_error_string(int s)
{
    switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_NOT_CONVERGED: return "not converged";
    case MG_ERR_DIVERGED: return "diverged";
    case MG_ERR_NONFINITE: return "non-finite value";
    case MG_ERR_TIMEOUT: return "device wait timed out";
    case MG_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

const char *mg_last_error(void) { return g_err; }

}  // extern "C"
