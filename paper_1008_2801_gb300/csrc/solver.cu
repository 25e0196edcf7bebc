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

// CG on a coarsest level too large for a dense inverse: stop when
// <r, D^-1 r> has fallen by tol^2 or after the iteration cap (FP64 / FP32
// levels; FP32 rounding stalls the residual near sqrt(cond) x 6e-8, so the
// FP32 cycles of mixed precision stop earlier, which only costs cycles);
// kCgPartials bounds the CTAs of its launch.
constexpr double kCgTol64 = 1e-12, kCgTol32 = 1e-5;
constexpr int kCgMaxIt64 = 20000, kCgMaxIt32 = 3000;
constexpr int kCgPartials = 4096;
// Mixed precision with adaptive inner cycles (mg_opts.inner_cycles = 0): at
// most kInnerMax FP32 V-cycles per refinement step, a box leaving them once
// its update is expected to meet tol / 2, or its inner residual has dropped
// by kInnerFloor (the most a step asks of FP32 arithmetic)
constexpr int kInnerMax = 8;
constexpr double kInnerFloor = 1e-6;
constexpr int kInnerFixed = 2;   // inner cycles per step where the test is not available
constexpr int kInnerChunk = 64;  // restriction tiles per first-stage sum of the exit test

// ------------------------------------------------------------ building ----

// Device memory of a context: the caller's allocator when given, else
// cudaMalloc / cudaFree.
static cudaError_t dev_malloc(const Solver *s, void **p, size_t bytes)
{
    if (s->opts.dev_alloc) {
        *p = s->opts.dev_alloc(bytes, s->opts.alloc_user);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
static void dev_free(const Solver *s, void *p)
{
    if (!p) return;
    if (s->opts.dev_free) s->opts.dev_free(p, s->opts.alloc_user);
    else cudaFree(p);
}

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
            const long long E = level_elems(d[0], d[1], d[2], s->wide);
            const long long Q = pitch_plane(d[0], d[1], s->wide);
            auto arr = [&]() {
                T *p = bump.take<T>((size_t)E);
                return p ? p + Q : nullptr;
            };
            LevelBufs<T> &L = H.lv[b][l];
            if (s->shared && b > 0) {
                const LevelBufs<T> &Z = H.lv[0][l];
                L.wx = Z.wx;
                L.wy = Z.wy;
                L.wz = Z.wz;
                L.invD = Z.invD;
                L.D = Z.D;
            } else {
                L.wx = arr();
                L.wy = arr();
                L.wz = arr();
                L.invD = arr();
                if (sizeof(T) == sizeof(double)) L.D = arr();
            }
            if (full || l == 0) {
                L.phi = arr();
                L.phi2 = arr();
                L.f = arr();
            }
        }
        const auto &db = s->dims[b][s->nlev[b] - 1];
        const size_t nb = (size_t)db[0] * db[1] * db[2];
        if (s->cg_bottom) {
            // no dense inverse: p and q of the CG on the coarsest level
            const long long E = level_elems(db[0], db[1], db[2]);
            const long long Q = pitch_plane(db[0], db[1]);
            T *pp = bump.take<T>((size_t)E), *qq = bump.take<T>((size_t)E);
            H.cgp = pp ? pp + Q : nullptr;
            H.cgq = qq ? qq + Q : nullptr;
        } else if (!s->xmode) {
            H.ainv[b] = (s->shared && b > 0) ? H.ainv[0] : bump.take<T>(nb * nb);
        }
    }
    if (s->xmode) H.uinv = bump.take<T>((size_t)s->ub.n * s->ub.n);
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
    B.P = (int)pitch_row(d[0], s->wide);
    B.Q = pitch_plane(d[0], d[1], s->wide);
    if (l + 1 < s->nlev[b]) {
        const LevelBufs<T> &C = H.lv[b][l + 1];
        const auto &c = s->dims[b][l + 1];
        B.phic = C.phi;
        B.fc = C.f;
        B.cP = (int)pitch_row(c[0], s->wide);
        B.cQ = pitch_plane(c[0], c[1], s->wide);
    }
    if (l == s->nlev[b] - 1) B.ainv = s->xmode ? H.uinv : H.ainv[b];
    B.box = b;
    B.zc = kSweepZ;
    if (s->xmode) {
        auto parity = [&](int lev) {
            const auto &o = s->lo[b][lev];
            return (((o[0] + o[1] + o[2]) % 2) + 2) % 2;
        };
        B.par = parity(l);
        if (l + 1 < s->nlev[b]) B.cpar = parity(l + 1);
    }
    // FP64 levels keep f, 1/D and D colour-split: a single-colour pass then
    // reads only its own colour's sectors of them
    B.rb = sizeof(T) == sizeof(double) ? 1 : 0;
    return B;
}

// Host image of the descriptor arena; sets are patched to device addresses
// after upload.
struct DescBlob {
    std::vector<char> bytes;
    size_t put(const void *p, size_t n, int align = 64)
    {
        size_t o = (size_t)round_up((long long)bytes.size(), align);
        bytes.resize(o + n);
        if (n) memcpy(bytes.data() + o, p, n);
        return o;
    }
};

template <class D>
struct SetPlan {
    DescSet<D> *target;
    size_t boxes_off;
    size_t ts_off[TK_NKIND];
};

template <class D>
static SetPlan<D> plan_set(DescBlob &blob, DescSet<D> *target, const std::vector<D> &boxes)
{
    SetPlan<D> p{};
    p.target = target;
    *target = DescSet<D>{};
    target->nbox = (int)boxes.size();
    p.boxes_off = blob.put(boxes.data(), boxes.size() * sizeof(D));
    for (int k = 0; k < TK_NKIND; ++k) {
        std::vector<int> ts(boxes.size() + 1, 0);
        for (size_t i = 0; i < boxes.size(); ++i) {
            const int zc = boxes[i].zc > 0 ? boxes[i].zc : kSweepZ;
            ts[i + 1] = ts[i] + tiles_of(k, boxes[i].nx, boxes[i].ny, boxes[i].nz, zc);
            int ex, ey, ez;
            tile_extent(k, boxes[i].nx, boxes[i].ny, boxes[i].nz, ex, ey, ez, zc);
            if (tile_flat(k, ex)) target->flat |= 1 << k;
        }
        target->ntiles[k] = ts.back();
        p.ts_off[k] = blob.put(ts.data(), ts.size() * sizeof(int));
    }
    return p;
}

template <class D>
static void patch_set(const SetPlan<D> &p, char *dev)
{
    p.target->boxes = reinterpret_cast<const D *>(dev + p.boxes_off);
    for (int k = 0; k < TK_NKIND; ++k)
        p.target->tstart[k] = reinterpret_cast<const int *>(dev + p.ts_off[k]);
}

// Planes per CTA of the fused sweep for a set of boxes.  A z-marching CTA
// takes zc + 2 steps (the planes below and above its chunk included), and the
// CTAs run in waves of `slots` resident ones, so the sweep takes about
// waves * (zc + 2) steps.  For each chunk count m the shortest chunk length
// is ceil(nz / m) (equal chunks; a longer one only lengthens the critical
// path); the m with the fewest steps wins.  Returns zc and its efficiency
// (steps of useful plane work per resident slot over steps taken, 1 = perfect).
template <class T>
static int choose_zc(const std::vector<Box<T>> &boxes, long long slots, double *score)
{
    int maxnz = 1;
    double planes = 0.0;  // tile-planes of useful work
    for (const auto &B : boxes) {
        maxnz = std::max(maxnz, B.nz);
        planes += (double)tiles_of(TK_SWEEP, B.nx, B.ny, B.nz, B.nz) * B.nz;
    }
    int best = std::min(kSweepZ, maxnz);
    double best_cost = -1.0;
    int last = -1;
    for (int m = 1; m <= maxnz; ++m) {
        const int Z = (maxnz + m - 1) / m;
        if (Z == last) continue;
        last = Z;
        long long ctas = 0;
        for (const auto &B : boxes) ctas += tiles_of(TK_SWEEP, B.nx, B.ny, B.nz, Z);
        const long long waves = (ctas + slots - 1) / slots;
        const double cost = (double)waves * (Z + 2);
        if (best_cost < 0.0 || cost < best_cost - 1e-9) {
            best_cost = cost;
            best = Z;
        }
    }
    *score = planes / ((double)slots * best_cost);
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

// Tensor maps of every box of an FP32 level set (TMA sweep); false if the
// driver cannot encode them.
// TMA maps of a level's boxes; *prol: they also hold each box's coarse phi
// (the fused prolongation), which every box's coarse level must allow.
template <class T>
static bool plan_maps(const std::vector<Box<T>> &set, DescBlob &blob, size_t *off, bool *prol)
{
    *prol = false;
    if (sizeof(T) != sizeof(float)) return false;
    bool cp = true;
    for (const Box<T> &B : set) {
        if (!sweep_tma_fits(B.nx, B.ny)) return false;
        cp = cp && B.phic && sweep_tma_prol_fits(B.nx, B.ny, B.nx / 2, B.ny / 2) &&
             B.nz % 2 == 0;
    }
    const size_t one = sweep_maps_size();
    std::vector<char> bytes(one * set.size() + 128);   // tensor maps are 128-byte aligned
    char *base = reinterpret_cast<char *>(round_up((long long)(uintptr_t)bytes.data(), 128));
    for (size_t i = 0; i < set.size(); ++i) {
        const Box<T> &B = set[i];
        const long long Q = B.Q;
        auto lb = [&](const T *p) { return reinterpret_cast<const float *>(p - Q); };
        const float *pc = cp ? reinterpret_cast<const float *>(B.phic - B.cQ) : nullptr;
        if (!encode_sweep_maps(reinterpret_cast<SweepMaps *>(base + i * one), B.nx, B.ny, B.nz,
                               lb(B.phi), lb(B.phi2), lb(B.f), lb(B.wx), lb(B.wy), lb(B.wz), pc,
                               B.nx / 2, B.ny / 2, B.nz / 2))
            return false;
    }
    *off = blob.put(base, one * set.size(), 128);
    *prol = cp;
    return true;
}

template <class T>
static void plan_hier(Solver *s, Hier<T> &H, DescBlob &blob,
                      std::vector<SetPlan<Box<T>>> &plans, size_t *jobs_off,
                      std::vector<std::pair<int, size_t>> *map_offs)
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
        if (lim > 0 && !s->cg_bottom) {
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
    H.maps.assign(H.smooth.size(), nullptr);
    H.prol.assign(H.smooth.size(), 0);
    const bool tma = sizeof(T) == sizeof(float) && s->tma;
    const long long slots =
        (long long)s->sms * (tma ? sweep_tma_ctas_per_sm() : sweep_ctas_per_sm<T>());
    for (int l = 0; l + 1 < s->maxlev; ++l) {
        std::vector<Box<T>> set;
        for (int b = 0; b < s->nbox; ++b)
            if (l < H.lc[b]) set.push_back(make_box(s, H, b, l));
        if (!set.empty()) {
            double score = 0.0;
            int zc = choose_zc(set, slots, &score);
            if (s->opts.sweep_zc > 0) {   // the tile depth given (autotuned) instead
                int maxnz = 1;
                for (const auto &B : set) maxnz = std::max(maxnz, B.nz);
                zc = std::min(s->opts.sweep_zc, maxnz);
            }
            for (auto &B : set) B.zc = zc;
            // fused sweeps when the grid can keep the GPU busy, and only in
            // FP32: FP64 smoothing is bound by the FP64 pipe, where the red
            // ring the fused sweep recomputes costs more than the DRAM
            // traffic it saves (measured 22% slower at 256^3)
            bool small = true;  // 32-bit offsets inside the fused sweep
            for (const auto &B : set) small = small && level_elems(B.nx, B.ny, B.nz) <= kSweepMaxElems;
            const bool ok = score >= 0.7;
            // (FP64 levels never: their f and 1/D are colour-split, which
            // the fused sweep does not read)
            H.fused[l] = small && sizeof(T) == sizeof(float) &&
                         (s->opts.smoother == 2 || (s->opts.smoother == 0 && ok));
            size_t moff = 0;
            bool prol = false;
            if (H.fused[l] && tma && s->tma && plan_maps(set, blob, &moff, &prol)) {
                map_offs->push_back({l, moff});  // else: plain-load sweeps on this level
                H.prol[l] = prol ? 1 : 0;
            }
        }
        plans.push_back(plan_set(blob, &H.smooth[l], set));
    }
    H.njobs = (int)jobs.size();
    *jobs_off = blob.put(jobs.data(), jobs.size() * sizeof(CoarseJob<T>));
    if (s->cg_bottom) {
        const auto &db = s->dims[0][s->nlev[0] - 1];
        H.cggrid = std::max(1, std::min({cg_bottom_ctas_per_sm<T>() * s->sms, kCgPartials,
                                         tiles_of(TK_CELL, db[0], db[1], db[2])}));
    }
    if (s->opts.persistent) {
        int per_sm = level_ctas_per_sm<T>();
        if (s->opts.level_ctas > 0) per_sm = std::min(per_sm, s->opts.level_ctas);
        H.pgrid = per_sm * s->sms;
    }
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
    if (o->inner_cycles < 0 || o->inner_cycles > 8)
        return set_error(MG_ERR_INVALID_ARG, "inner_cycles must be in 0..8");
    if (o->krylov < 0 || o->krylov > 1) return set_error(MG_ERR_INVALID_ARG, "krylov must be 0 or 1");
    if (o->wait_limit < -1) return set_error(MG_ERR_INVALID_ARG, "wait_limit must be >= -1");
    if (o->tma < -1 || o->tma > 1) return set_error(MG_ERR_INVALID_ARG, "tma must be -1, 0 or 1");
    if (o->persistent < 0 || o->persistent > 2)
        return set_error(MG_ERR_INVALID_ARG, "persistent must be 0, 1 or 2");
    if (o->sweep_zc < 0 || o->sweep_zc > 4096)
        return set_error(MG_ERR_INVALID_ARG, "sweep_zc must be in 0..4096");
    if (o->level_ctas < 0 || o->level_ctas > 64)
        return set_error(MG_ERR_INVALID_ARG, "level_ctas must be in 0..64");
    if (o->fp32_setup < 0 || o->fp32_setup > 1)
        return set_error(MG_ERR_INVALID_ARG, "fp32_setup must be 0 or 1");
    if ((o->dev_alloc == nullptr) != (o->dev_free == nullptr))
        return set_error(MG_ERR_INVALID_ARG, "dev_alloc and dev_free come together");
    return MG_OK;
}

// Level structure of a coupled level: halve while every box's dims and
// lower corners are even (boxes may end as single cells: their neighbours
// are in other boxes, and a small union keeps the dense coarsest solve,
// O(n^3) on one SM at set-up, cheap).  Fills dims and lower corners per box
// and level; returns the level count.
static int max_record_cells(const std::vector<ExchRec> &recs)
{
    int m = 0;
    for (const ExchRec &r : recs) m = std::max(m, r.ex * r.ey * r.ez);
    return m;
}

static int coupled_levels(int nbox, const int (*lo)[3], const int (*n)[3],
                          std::vector<std::vector<std::array<int, 3>>> &dims,
                          std::vector<std::vector<std::array<int, 3>>> &los)
{
    dims.assign(nbox, {});
    los.assign(nbox, {});
    for (int b = 0; b < nbox; ++b) {
        dims[b].push_back({n[b][0], n[b][1], n[b][2]});
        los[b].push_back({lo[b][0], lo[b][1], lo[b][2]});
    }
    int L = 1;
    while (L < 32) {
        bool ok = true;
        for (int b = 0; b < nbox && ok; ++b)
            for (int d = 0; d < 3 && ok; ++d) {
                const int m = dims[b][L - 1][d], c = los[b][L - 1][d];
                ok = m % 2 == 0 && m >= 2 && c % 2 == 0;
            }
        if (!ok) break;
        for (int b = 0; b < nbox; ++b) {
            const auto &m = dims[b][L - 1];
            const auto &c = los[b][L - 1];
            dims[b].push_back({m[0] / 2, m[1] / 2, m[2] / 2});
            los[b].push_back({c[0] / 2, c[1] / 2, c[2] / 2});
        }
        ++L;
    }
    return L;
}

static bool create_events(cudaEvent_t *e, int n)
{
    for (int i = 0; i < n; ++i)
        if (cudaEventCreateWithFlags(&e[i], cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
}

int solver_create(Solver **out, int nbox, const int (*n)[3], const double *dx, int bc,
                  const mg_opts *opts, bool shared_weights, const int (*lo)[3], int cut)
{
    if (!out) return set_error(MG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nbox < 1 || !n || !dx) return set_error(MG_ERR_INVALID_ARG, "need nbox >= 1, n, dx");
    if (bc < 0 || bc > 511)
        return set_error(MG_ERR_INVALID_ARG, "bc must be a wall mask in 0..511");
    for (int d = 0; d < 3; ++d)
        if (((bc >> (6 + d)) & 1) && ((bc >> (2 * d)) & 3))
            return set_error(MG_ERR_INVALID_ARG, "axis %d is periodic and has a Neumann wall", d);
    const bool coupled = lo != nullptr;
    const bool periodic = (bc >> 6) != 0;
    if (coupled && bc != 0)
        return set_error(MG_ERR_INVALID_ARG, "a coupled level has Dirichlet walls (bc = 0)");
    if (periodic && nbox != 1)
        return set_error(MG_ERR_UNSUPPORTED,
                         "periodic axes are implemented for one box per context (mg_create)");
    mg_opts o;
    mg_default_opts(&o);
    if (opts) o = *opts;
    CKS(validate_opts(&o));
    if (o.krylov) {
        bool all_neumann = true;
        for (int d = 0; d < 3; ++d) all_neumann = all_neumann && ((bc >> (2 * d)) & 3) == 3;
        if (coupled || periodic || all_neumann)
            return set_error(MG_ERR_UNSUPPORTED,
                             "krylov = 1 needs independent boxes, no periodic axis and a "
                             "Dirichlet wall");
        if (o.nu1 != o.nu2 || o.nu1 < 1)
            return set_error(MG_ERR_UNSUPPORTED,
                             "krylov = 1 needs nu1 = nu2 >= 1 (a symmetric preconditioner)");
        o.smoother = 1;  // single-colour passes: the post-smoother runs black first
    }
    if (coupled || periodic) {
        // ghost exchanges between boxes (or across periodic faces) before
        // every stencil: single-colour passes; a coupled level launches
        // every level down to the dense bottom solve of the union (a
        // periodic box runs its coarse levels in the one-CTA kernel, which
        // does its own exchanges)
        o.smoother = 1;
        if (coupled) o.coarse_cells = -1;
        o.tma = -1;
    }
    std::vector<std::vector<std::array<int, 3>>> cdims, clos;
    std::vector<Brick> bricks;
    int clev = 0, ucells = 0;
    if (coupled) {
        for (int b = 0; b < nbox; ++b) {
            Brick B;
            for (int d = 0; d < 3; ++d) {
                if (n[b][d] < 1) return set_error(MG_ERR_INVALID_ARG, "box %d: need n >= 1", b);
                B.lo[d] = lo[b][d];
                B.n[d] = n[b][d];
            }
            if (dx[b] != dx[0])
                return set_error(MG_ERR_INVALID_ARG, "a coupled level has one spacing dx");
            bricks.push_back(B);
        }
        int a = 0, c = 0;
        if (level_check_disjoint(bricks, &a, &c))
            return set_error(MG_ERR_INVALID_ARG, "boxes %d and %d overlap", a, c);
        clev = coupled_levels(nbox, lo, n, cdims, clos);
        if (cut > 0) {
            // levels 0 .. cut - 1 only; the last one is solved elsewhere
            if (clev < cut)
                return set_error(MG_ERR_UNSUPPORTED, "the boxes halve %d times, %d wanted",
                                 clev - 1, cut - 1);
            clev = cut;
            for (int b = 0; b < nbox; ++b) {
                cdims[b].resize(cut);
                clos[b].resize(cut);
            }
        }
        for (int b = 0; b < nbox; ++b) {
            const auto &d = cdims[b][clev - 1];
            ucells += d[0] * d[1] * d[2];
        }
        if (cut > 0) ucells = 0;   // no dense bottom of its own
        if (ucells > MG_MAX_BOTTOM)
            return set_error(MG_ERR_UNSUPPORTED,
                             "coarsest level of the union has %d cells (> %d): box dims and "
                             "corners must halve further together",
                             ucells, MG_MAX_BOTTOM);
    }

    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    Solver *s = new Solver();
    s->dev = dev;
    s->sms = sms;
    s->shared = shared_weights;
    s->nbox = nbox;
    s->opts = o;
    s->has32 = o.precision == MG_MIXED;
    s->tma = s->has32 && o.tma >= 0;
    s->pcg = o.krylov == 1;
    s->bc = bc;
    // A singular (constants in the null space): no axis has a Dirichlet wall
    s->singular = true;
    for (int d = 0; d < 3; ++d)
        if (!((bc >> (6 + d)) & 1) && ((bc >> (2 * d)) & 3) != 3) s->singular = false;
    s->coupled = coupled;
    s->cut = cut;
    s->xmode = coupled || periodic;
    s->wide = s->xmode;
    s->coarse32 = s->has32 && !s->xmode && o.fp32_setup == 0;
    if (coupled) {
        s->lo = clos;
        s->ub.n = ucells;
        s->ub.nbox = nbox;
    }
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
        s->dims.push_back(coupled ? cdims[b] : level_dims(nx, ny, nz));
        s->nlev.push_back((int)s->dims.back().size());
        s->maxlev = std::max(s->maxlev, s->nlev.back());
        const std::array<int, 3> db = s->dims.back().back();
        const int cells = db[0] * db[1] * db[2];
        if (!coupled && cells > MG_MAX_BOTTOM) {
            // too large for a dense inverse: one box with a Dirichlet wall
            // solves its coarsest level by conjugate gradients
            if (nbox == 1 && !periodic && !s->singular) {
                s->cg_bottom = true;
            } else {
                delete s;
                return set_error(MG_ERR_UNSUPPORTED,
                                 "box %d: coarsest level %dx%dx%d has %d cells (> %d); with "
                                 "several boxes, periodic axes or every wall Neumann the dims "
                                 "must halve down to a small level",
                                 b, db[0], db[1], db[2], cells, MG_MAX_BOTTOM);
            }
        }
        s->max_bottom = std::max(s->max_bottom, cells);
        s->off[b + 1] = s->off[b] + (long long)nx * ny * nz;
    }
    s->total = s->off[nbox];
    if (periodic) {  // one box: corners at 0, its coarsest level is the bottom
        s->lo.assign(1, std::vector<std::array<int, 3>>(s->nlev[0], {0, 0, 0}));
        const auto &db = s->dims[0].back();
        s->ub.n = db[0] * db[1] * db[2];
        s->ub.nbox = 1;
    }

    // level arrays: dry run for the size, then carve the zero-filled arena
    Bump bump;
    carve(s, s->h64, bump, true);
    if (s->has32) carve(s, s->h32, bump, true);
    size_t work_elems = 0, ntiles0 = 0;
    std::vector<size_t> work_off(nbox, 0);
    for (int b = 0; b < nbox; ++b) {
        const auto &db = s->dims[b].back();
        const size_t nb = s->cg_bottom ? 0 : (size_t)db[0] * db[1] * db[2];
        work_off[b] = work_elems;
        work_elems += nb * nb;
        ntiles0 += (size_t)tiles_of(TK_CELL, s->n[b][0], s->n[b][1], s->n[b][2]);
    }
    if (s->xmode) {  // one dense inverse for the union of the coarsest levels
        work_elems = (size_t)s->ub.n * s->ub.n;
        std::fill(work_off.begin(), work_off.end(), 0);
    }
    // CG: p and q of every box in the level-0 layout (zero guards), the
    // per-box scalars and the two device pointer tables
    auto pcg_arrays = [&](Bump &bb, std::vector<double *> &pp, std::vector<double *> &qq) {
        pp.assign(nbox, nullptr);
        qq.assign(nbox, nullptr);
        if (!s->pcg) return;
        for (int b = 0; b < nbox; ++b) {
            const long long E = level_elems(s->n[b][0], s->n[b][1], s->n[b][2]);
            const long long Q = pitch_plane(s->n[b][0], s->n[b][1]);
            for (auto *v : {&pp, &qq}) {
                double *a = bb.take<double>((size_t)E);
                (*v)[b] = a ? a + Q : nullptr;
            }
        }
        s->sc.rz = bb.take<double>(nbox);
        s->sc.rzn = bb.take<double>(nbox);
        s->sc.pq = bb.take<double>(nbox);
        s->sc.beta = bb.take<double>(nbox);
        s->sc.alpha = bb.take<double>(nbox);
        s->pcg_p = bb.take<double *>(nbox);
        s->pcg_q = bb.take<double *>(nbox);
    };
    std::vector<double *> pcg_p, pcg_q;
    pcg_arrays(bump, pcg_p, pcg_q);
    bump.take<double>(s->total);      // beta copy
    bump.take<double>(work_elems);    // inverse scratch
    bump.take<double>(ntiles0);       // partials
    for (int i = 0; i < 7; ++i) bump.take<double>(nbox);
    bump.take<int>(nbox);
    bump.take<int>(nbox);   // inner flags
    bump.take<int>(2);      // inner cycle counters (this step, this solve)
    bump.take<int>(1);  // error word
    bump.take<unsigned>(1);  // grid-barrier word
    if (s->cg_bottom) bump.take<double>(2 * kCgPartials);   // CG partial sums
    // judge block: hist | rel0 | best | tol | status | cycles | stall | step
    const size_t jbytes = sizeof(double) * ((size_t)nbox * MG_MAX_HIST + 2 * nbox + 1) +
                          sizeof(int) * (3 * (size_t)nbox + 1);
    bump.take<char>(jbytes);
    const size_t bytes = bump.used;
    cudaError_t e = dev_malloc(s, reinterpret_cast<void **>(&s->arena), bytes);
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
    pcg_arrays(real, pcg_p, pcg_q);
    if (s->pcg) {
        e = cudaMemcpy(s->pcg_p, pcg_p.data(), sizeof(double *) * nbox, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(s->pcg_q, pcg_q.data(), sizeof(double *) * nbox, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            solver_destroy(s);
            return set_error(MG_ERR_CUDA, "CG pointer tables: %s", cudaGetErrorString(e));
        }
    }
    s->beta = real.take<double>(s->total);
    s->work = real.take<double>(work_elems);
    s->partials = real.take<double>(ntiles0);
    s->dnorm = real.take<double>(nbox);
    s->dnormf = real.take<double>(nbox);
    s->dinv = real.take<double>(nbox);
    s->se = real.take<double>(nbox);
    s->sr = real.take<double>(nbox);
    s->sr_inv = real.take<double>(nbox);
    s->dmean = real.take<double>(nbox);
    s->active = real.take<int>(nbox);
    s->active32 = real.take<int>(nbox);
    s->icount = real.take<int>(2);
    s->derr = real.take<int>(1);
    s->gbar = real.take<unsigned>(1);
    if (s->cg_bottom) s->cgpart = real.take<double>(2 * kCgPartials);
    s->jbytes = jbytes;
    s->jblock = real.take<char>(jbytes);
    {
        char *q = s->jblock;
        s->J.hist = reinterpret_cast<double *>(q);
        q += sizeof(double) * (size_t)nbox * MG_MAX_HIST;
        s->J.rel0 = reinterpret_cast<double *>(q);
        q += sizeof(double) * nbox;
        s->J.best = reinterpret_cast<double *>(q);
        q += sizeof(double) * nbox;
        s->J.tol = reinterpret_cast<double *>(q);
        q += sizeof(double);
        s->J.status = reinterpret_cast<int *>(q);
        q += sizeof(int) * nbox;
        s->J.cycles = reinterpret_cast<int *>(q);
        q += sizeof(int) * nbox;
        s->J.stall = reinterpret_cast<int *>(q);
        q += sizeof(int) * nbox;
        s->J.step = reinterpret_cast<int *>(q);
        s->J.max_cycles = o.max_cycles;
        s->J.stall_limit = o.krylov ? 0 : 5;
    }

    // launch-set descriptors (+ packed offsets and side flags)
    DescBlob blob;
    std::vector<SetPlan<Box<double>>> p64;
    std::vector<SetPlan<Box<float>>> p32;
    size_t jobs64 = 0, jobs32 = 0;
    std::vector<std::pair<int, size_t>> maps64, maps32;
    plan_hier(s, s->h64, blob, p64, &jobs64, &maps64);
    if (s->has32) plan_hier(s, s->h32, blob, p32, &jobs32, &maps32);
    // adaptive inner cycles: the exit test reads the red-only restriction of
    // the finest FP32 level (after a black pass: nu1 > 0, no full residual)
    s->inner_adapt = s->has32 && !s->pcg && o.inner_cycles == 0 && o.nu1 > 0 &&
                     !o.full_residual && !s->h32.smooth.empty() &&
                     s->h32.smooth[0].nbox > 0;
    // FP64 look-ahead norm: needs a red pass first (nu1 > 0), a black pass
    // last (nu2 > 0, so black residuals vanish), single-colour passes on every
    // box's finest level, and the red-only residual reading
    s->lookahead = !s->has32 && !s->pcg && o.nu1 > 0 && o.nu2 > 0 && !o.full_residual &&
                   !s->h64.smooth.empty() && s->h64.smooth[0].nbox == nbox &&
                   !s->h64.fused[0];
    // set-up sets: every box that has level l; boxes that have l + 1; bottoms
    std::vector<SetPlan<SetupBox>> psu;
    s->setup_lv.assign(s->maxlev, SetupSet{});
    s->setup_coarsen.assign(std::max(s->maxlev - 1, 0), SetupSet{});
    auto setup_box = [&](int b, int l) {
        SetupBox B;
        memset(&B, 0, sizeof B);
        const LevelBufs<double> &L = s->h64.lv[b][l];
        const auto &d = s->dims[b][l];
        B.wx = L.wx;
        B.wy = L.wy;
        B.wz = L.wz;
        B.invD = s->has32 ? nullptr : L.invD;  // mixed: FP64 levels never smooth
        B.D = L.D;
        if (l + 1 < s->nlev[b]) {
            const LevelBufs<double> &C = s->h64.lv[b][l + 1];
            const auto &c = s->dims[b][l + 1];
            B.cwx = C.wx;
            B.cwy = C.wy;
            B.cwz = C.wz;
            B.cP = (int)pitch_row(c[0], s->wide);
            B.cQ = pitch_plane(c[0], c[1], s->wide);
        }
        if (s->has32) {
            const LevelBufs<float> &M = s->h32.lv[b][l];
            B.wx32 = M.wx;
            B.wy32 = M.wy;
            B.wz32 = M.wz;
            B.invD32 = M.invD;
            if (l + 1 < s->nlev[b]) {
                const LevelBufs<float> &C = s->h32.lv[b][l + 1];
                B.cwx32 = C.wx;
                B.cwy32 = C.wy;
                B.cwz32 = C.wz;
            }
        }
        B.beta = s->beta + s->off[b];
        B.inv_h2 = 1.0 / (s->dx[b] * s->dx[b]);
        B.w32src = s->coarse32 ? 1 : 0;
        B.nx = d[0];
        B.ny = d[1];
        B.nz = d[2];
        B.P = (int)pitch_row(d[0], s->wide);
        B.Q = pitch_plane(d[0], d[1], s->wide);
        B.zc = kSweepZ;
        B.bc = s->bc;
        if (s->xmode && l == 0) B.betaL = L.phi;  // beta is staged in phi during set-up
        B.rb = 1;                                  // FP64 invD and D colour-split
        if (s->xmode) {
            const auto &o = s->lo[b][l];
            B.par = (((o[0] + o[1] + o[2]) % 2) + 2) % 2;
        }
        if (l == s->nlev[b] - 1) {
            B.work = s->work + work_off[b];
            B.inv64 = s->has32 ? nullptr : s->h64.ainv[b];  // mixed: FP32 inverse only
            B.inv32 = s->has32 ? s->h32.ainv[b] : nullptr;
        }
        return B;
    };
    const int nsetup = s->shared ? 1 : nbox;  // shared weights are set up once
    for (int l = 0; l < s->maxlev; ++l) {
        std::vector<SetupBox> all, coarse;
        for (int b = 0; b < nsetup; ++b) {
            if (l < s->nlev[b]) all.push_back(setup_box(b, l));
            if (l + 1 < s->nlev[b]) coarse.push_back(setup_box(b, l));
        }
        psu.push_back(plan_set(blob, &s->setup_lv[l], all));
        if (l + 1 < s->maxlev) psu.push_back(plan_set(blob, &s->setup_coarsen[l], coarse));
    }
    {
        std::vector<SetupBox> bot;
        for (int b = 0; b < nsetup; ++b) bot.push_back(setup_box(b, s->nlev[b] - 1));
        s->bottom_packed = 0;
        for (const SetupBox &B : bot)
            s->bottom_packed = std::max(s->bottom_packed,
                                        packed_bottom_bytes(B.nx * B.ny * B.nz, B.inv64 != nullptr));
        psu.push_back(plan_set(blob, &s->setup_bottom, bot));
    }
    // coupled level: ghost exchange records of every level (the cached
    // communication pattern) and the union numbering of the coarsest cells
    std::vector<size_t> xrec_at;
    size_t uoff_at = 0;
    if (periodic) {
        for (int l = 0; l < s->nlev[0]; ++l) {
            const auto &d = s->dims[0][l];
            Brick bl;
            int period[3];
            for (int q = 0; q < 3; ++q) {
                bl.lo[q] = 0;
                bl.n[q] = d[q];
                period[q] = ((bc >> (6 + q)) & 1) ? d[q] : 0;
            }
            const std::vector<ExchRec> recs = periodic_exchange(bl, period);
            s->nxrec.push_back((int)recs.size());
            s->xmax.push_back(max_record_cells(recs));
            xrec_at.push_back(blob.put(recs.data(), recs.size() * sizeof(ExchRec)));
        }
        std::vector<int> uo = {0, s->ub.n};
        uoff_at = blob.put(uo.data(), uo.size() * sizeof(int));
    }
    if (coupled) {
        for (int l = 0; l < clev; ++l) {
            std::vector<Brick> bl(nbox);
            for (int b = 0; b < nbox; ++b)
                for (int d = 0; d < 3; ++d) {
                    bl[b].lo[d] = clos[b][l][d];
                    bl[b].n[d] = cdims[b][l][d];
                }
            const std::vector<ExchRec> recs = level_exchange(bl);
            s->nxrec.push_back((int)recs.size());
            s->xmax.push_back(max_record_cells(recs));
            xrec_at.push_back(blob.put(recs.data(), recs.size() * sizeof(ExchRec)));
        }
        std::vector<int> uo(nbox + 1, 0);
        for (int b = 0; b < nbox; ++b) {
            const auto &d = cdims[b][clev - 1];
            uo[b + 1] = uo[b] + d[0] * d[1] * d[2];
        }
        uoff_at = blob.put(uo.data(), uo.size() * sizeof(int));
    }
    const size_t off_at = blob.put(s->off.data(), s->off.size() * sizeof(long long));
    std::vector<int> zeros(nbox, 0);
    const size_t side_at = blob.put(zeros.data(), zeros.size() * sizeof(int));
    // adaptive inner cycles: chunks of kInnerChunk restriction tiles of one
    // box each (the first stage of the exit test's sums), their start per box
    size_t icst_at = 0;
    if (s->inner_adapt) {
        const SetPlan<Box<float>> *p0 = nullptr;
        for (const auto &p : p32)
            if (p.target == &s->h32.smooth[0]) p0 = &p;
        const int nb = s->h32.smooth[0].nbox;
        std::vector<int> ts(nb + 1), cst(nb + 1, 0);
        memcpy(ts.data(), blob.bytes.data() + p0->ts_off[TK_COARSE], sizeof(int) * (nb + 1));
        for (int b = 0; b < nb; ++b)
            cst[b + 1] = cst[b] + (ts[b + 1] - ts[b] + kInnerChunk - 1) / kInnerChunk;
        s->inner_chunks = cst[nb];
        icst_at = blob.put(cst.data(), cst.size() * sizeof(int));
    }
    e = dev_malloc(s, reinterpret_cast<void **>(&s->desc), blob.bytes.size());
    if (e != cudaSuccess) {
        solver_destroy(s);
        return set_error(MG_ERR_OOM, "cudaMalloc(descriptors): %s", cudaGetErrorString(e));
    }
    if (s->inner_adapt) {   // the restriction's per-warp sums and their chunk sums
        const size_t np = (size_t)s->h32.smooth[0].ntiles[TK_COARSE] * (kThreads / 32);
        e = dev_malloc(s, reinterpret_cast<void **>(&s->ipart),
                       (np + (size_t)s->inner_chunks) * sizeof(double));
        if (e != cudaSuccess) {
            solver_destroy(s);
            return set_error(MG_ERR_OOM, "cudaMalloc(inner sums): %s", cudaGetErrorString(e));
        }
        s->ichunk = s->ipart + np;
        s->icstart = reinterpret_cast<const int *>(s->desc + icst_at);
    }
    if (periodic) {
        // the coarse jobs' exchange records, now that their address is known
        auto link = [&](size_t at, int lc, auto *tag) {
            using J = std::remove_pointer_t<decltype(tag)>;
            J *job = reinterpret_cast<J *>(blob.bytes.data() + at);
            for (int l = 0; l < job->nlev; ++l) {
                job->rec[l] = reinterpret_cast<const ExchRec *>(s->desc + xrec_at[lc + l]);
                job->nrec[l] = s->nxrec[lc + l];
            }
        };
        link(jobs64, s->h64.lc[0], (CoarseJob<double> *)nullptr);
        if (s->has32) link(jobs32, s->h32.lc[0], (CoarseJob<float> *)nullptr);
    }
    e = cudaMemcpy(s->desc, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        solver_destroy(s);
        return set_error(MG_ERR_CUDA, "descriptor upload: %s", cudaGetErrorString(e));
    }
    for (auto &p : p64) patch_set(p, s->desc);
    for (auto &p : p32) patch_set(p, s->desc);
    for (auto &p : psu) patch_set(p, s->desc);
    if (s->tma)
        for (auto &m : maps32)
            s->h32.maps[m.first] = reinterpret_cast<const SweepMaps *>(s->desc + m.second);
    s->h64.jobs = reinterpret_cast<const CoarseJob<double> *>(s->desc + jobs64);
    if (s->has32) s->h32.jobs = reinterpret_cast<const CoarseJob<float> *>(s->desc + jobs32);
    s->doff = reinterpret_cast<const long long *>(s->desc + off_at);
    s->dside = reinterpret_cast<int *>(s->desc + side_at);
    if (s->xmode) {
        for (size_t l = 0; l < xrec_at.size(); ++l)
            s->xrec.push_back(reinterpret_cast<const ExchRec *>(s->desc + xrec_at[l]));
        s->ub.off = reinterpret_cast<const int *>(s->desc + uoff_at);
        s->ub.rec = s->xrec.back();
        s->ub.nrec = s->nxrec.back();
        s->ub.singular = s->singular ? 1 : 0;
    }

    if (cudaMallocHost(&s->hjblock, s->jbytes) != cudaSuccess ||
        cudaMallocHost(&s->hnorm, sizeof(double) * 2 * nbox) != cudaSuccess ||
        cudaMallocHost(&s->hactive, sizeof(int) * nbox) != cudaSuccess ||
        cudaMallocHost(&s->hflags, sizeof(int) * nbox) != cudaSuccess ||
        cudaMallocHost(&s->hside, sizeof(int) * (nbox + 1)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        !create_events(s->ev_slab, Solver::kBetaSlabs) ||
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
    // a caller's allocator may hand the memory out again at once: let the
    // context's queued work (e.g. a set-up without a solve yet) finish first
    if (s->opts.dev_free) cudaDeviceSynchronize();
    for (auto *v : {&s->slots64, &s->slots32, &s->slots_head, &s->slots_down0, &s->slots_rest,
                    &s->direct})
        for (auto &sl : *v) {
            cudaEventDestroy(sl.b);
            cudaEventDestroy(sl.e);
        }
    for (auto e : s->ev_free) cudaEventDestroy(e);
    if (s->h64.head) cudaGraphExecDestroy(s->h64.head);
    if (s->h64.graph) cudaGraphExecDestroy(s->h64.graph);
    if (s->h32.graph) cudaGraphExecDestroy(s->h32.graph);
    if (s->h32.down0) cudaGraphExecDestroy(s->h32.down0);
    if (s->h32.rest) cudaGraphExecDestroy(s->h32.rest);
    if (s->loop64) cudaGraphExecDestroy(s->loop64);
    if (s->loop32) cudaGraphExecDestroy(s->loop32);
    if (s->loop_pcg) cudaGraphExecDestroy(s->loop_pcg);
    if (s->hjblock) cudaFreeHost(s->hjblock);
    dev_free(s, s->arena);
    dev_free(s, s->desc);
    dev_free(s, s->ipart);
    dev_free(s, s->stage_a);
    if (s->hnorm) cudaFreeHost(s->hnorm);
    if (s->hactive) cudaFreeHost(s->hactive);
    if (s->hflags) cudaFreeHost(s->hflags);
    if (s->hside) cudaFreeHost(s->hside);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->cap2) cudaStreamDestroy(s->cap2);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    for (cudaEvent_t &e : s->ev_slab)
        if (e) cudaEventDestroy(e);
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

// Page-locked host memory (cudaMallocHost / cudaHostRegister).
static bool is_pinned_host(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

static int ensure_stage(Solver *s)
{
    if (s->stage_a) return MG_OK;
    const cudaError_t e =
        dev_malloc(s, reinterpret_cast<void **>(&s->stage_a), sizeof(double) * 3 * (size_t)s->total);
    if (e != cudaSuccess)
        return set_error(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                         "staging buffers: %s", cudaGetErrorString(e));
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
// side: copy a host array in on the copy stream (the caller's stream waits
// for it), so that it overlaps work already queued on st.
static int device_view(Solver *s, const double *p, int which, bool copy_in, cudaStream_t st,
                       const double **dv, bool *staged, long long count = -1, bool side = false)
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
    if (count < 0) count = s->total;
    if (copy_in && side) {
        CK(cudaMemcpyAsync(stage, p, sizeof(double) * count, cudaMemcpyHostToDevice, s->copy));
        CK(cudaEventRecord(s->ev_in, s->copy));
        CK(cudaStreamWaitEvent(st, s->ev_in, 0));
    } else if (copy_in) {
        CK(cudaStreamWaitEvent(st, s->ev_in, 0));  // an earlier side copy into the buffer
        CK(cudaMemcpyAsync(stage, p, sizeof(double) * count, cudaMemcpyHostToDevice, st));
    }
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
    const long long nbeta = s->shared ? s->off[1] : s->total;
    // one box, beta in pinned host memory: copied in by slabs of planes on
    // the copy stream (after the caller's stream has finished with the
    // previous beta), each slab's face weights launched once it is in
    // (face positions of planes [a, b) read beta planes a-1 .. b-1)
    const int nx = s->n[0][0], ny = s->n[0][1], nz = s->n[0][2];
    const long long plane = (long long)nx * ny;
    // mixed precision's finest level takes its FP32 copies with its faces
    // (step 5) and its FP32 1/D with its diagonal (step 6); a coupled level's
    // faces come from step 4, and its copies from step 3.  With coarse32 the
    // coarser levels are FP32 only, averaged from the finer FP32 weights
    // (step 9) with their 1/D (step 8).
    const bool c32 = s->coarse32;
    const int face_step = s->has32 ? 5 : 0;
    int slabs = (int)std::max<long long>(
        1, std::min<long long>(Solver::kBetaSlabs, (long long)sizeof(double) * nbeta >> 22));  // >= 4 MiB each
    if (s->xmode || !(s->nbox == 1 || s->shared) || !is_pinned_host(beta) || nz < 2 * slabs)
        slabs = 1;
    if (slabs > 1) {
        int ex, ey, ez;
        tile_extent(TK_FACE, nx, ny, nz, ex, ey, ez);
        const int per_plane = tiles_of(TK_FACE, nx, ny, nz) / ez;
        const int zs = (nz + slabs - 1) / slabs;
        CK(cudaEventRecord(s->ev_fork, st));
        CK(cudaStreamWaitEvent(s->copy, s->ev_fork, 0));
        for (int c = 0, a = 0; a < nz; ++c, a += zs) {
            const int b = std::min(nz, a + zs);
            CK(cudaMemcpyAsync(s->beta + a * plane, beta + a * plane,
                               sizeof(double) * plane * (b - a), cudaMemcpyHostToDevice, s->copy));
            CK(cudaEventRecord(s->ev_slab[c], s->copy));
        }
        for (int c = 0, a = 0; a < nz; ++c, a += zs) {
            const int b = a + zs >= nz ? nz + 1 : a + zs;  // the last slab takes the top faces
            CK(cudaStreamWaitEvent(st, s->ev_slab[c], 0));
            CK(launch_setup_tiles(s->setup_lv[0], face_step, a * per_plane, b * per_plane, st));
        }
    } else {
        CK(cudaMemcpyAsync(s->beta, beta, sizeof(double) * nbeta, cudaMemcpyDefault, st));
    }
    if (s->xmode) {
        // beta into the level layout of level 0 (staged in phi), guard cells
        // -1 (the union's boundary) except where the exchange brings the
        // neighbouring box's beta; faces from there
        CK(launch_guard_fill(s->h64.fine, -1.0, st));
        CK(launch_pack(s->h64.fine, s->doff, s->beta, 0, st));
        CK(launch_exchange(s->h64.fine, nullptr, s->xrec[0], s->nxrec[0], s->xmax[0], st));
        CK(launch_setup(s->setup_lv[0], 4, st));
    } else if (slabs == 1) {
        // one launch per step and level over every box
        CK(launch_setup(s->setup_lv[0], face_step, st));
    }
    if (c32) {
        // the finest level's D and FP32 1/D; level l's FP32 weights averaged
        // into l + 1, then its FP32 1/D (no FP64 level below the finest)
        CK(launch_setup(s->setup_lv[0], 6, st));
        for (size_t l = 0; l < s->setup_coarsen.size(); ++l) {
            CK(launch_setup(s->setup_coarsen[l], 9, st));
            CK(launch_setup(s->setup_lv[l + 1], 8, st));
        }
    } else {
        for (size_t l = 0; l < s->setup_coarsen.size(); ++l)
            CK(launch_setup(s->setup_coarsen[l], 1, st));
    }
    // the dense coarsest inverses need the coarsest weights only: forked to
    // the side stream (one CTA per box, on as many SMs), they overlap the
    // diagonal and FP32 steps of the finer levels on the others (with
    // coarse32 those came first: the coarsest FP32 weights end that chain)
    if (!s->xmode) {
        CK(cudaEventRecord(s->ev_fork, st));
        CK(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
        if (!s->cg_bottom) CK(launch_setup_bottom(s->setup_bottom, s->bottom_packed, s->side));
        CK(cudaEventRecord(s->ev_join, s->side));
    }
    for (int l = 0; l < s->maxlev && !c32; ++l) {
        const bool fused32 = s->has32 && l == 0 && !s->xmode;
        CK(launch_setup(s->setup_lv[l], fused32 ? 6 : 2, st));
        if (s->has32 && !fused32) CK(launch_setup(s->setup_lv[l], 3, st));
    }
    if (s->xmode) {
        CK(launch_union_inverse(s->setup_bottom, s->ub, s->work, s->h64.uinv,
                                s->has32 ? s->h32.uinv : nullptr, st));
        CK(launch_guard_fill(s->h64.fine, 0.0, st));  // Dirichlet zeros again
    } else {
        CK(cudaStreamWaitEvent(st, s->ev_join, 0));
    }
    CK(cudaEventRecord(s->ev_setup1, st));
    s->kernels += launch_counter() - k0;
    s->beta_set = true;
    s->setup_pending = true;
    return MG_OK;
}

int solver_setup_from_weights(Solver *s, cudaStream_t st)
{
    if (!s || s->xmode || s->has32)
        return set_error(MG_ERR_INVALID_ARG, "set-up from weights: one FP64 box context");
    DeviceGuard g(s->dev);
    CK(cudaEventRecord(s->ev_setup0, st));
    const long long k0 = launch_counter();
    for (size_t l = 0; l < s->setup_coarsen.size(); ++l) CK(launch_setup(s->setup_coarsen[l], 1, st));
    if (!s->cg_bottom) CK(launch_setup_bottom(s->setup_bottom, s->bottom_packed, st));
    for (int l = 0; l < s->maxlev; ++l) CK(launch_setup(s->setup_lv[l], 2, st));
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

// Open a timed stretch of stage class `kind` holding `launches` launches of
// that class back to back; returns its slot or -1.
static int prof_begin(Solver *s, int kind, cudaStream_t st, int launches = 1)
{
    if (!s->prof || !s->rec) return -1;
    ProfSlot sl{kind, take_event(s), take_event(s), launches};
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
                s->prof_n[sl.kind] += sl.launches;
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

// prolong: the TMA sweep applies the level's prolongation to what it reads
// (only with maps that hold the coarse phi)
static cudaError_t sweep_launch(Solver *s, const BoxSet<double> &S, const SweepMaps *,
                                int src, cudaStream_t st, bool = false)
{
    return launch_rbgs_sweep(S, s->active, src, st);
}

static cudaError_t sweep_launch(Solver *s, const BoxSet<float> &S, const SweepMaps *maps, int src,
                                cudaStream_t st, bool prolong = false)
{
    if (maps)
        return launch_rbgs_sweep_tma(S, maps, s->active, src, s->derr, st,
                                     sweep_wait_polls(s->opts.wait_limit), prolong);
    return launch_rbgs_sweep(S, s->active, src, st);
}

// Coupled level: fill the guard cells of level lvl's boxes from their
// neighbours (no-op otherwise).
// second: fill phi2's guard cells (the out-of-place passes of the look-ahead).
template <class T>
static cudaError_t exch(Solver *s, const BoxSet<T> &S, int lvl, cudaStream_t st,
                        bool second = false)
{
    if (!s->xmode) return cudaSuccess;
    return launch_exchange(S, s->active, s->xrec[lvl], s->nxrec[lvl], s->xmax[lvl], st,
                           second ? 1 : 0);
}

// Coupled level: one norm for the union (no-op otherwise).
static cudaError_t combine(Solver *s, double *norm, cudaStream_t st)
{
    if (!s->coupled) return cudaSuccess;
    return launch_norm_combine(s->nbox, norm, st);
}

// The boxes are right-hand sides of one box (shared weights): on a level
// whose one box alone fills the GPU (at least 4 tiles per SM), passes read
// each cell's weights once for all of them.  On smaller levels the
// per-box launch keeps more CTAs in flight, which matters more there
// (measured at 128^3 x 8: the multi-RHS passes took the finest level's
// passes from 10.4 to 9.7 ms, but made the coarser levels 50% slower).
static bool rhs_shared(const Solver *s) { return s->shared && s->nbox > 1 && !s->xmode; }

template <class T>
static bool rhs_shared_level(const Solver *s, const BoxSet<T> &S)
{
    return rhs_shared(s) && S.nbox == s->nbox &&
           S.ntiles[TK_PAIR] / S.nbox >= 4 * s->sms;
}

template <class T>
static cudaError_t pass_launch(Solver *s, const BoxSet<T> &S, int color, cudaStream_t st)
{
    if (rhs_shared_level(s, S)) return launch_rbgs_pass_multi(S, s->active, color, 0, 0, st);
    return launch_rbgs_pass(S, s->active, color, st);
}

// reverse: black before red in each sweep (single-colour passes only).
// prolong_first: the first sweep also applies the level's prolongation
// (fused TMA sweeps whose maps hold the coarse phi, nu >= 2).
template <class T>
static cudaError_t smooth(Solver *s, const BoxSet<T> &S, int nu, bool fine, bool fused,
                          const SweepMaps *maps, cudaStream_t st, int lvl = 0,
                          bool reverse = false, bool prolong_first = false)
{
    // one timed stretch per group of back-to-back launches, so that the
    // event records between launches do not count in each launch's time
    cudaError_t e = cudaSuccess;
    int left = nu;
    if (fused && !reverse && left >= 2) {
        int nsw = left / 2 * 2;
        if (prolong_first) {   // timed as its own class: it also does the prolongation
            const int sl = fine ? prof_begin(s, MG_PROF_SWEEP_PROLONG, st) : -1;
            if ((e = sweep_launch(s, S, maps, 0, st, true)) != cudaSuccess) return e;
            prof_end(s, sl, st);
            --nsw;
        }
        const int sl = fine ? prof_begin(s, MG_PROF_SWEEP, st, nsw) : -1;
        for (int i = prolong_first ? 1 : 0; i < left / 2 * 2; ++i)
            if ((e = sweep_launch(s, S, maps, i & 1, st)) != cudaSuccess) return e;
        prof_end(s, sl, st);
        left -= left / 2 * 2;
    }
    if (left > 0) {
        const int sl = fine ? prof_begin(s, MG_PROF_PASS, st, 2 * left) : -1;
        for (; left > 0; --left) {
            for (int color = 0; color < 2; ++color) {
                if ((e = exch(s, S, lvl, st)) != cudaSuccess) return e;
                if ((e = pass_launch(s, S, reverse ? 1 - color : color, st)) != cudaSuccess)
                    return e;
            }
        }
        prof_end(s, sl, st);
    }
    return e;
}

// CTAs of work per exchange record (as launch_exchange: about 4 cells per
// thread on the largest record).
static int exch_chunks(int max_cells)
{
    return std::max(1, std::min(1024, (max_cells + 4 * kThreads - 1) / (4 * kThreads)));
}

// Level l of H as one persistent launch (mg_opts.persistent): going down,
// nu pre-smoothing sweeps then the residual and restriction; coming up,
// prolongation then nu post-smoothing sweeps (sym: black before red).
// Inner cycles of an adaptive refinement step: the finest FP32 level's
// restriction also sums squared residuals (into the partials array), and the
// exit test follows it.  FP64 hierarchies never take part.
static double *inner_partials(const Solver *s, const Hier<float> &H, int l)
{
    return (s->inner_norm && l == 0 && &H == &s->h32) ? s->ipart : nullptr;
}
static double *inner_partials(const Solver *, const Hier<double> &, int) { return nullptr; }

static cudaError_t inner_judge(Solver *s, const BoxSet<float> &S, cudaStream_t st)
{
    return launch_inner_judge(S, s->active, s->ipart, s->icstart, s->inner_chunks, kInnerChunk,
                              s->ichunk, s->se, s->sr, s->dnormf, s->J.tol, kInnerFloor,
                              s->coupled ? 1 : 0, st);
}
static cudaError_t inner_judge(Solver *, const BoxSet<double> &, cudaStream_t)
{
    return cudaSuccess;
}

template <class T>
static cudaError_t level_launch(Solver *s, const Hier<T> &H, int l, bool up, int nu,
                                bool head_done, bool sym, cudaStream_t st)
{
    const BoxSet<T> &S = H.smooth[l];
    LevelOps op{};
    op.nu = nu;
    op.head_done = head_done ? 1 : 0;
    op.red = (!up && s->opts.nu1 > 0 && !s->opts.full_residual) ? 1 : 0;
    op.reverse = sym ? 1 : 0;
    if (s->xmode && s->nxrec[l] > 0) {
        op.rec = s->xrec[l];
        op.nrec = s->nxrec[l];
        op.chunks = exch_chunks(s->xmax[l]);
    }
    op.flat = (S.flat >> TK_COARSE) & 1;
    op.partials = (!up && op.red) ? inner_partials(s, H, l) : nullptr;
    GridSync g{s->gbar, s->derr, sweep_wait_polls(s->opts.wait_limit)};
    const long long work = std::max<long long>(
        std::max(S.ntiles[TK_PAIR], S.ntiles[TK_COARSE]), (long long)op.nrec * op.chunks);
    const int grid = (int)std::min<long long>(work, H.pgrid);
    const int sl = l == 0 ? prof_begin(s, MG_PROF_LEVEL, st) : -1;
    cudaError_t e = launch_level(S, s->active, up ? 1 : 0, op, g, grid, st);
    prof_end(s, sl, st);
    if (e == cudaSuccess && op.partials) e = inner_judge(s, S, st);
    return e;
}

// Level l of H runs as persistent launches: persistent = 2 every level
// smoothed with passes; 1 only those whose largest stage fits in one wave
// of the persistent grid.
template <class T>
static bool level_persistent(const Solver *s, const Hier<T> &H, int l)
{
    if (H.pgrid <= 0 || H.fused[l]) return false;
    if (s->opts.persistent == 2) return true;
    const BoxSet<T> &S = H.smooth[l];
    return std::max(S.ntiles[TK_PAIR], S.ntiles[TK_COARSE]) <= H.pgrid;
}

// head_done: the finest level's first red pass already ran out of place
// (phi -> phi2, look-ahead); the cycle goes on with the black pass phi2 -> phi.
// sym: post-smoothing sweeps run black then red, the adjoint of the
// pre-smoother, so that with nu1 = nu2 and a zero start the cycle is a
// symmetric linear operator (the CG preconditioner).
template <class T>
// part: 0 the whole cycle; 1 only the finest level's down leg (smoothing,
// restriction); 2 the rest (what part 1 leaves out).
static cudaError_t enqueue_vcycle(Solver *s, const Hier<T> &H, cudaStream_t st,
                                  bool head_done = false, bool sym = false, int part = 0)
{
    cudaError_t e;
    const int nl = (int)H.smooth.size();
    int coarse = part == 2 ? prof_begin(s, MG_PROF_COARSE, st) : -1;
    for (int l = part == 2 ? 1 : 0; l < (part == 1 ? std::min(nl, 1) : nl); ++l) {
        const BoxSet<T> &S = H.smooth[l];
        if (S.nbox == 0) continue;
        if (level_persistent(s, H, l)) {
            if ((e = level_launch(s, H, l, false, s->opts.nu1, l == 0 && head_done, false, st)) !=
                cudaSuccess)
                return e;
            if (l == 0 && part == 0) coarse = prof_begin(s, MG_PROF_COARSE, st);
            continue;
        }
        int nu1 = s->opts.nu1;
        if (l == 0 && head_done) {
            int sl = prof_begin(s, MG_PROF_PASS, st);
            if ((e = exch(s, S, 0, st, true)) != cudaSuccess) return e;
            e = rhs_shared_level(s, S) ? launch_rbgs_pass_multi(S, s->active, 1, 1, 1, st)
                                       : launch_rbgs_pass_oop(S, s->active, 1, 1, nullptr, st);
            if (e != cudaSuccess) return e;
            prof_end(s, sl, st);
            --nu1;
        }
        if ((e = smooth(s, S, nu1, l == 0, H.fused[l] != 0, H.maps[l], st, l)) != cudaSuccess)
            return e;
        int sl = l == 0 ? prof_begin(s, MG_PROF_RESTRICT, st) : -1;
        if ((e = exch(s, S, l, st)) != cudaSuccess) return e;
        const bool red = s->opts.nu1 > 0 && !s->opts.full_residual;
        double *ip = red ? inner_partials(s, H, l) : nullptr;
        e = red ? launch_resid_restrict_red(S, s->active, st, ip)
                : launch_resid_restrict(S, s->active, st);
        if (e != cudaSuccess) return e;
        prof_end(s, sl, st);
        if (ip && (e = inner_judge(s, S, st)) != cudaSuccess) return e;
        if (l == 0 && part == 0) coarse = prof_begin(s, MG_PROF_COARSE, st);
    }
    if (part == 1) return cudaSuccess;
    if (part == 0 && (nl == 0 || H.smooth[0].nbox == 0)) coarse = prof_begin(s, MG_PROF_COARSE, st);
    if (s->coupled)
        e = launch_union_bottom(H.bottom, s->ub, H.uinv, s->active, st);
    else if (s->cg_bottom)
        e = launch_cg_bottom(H.bottom, s->active, H.cgp, H.cgq, s->cgpart,
                             GridSync{s->gbar, s->derr, sweep_wait_polls(s->opts.wait_limit)},
                             H.cggrid, sizeof(T) == sizeof(double) ? kCgTol64 : kCgTol32,
                             sizeof(T) == sizeof(double) ? kCgMaxIt64 : kCgMaxIt32, st);
    else
        e = launch_coarse_vcycle(H.jobs, H.njobs, s->active, s->opts.nu1, s->opts.nu2, st,
                                 sym ? 1 : 0);
    if (e != cudaSuccess) return e;
    for (int l = nl - 1; l >= 0; --l) {
        const BoxSet<T> &S = H.smooth[l];
        if (S.nbox == 0) continue;
        if (l == 0) {
            prof_end(s, coarse, st);
            coarse = -1;
        }
        if (level_persistent(s, H, l)) {
            if ((e = level_launch(s, H, l, true, s->opts.nu2, false, sym, st)) != cudaSuccess)
                return e;
            continue;
        }
        // fused TMA sweeps whose maps hold the coarse phi take the
        // prolongation into their first post-smoothing sweep
        const bool fuse = H.fused[l] && H.maps[l] && H.prol[l] && !sym && s->opts.nu2 >= 2;
        if (!fuse) {
            int sl = l == 0 ? prof_begin(s, MG_PROF_PROLONG, st) : -1;
            if ((e = launch_prolong(S, s->active, st)) != cudaSuccess) return e;
            prof_end(s, sl, st);
        }
        if ((e = smooth(s, S, s->opts.nu2, l == 0, H.fused[l] != 0, H.maps[l], st, l, sym,
                        fuse)) != cudaSuccess)
            return e;
    }
    prof_end(s, coarse, st);
    return cudaSuccess;
}

cudaError_t solver_enqueue_vcycle64(Solver *s, cudaStream_t st)
{
    return enqueue_vcycle(s, s->h64, st);
}

// FP64: V-cycle followed by the fine residual norm into dnorm.
static cudaError_t enqueue_step64(Solver *s, cudaStream_t st)
{
    cudaError_t e = enqueue_vcycle(s, s->h64, st);
    if (e != cudaSuccess) return e;
    int sl = prof_begin(s, MG_PROF_NORM, st);
    const int mode = (s->opts.nu2 > 0 && !s->opts.full_residual) ? 2 : 0;
    if ((e = exch(s, s->h64.fine, 0, st)) != cudaSuccess) return e;
    if ((e = launch_norm_partials(s->h64.fine, s->active, mode, s->partials, st)) != cudaSuccess)
        return e;
    e = launch_norm_finish(s->h64.fine, s->active, s->partials, s->dnorm, nullptr, nullptr, st,
                           nullptr, mode);
    if (e == cudaSuccess) e = combine(s, s->dnorm, st);
    prof_end(s, sl, st);
    return e;
}

// Look-ahead head: the finest level's first red pass, out of place, whose
// partial sums give the residual norm of the iterate it starts from.
static cudaError_t enqueue_head64(Solver *s, cudaStream_t st)
{
    const BoxSet<double> &S = s->h64.smooth[0];
    int sl = prof_begin(s, MG_PROF_PASS, st);
    cudaError_t e = exch(s, S, 0, st);
    if (e != cudaSuccess) return e;
    e = launch_rbgs_pass_oop(S, s->active, 0, 0, s->partials, st);
    if (e != cudaSuccess) return e;
    prof_end(s, sl, st);
    sl = prof_begin(s, MG_PROF_NORM, st);
    e = launch_norm_finish(S, s->active, s->partials, s->dnorm, nullptr, nullptr, st, nullptr, 2);
    if (e == cudaSuccess) e = combine(s, s->dnorm, st);
    prof_end(s, sl, st);
    return e;
}

// Look-ahead tail: the rest of the V-cycle.
static cudaError_t enqueue_tail64(Solver *s, cudaStream_t st)
{
    return enqueue_vcycle(s, s->h64, st, true);
}

// Host-judged inner cycles: the parts of one cycle on the inner flags.
static cudaError_t enqueue_inner_part(Solver *s, cudaStream_t st, int part)
{
    int *const outer = s->active;
    s->active = s->active32;
    s->inner_norm = true;
    cudaError_t e = enqueue_vcycle(s, s->h32, st, false, false, part);
    s->active = outer;
    s->inner_norm = false;
    return e;
}
static cudaError_t enqueue_inner_down0(Solver *s, cudaStream_t st)
{
    return enqueue_inner_part(s, st, 1);
}
static cudaError_t enqueue_inner_rest(Solver *s, cudaStream_t st)
{
    return enqueue_inner_part(s, st, 2);
}

// Mixed: FP32 V-cycles on r32, from e = 0 (zeroed by the prologue, and after
// that by each refinement update once it has used e).  inner_cycles > 0: that
// many.  Adaptive (inner_cycles = 0): up to kInnerMax, run on the inner flags
// (a copy of the step's); after each cycle's pre-smoothing on the finest level
// the exit test clears the flag of every box whose inner residual meets its
// target, so the rest of that cycle and the later ones skip the box, whose e
// is then the iterate the test measured.
static cudaError_t enqueue_step32(Solver *s, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (!s->inner_adapt) {
        const int inner = s->opts.inner_cycles > 0 ? s->opts.inner_cycles : kInnerFixed;
        for (int i = 0; i < inner; ++i)
            if ((e = enqueue_vcycle(s, s->h32, st)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    // adaptive: only inside the device loop's captured body (the host-judged
    // loop runs run_inner_host instead): a WHILE node whose body is one cycle
    // followed by the loop-end kernel (at most kInnerMax iterations)
    if (!s->inner_while) return cudaErrorInvalidValue;
    int *const outer = s->active;
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &nd)) != cudaSuccess)
        return e;
    if (cs != cudaStreamCaptureStatusActive || !cg) return cudaErrorStreamCaptureInvalidated;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, cg, 0, 0)) != cudaSuccess) return e;
    if ((e = launch_inner_begin(s->nbox, outer, s->active32, s->icount, h, 1, st)) != cudaSuccess)
        return e;
    if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &nd)) != cudaSuccess)
        return e;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return e;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(s->cap2, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return e;
    s->active = s->active32;
    s->inner_norm = true;
    const long long k0 = launch_counter();
    e = enqueue_vcycle(s, s->h32, s->cap2);
    if (e == cudaSuccess) e = launch_inner_end(s->nbox, s->active32, s->icount, kInnerMax, h, s->cap2);
    s->inner_cycle_kernels = launch_counter() - k0;
    s->active = outer;
    s->inner_norm = false;
    cudaError_t ee = cudaStreamEndCapture(s->cap2, &body);
    return e != cudaSuccess ? e : ee;
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
        if (s->h64.graph) cudaGraphExecDestroy(s->h64.graph);
        s->h64.graph = nullptr;
        if (s->h64.head) cudaGraphExecDestroy(s->h64.head);
        s->h64.head = nullptr;
        if (s->h32.graph) cudaGraphExecDestroy(s->h32.graph);
        s->h32.graph = nullptr;
        if (s->h32.down0) cudaGraphExecDestroy(s->h32.down0);
        s->h32.down0 = nullptr;
        if (s->h32.rest) cudaGraphExecDestroy(s->h32.rest);
        s->h32.rest = nullptr;
        for (auto *v : {&s->slots64, &s->slots32, &s->slots_head, &s->slots_down0,
                        &s->slots_rest}) {
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

// ---------------------------------------------- on-device convergence ----

// Body of the FP64 loop: V-cycle, residual norm, decision.  With look-ahead:
// head (red pass + norm of the previous iterate), decision, rest of the cycle
// (which skips the boxes just decided, so their solution stays in phi).
static cudaError_t enqueue_body64(Solver *s, cudaStream_t st, cudaGraphConditionalHandle h)
{
    cudaError_t e;
    if (s->lookahead) {
        if ((e = enqueue_head64(s, st)) != cudaSuccess) return e;
        if ((e = launch_judge(s->nbox, s->dnorm, s->dnormf, s->active, s->J, h, 1, st)) !=
            cudaSuccess)
            return e;
        return enqueue_tail64(s, st);
    }
    if ((e = enqueue_step64(s, st)) != cudaSuccess) return e;
    return launch_judge(s->nbox, s->dnorm, s->dnormf, s->active, s->J, h, 1, st);
}

// Body of the mixed loop: FP32 V-cycles on r32, FP64 update + residual +
// norm, scales for the next step, decision.
static cudaError_t enqueue_body32(Solver *s, cudaStream_t st, cudaGraphConditionalHandle h)
{
    s->inner_while = s->inner_adapt;
    cudaError_t e = enqueue_step32(s, st);
    s->inner_while = false;
    if (e != cudaSuccess) return e;
    if ((e = launch_refine_update(s->h64.fine, s->h32.fine, s->active, s->se, st)) != cudaSuccess)
        return e;
    if ((e = exch(s, s->h64.fine, 0, st)) != cudaSuccess) return e;
    if ((e = launch_refine_residual(s->h64.fine, s->h32.fine, s->active, s->sr_inv, s->partials,
                                    st)) != cudaSuccess)
        return e;
    if ((e = launch_norm_finish(s->h64.fine, s->active, s->partials, s->dnorm, nullptr, nullptr,
                                st, s->sr)) != cudaSuccess)
        return e;
    if ((e = combine(s, s->dnorm, st)) != cudaSuccess) return e;
    if ((e = launch_scales(s->nbox, s->active, 0, s->dnorm, s->dnormf, s->se, s->sr, s->sr_inv,
                           st)) != cudaSuccess)
        return e;
    return launch_judge(s->nbox, s->dnorm, s->dnormf, s->active, s->J, h, 1, st);
}

// One CG iteration (krylov = 1) on every active box: z = V r (phi was zeroed
// by the previous iteration's update or at the start), rz = <r, z>,
// beta = rz / rz_prev, p = z + beta p, q = A p, alpha = rz / <p, q>,
// x += alpha p, r -= alpha q, ||r|| into dnorm.  A and the V-cycle are both
// negative definite; the signs cancel in alpha and beta.
static cudaError_t enqueue_pcg(Solver *s, cudaStream_t st)
{
    cudaError_t e;
    if (s->has32) {
        // mixed: the symmetric V-cycle in FP32 on r / ||r||, scaled back
        if ((e = launch_pcg_mixed(s->h64.fine, s->h32.fine, s->active, 0, s->dnorm, st)) !=
                cudaSuccess ||
            (e = enqueue_vcycle(s, s->h32, st, false, true)) != cudaSuccess ||
            (e = launch_pcg_mixed(s->h64.fine, s->h32.fine, s->active, 1, s->dnorm, st)) !=
                cudaSuccess)
            return e;
    } else if ((e = enqueue_vcycle(s, s->h64, st, false, true)) != cudaSuccess) {
        return e;
    }
    const BoxSet<double> &F = s->h64.fine;
    const int sl = prof_begin(s, MG_PROF_KRYLOV, st);
    if ((e = launch_pcg(F, s->active, 0, s->pcg_p, s->pcg_q, s->sc, s->partials, s->sc.rzn, st)) !=
            cudaSuccess ||
        (e = launch_pcg_scalars(s->nbox, s->active, 0, s->sc, st)) != cudaSuccess ||
        (e = launch_pcg(F, s->active, 1, s->pcg_p, s->pcg_q, s->sc, nullptr, nullptr, st)) !=
            cudaSuccess ||
        (e = launch_pcg(F, s->active, 2, s->pcg_p, s->pcg_q, s->sc, s->partials, s->sc.pq, st)) !=
            cudaSuccess ||
        (e = launch_pcg_scalars(s->nbox, s->active, 1, s->sc, st)) != cudaSuccess ||
        (e = launch_pcg(F, s->active, 3, s->pcg_p, s->pcg_q, s->sc, s->partials, s->dnorm, st)) !=
            cudaSuccess)
        return e;
    prof_end(s, sl, st);
    return cudaSuccess;
}

static cudaError_t enqueue_body_pcg(Solver *s, cudaStream_t st, cudaGraphConditionalHandle h)
{
    cudaError_t e = enqueue_pcg(s, st);
    if (e != cudaSuccess) return e;
    return launch_judge(s->nbox, s->dnorm, s->dnormf, s->active, s->J, h, 1, st);
}

// Run the whole convergence loop as one graph launch: a conditional WHILE
// node whose body is captured once and whose condition the judge kernel sets.
template <class F>
static int run_loop(Solver *s, cudaGraphExec_t *exec, long long *per_iter, F body,
                    cudaStream_t st)
{
    if (!*exec) {
        cudaGraph_t g = nullptr;
        CK(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        if (e == cudaSuccess) {
            cudaGraph_t bodyg = np.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(s->cap, bodyg, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const long long k0 = launch_counter();
                cudaError_t eb = body(s, s->cap, h);
                *per_iter = launch_counter() - k0;
                s->cap_kernels += *per_iter;
                cudaError_t ee = cudaStreamEndCapture(s->cap, &bodyg);
                e = eb != cudaSuccess ? eb : ee;
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            *exec = nullptr;
            return set_error(MG_ERR_CUDA, "convergence-loop graph: %s", cudaGetErrorString(e));
        }
    }
    CK(cudaGraphLaunch(*exec, st));
    return MG_OK;
}

// Host image of the judge block for the boxes still running; upload.
static int upload_judge(Solver *s, const std::vector<struct BoxState> &bs, double tol,
                        cudaStream_t st);
static int download_judge(Solver *s, std::vector<struct BoxState> &bs, long long per_iter,
                          cudaStream_t st);

#define RUN64(s, st) run_step(s, &(s)->h64.graph, &(s)->slots64, &(s)->graph_kernels64, enqueue_step64, st)
#define RUN32(s, st) run_step(s, &(s)->h32.graph, &(s)->slots32, &(s)->graph_kernels32, enqueue_step32, st)
#define RUNHEAD(s, st) run_step(s, &(s)->h64.head, &(s)->slots_head, &(s)->graph_kernels_head, enqueue_head64, st)
#define RUNTAIL(s, st) run_step(s, &(s)->h64.graph, &(s)->slots64, &(s)->graph_kernels64, enqueue_tail64, st)
#define RUNDOWN0(s, st) run_step(s, &(s)->h32.down0, &(s)->slots_down0, &(s)->graph_kernels_down0, enqueue_inner_down0, st)
#define RUNREST(s, st) run_step(s, &(s)->h32.rest, &(s)->slots_rest, &(s)->graph_kernels_rest, enqueue_inner_rest, st)

// Adaptive inner cycles of one refinement step in the host-judged loop: the
// finest level's down leg (with the exit test), the inner flags read back,
// and the rest of the cycle only while some box is still in; at most
// kInnerMax cycles.  The same work on every box as the device loop's WHILE
// form, whose last cycle runs its rest on no box.
static int run_inner_host(Solver *s, cudaStream_t st)
{
    CK(launch_inner_begin(s->nbox, s->active, s->active32, s->icount, 0, 0, st));
    for (int i = 0; i < kInnerMax; ++i) {
        CKS(RUNDOWN0(s, st));
        CK(cudaMemcpyAsync(s->hflags, s->active32, sizeof(int) * s->nbox, cudaMemcpyDeviceToHost,
                           st));
        CK(cudaStreamSynchronize(st));
        bool any = false;
        for (int b = 0; b < s->nbox; ++b) any = any || s->hflags[b] != 0;
        if (!any) break;
        CKS(RUNREST(s, st));
    }
    return MG_OK;
}

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
// stall_limit: cycles without a 10% gain that end the solve (0: no such rule).
static bool judge(BoxState &B, double rel, double tol, int cycle, int max_cycles,
                  int stall_limit = 5)
{
    if (B.nh < MG_MAX_HIST) B.hist[B.nh++] = rel;
    B.cycles = cycle;
    if (!std::isfinite(rel)) { B.status = MG_ERR_NONFINITE; return true; }
    if (rel <= tol) { B.status = MG_OK; return true; }
    if (rel > 1e3 * std::max(B.rel0, tol)) { B.status = MG_ERR_DIVERGED; return true; }
    if (rel > 0.9 * B.best) ++B.stall;
    else B.stall = 0;
    B.best = std::min(B.best, rel);
    if ((stall_limit > 0 && B.stall >= stall_limit) || cycle >= max_cycles) {
        B.status = MG_ERR_NOT_CONVERGED;
        return true;
    }
    return false;
}

static int upload_judge(Solver *s, const std::vector<BoxState> &bs, double tol,
                        cudaStream_t st)
{
    const int nb = s->nbox;
    char *q = s->hjblock;
    memset(q, 0, s->jbytes);
    double *hist = reinterpret_cast<double *>(q);
    double *rel0 = hist + (size_t)nb * MG_MAX_HIST;
    double *best = rel0 + nb;
    double *tl = best + nb;
    int *status = reinterpret_cast<int *>(tl + 1);
    int *cycles = status + nb;
    int *step = cycles + 2 * nb;
    // look-ahead FP64 loop: the first iteration's norm is of the start
    // iterate, already judged; the device judge starts one step early
    *step = (s->lookahead && !s->has32) ? -1 : 0;
    for (int b = 0; b < nb; ++b) {
        hist[(size_t)b * MG_MAX_HIST] = bs[b].rel0;
        rel0[b] = bs[b].rel0;
        best[b] = bs[b].best;
        status[b] = bs[b].status;
        cycles[b] = 0;
    }
    *tl = tol;
    CK(cudaMemcpyAsync(s->jblock, s->hjblock, s->jbytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(s->icount, 0, 2 * sizeof(int), st));
    return MG_OK;
}

static int download_judge(Solver *s, std::vector<BoxState> &bs, long long per_iter,
                          cudaStream_t st)
{
    CK(cudaMemcpyAsync(s->hjblock, s->jblock, s->jbytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int nb = s->nbox;
    const double *hist = reinterpret_cast<const double *>(s->hjblock);
    const double *tl = hist + (size_t)nb * MG_MAX_HIST + 2 * nb;
    const int *status = reinterpret_cast<const int *>(tl + 1);
    const int *cycles = status + nb;
    const int *step = cycles + 2 * nb;
    s->kernels += per_iter * (long long)(*step + ((s->lookahead && !s->has32) ? 1 : 0));
    if (s->inner_cycle_kernels > 0 && s->has32) {
        // the body counted one inner cycle per step; the WHILE node ran more
        int inner[2] = {0, 0};
        CK(cudaMemcpy(inner, s->icount, sizeof inner, cudaMemcpyDeviceToHost));
        s->kernels += s->inner_cycle_kernels * (long long)std::max(inner[1] - *step, 0);
    }
    for (int b = 0; b < nb; ++b) {
        if (bs[b].done) continue;
        bs[b].status = status[b];
        bs[b].cycles = cycles[b];
        bs[b].done = true;
        const int n = std::min(cycles[b] + 1, MG_MAX_HIST);
        for (int c = 1; c < n; ++c) bs[b].hist[c] = hist[(size_t)b * MG_MAX_HIST + c];
        bs[b].nh = n;
    }
    return MG_OK;
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
                 cudaStream_t stream, bool zero_guess, bool side_copy)
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

    // inputs into the level layout; host inputs come in on the copy stream
    // when the staging buffers are idle (the previous staged call returned
    // after synchronising), overlapping e.g. a set-up still running
    const bool side_in = side_copy && s->stage_clean;
    s->stage_clean = false;
    const double *fd = nullptr, *pd = nullptr;
    bool fst = false, pst = false;
    CKS(device_view(s, f, 0, true, stream, &fd, &fst, -1, side_in));
    // the pack also leaves the partial sums of ||f||^2 (bitwise those of the
    // norm pass), unless the mean of f is removed next
    const bool norm_in_pack = !s->singular;
    CK(launch_pack(H.fine, s->doff, fd, 1, stream, norm_in_pack ? s->partials : nullptr));
    // every wall Neumann: only the zero-mean part of f is in the range of A
    if (s->singular) CK(launch_remove_mean(H.fine, 0, s->partials, s->dmean, stream));
    for (int b = 0; b < nbox; ++b) s->hactive[b] = 1;
    CK(cudaMemcpyAsync(s->active, s->hactive, sizeof(int) * nbox, cudaMemcpyHostToDevice, stream));
    // the persistent launches' barrier word starts every solve at zero (a
    // barrier that gave up in an earlier solve may have left it mid-count)
    if (s->opts.persistent || s->cg_bottom)
        CK(cudaMemsetAsync(s->gbar, 0, sizeof(unsigned), stream));
    if (zero_guess) {
        CK(launch_zero(H.fine, nullptr, stream));
    } else {
        CKS(device_view(s, phi, 1, true, stream, &pd, &pst, -1, side_in));
        CK(launch_pack(H.fine, s->doff, pd, 0, stream));
    }
    // ||f|| and the starting residual r0 = f - A phi0.  In mixed precision
    // r0 comes from refinement step 0 (FP64 residual, no update), which also
    // leaves r32 = r0 / ||f|| and the scales for the first FP32 cycles.
    if (!norm_in_pack) CK(launch_norm_partials(H.fine, nullptr, 1, s->partials, stream));
    CK(launch_norm_finish(H.fine, nullptr, s->partials, s->dnormf, nullptr, nullptr, stream));
    CK(combine(s, s->dnormf, stream));
    if (!mixed && zero_guess) {
        // phi0 = 0: the starting residual is f itself
        CK(cudaMemcpyAsync(s->dnorm, s->dnormf, sizeof(double) * nbox, cudaMemcpyDeviceToDevice,
                           stream));
    } else if (!mixed) {
        CK(exch(s, H.fine, 0, stream));
        CK(launch_norm_partials(H.fine, nullptr, 0, s->partials, stream));
        CK(launch_norm_finish(H.fine, nullptr, s->partials, s->dnorm, nullptr, nullptr, stream));
        CK(combine(s, s->dnorm, stream));
    } else {
        CK(exch(s, H.fine, 0, stream));
        CK(launch_zero(s->h32.fine, nullptr, stream));
        CK(launch_scales(nbox, nullptr, 1, s->dnorm, s->dnormf, s->se, s->sr, s->sr_inv, stream));
        // (zero guess: r0 = f, read without forming the stencil)
        CK(launch_refine_residual(H.fine, s->h32.fine, nullptr, s->sr_inv, s->partials, stream,
                                  zero_guess));
        CK(launch_norm_finish(H.fine, nullptr, s->partials, s->dnorm, nullptr, nullptr, stream,
                              s->sr));
        CK(combine(s, s->dnorm, stream));
        CK(launch_scales(nbox, nullptr, 0, s->dnorm, s->dnormf, s->se, s->sr, s->sr_inv, stream));
    }
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

    const bool device_loop = s->opts.use_graph && !s->prof;
    if (s->pcg) {
        // start: x = phi0 (into phi2), r = f - A x0 (into f), p = 0, then
        // phi = 0 (the first preconditioner's zero start), rz_prev = 0.  The
        // iteration judges the recursively updated residual; a box it
        // declares converged is checked against its true residual f - A x,
        // and restarts from it (at most 3 times) if that is above tol.
        if (any) {
            CK(launch_pcg(H.fine, nullptr, 4, s->pcg_p, s->pcg_q, s->sc, s->partials, s->dnorm,
                          stream));   // ||r0|| (the mixed preconditioner's first scale)
            CK(launch_zero(H.fine, nullptr, stream));
            CK(cudaMemsetAsync(s->sc.rz, 0, sizeof(double) * nbox, stream));
            for (int b = 0; b < nbox; ++b) side[b] = 1;
        }
        if (device_loop && any) {
            CKS(upload_judge(s, bs, tol, stream));
            CKS(run_loop(s, &s->loop_pcg, &s->loop_kernels_pcg, enqueue_body_pcg, stream));
            CKS(download_judge(s, bs, s->loop_kernels_pcg, stream));
            any = false;
        }
        std::vector<char> ran(nbox, 0);
        for (int b = 0; b < nbox; ++b) ran[b] = !bs[b].done || bs[b].cycles > 0;
        for (int restart = 0;; ++restart) {
            // host loop: the boxes still running (all of them without the
            // device loop, the restarted ones after a check)
            while (any) {
                s->rec = &s->direct;
                CK(enqueue_pcg(s, stream));
                s->rec = nullptr;
                CKS(read_norms(s, s->dnorm, s->hnorm, stream));
                if (s->prof) prof_collect(s);
                bool changed = false;
                any = false;
                for (int b = 0; b < nbox; ++b) {
                    if (bs[b].done) continue;
                    if (judge(bs[b], s->hnorm[b] / bs[b].nf, tol, bs[b].cycles + 1,
                              s->opts.max_cycles, 0)) {
                        bs[b].done = true;
                        changed = true;
                    } else {
                        any = true;
                    }
                }
                if (changed && any) CKS(upload_active(s, bs, stream));
            }
            // true residual of the boxes the iteration calls converged
            bool check = false;
            for (int b = 0; b < nbox; ++b) {
                s->hactive[b] = ran[b] && bs[b].status == MG_OK && bs[b].cycles > 0;
                check = check || s->hactive[b];
            }
            if (!check) break;
            CK(cudaMemcpyAsync(s->active, s->hactive, sizeof(int) * nbox, cudaMemcpyHostToDevice,
                               stream));
            CK(launch_pcg(H.fine, s->active, 5, s->pcg_p, s->pcg_q, s->sc, nullptr, nullptr,
                          stream));
            CK(launch_pack(H.fine, s->doff, fd, 1, stream));
            CK(launch_pcg(H.fine, s->active, 4, s->pcg_p, s->pcg_q, s->sc, s->partials, s->dnorm,
                          stream));
            CKS(read_norms(s, s->dnorm, s->hnorm, stream));
            for (int b = 0; b < nbox; ++b) {
                if (!s->hactive[b]) continue;
                const double rel = s->hnorm[b] / bs[b].nf;
                ran[b] = 0;  // checked
                if (bs[b].nh > 0) bs[b].hist[bs[b].nh - 1] = rel;
                if (rel <= tol || restart >= 3 || bs[b].cycles >= s->opts.max_cycles) {
                    if (rel > tol) bs[b].status = MG_ERR_NOT_CONVERGED;
                    continue;
                }
                bs[b].done = false;  // restart from the true residual
                bs[b].status = MG_ERR_NOT_CONVERGED;
                ran[b] = 1;
                any = true;
            }
            if (!any) break;
            CKS(upload_active(s, bs, stream));
            CK(launch_zero(H.fine, s->active, stream));
            CK(cudaMemsetAsync(s->sc.rz, 0, sizeof(double) * nbox, stream));
        }
    }
    if (!mixed && device_loop && any) {
        CKS(upload_judge(s, bs, tol, stream));
        CKS(run_loop(s, &s->loop64, &s->loop_kernels64, enqueue_body64, stream));
        CKS(download_judge(s, bs, s->loop_kernels64, stream));
        any = false;
    }
    if (!mixed && s->lookahead) {
        // iteration i: head (red pass out of place + norm of iterate i-1),
        // judge cycle i-1 (from i = 2 on), rest of cycle i for the boxes left
        for (int i = 1; any; ++i) {
            CKS(RUNHEAD(s, stream));
            CKS(read_norms(s, s->dnorm, s->hnorm, stream));
            if (s->prof) prof_collect(s);
            if (i >= 2) {
                bool changed = false;
                any = false;
                for (int b = 0; b < nbox; ++b) {
                    if (bs[b].done) continue;
                    if (judge(bs[b], s->hnorm[b] / bs[b].nf, tol, i - 1, s->opts.max_cycles)) {
                        bs[b].done = true;
                        changed = true;
                    } else {
                        any = true;
                    }
                }
                if (changed && any) CKS(upload_active(s, bs, stream));
            }
            if (any) CKS(RUNTAIL(s, stream));
        }
    } else if (!mixed) {
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
        // FP64 iterative refinement around FP32 V-cycles: step k >= 1 runs
        // FP32 V-cycles on r32 (inner_cycles of them, or adaptive), then
        // x += se e, the FP64 residual r_k = f - A x, r32 = r_k / sr for the
        // next step and ||r_k|| = sr ||r32|| (step 0 ran above).  The
        // adaptive exit test reads tol from the judge block, uploaded for
        // either loop.
        if (s->inner_adapt && any && !device_loop) CKS(upload_judge(s, bs, tol, stream));
        if (device_loop && any) {
            CKS(upload_judge(s, bs, tol, stream));
            CKS(run_loop(s, &s->loop32, &s->loop_kernels32, enqueue_body32, stream));
            CKS(download_judge(s, bs, s->loop_kernels32, stream));
            any = false;
        }
        for (int k = 1; any; ++k) {
            if (s->inner_adapt) CKS(run_inner_host(s, stream));
            else CKS(RUN32(s, stream));
            s->rec = &s->direct;
            const int sl = prof_begin(s, MG_PROF_REFINE, stream);
            CK(launch_refine_update(H.fine, s->h32.fine, s->active, s->se, stream));
            CK(exch(s, H.fine, 0, stream));
            CK(launch_refine_residual(H.fine, s->h32.fine, s->active, s->sr_inv, s->partials,
                                      stream));
            CK(launch_norm_finish(H.fine, s->active, s->partials, s->dnorm, nullptr, nullptr,
                                  stream, s->sr));
            CK(combine(s, s->dnorm, stream));
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
                if (judge(bs[b], s->hnorm[b] / bs[b].nf, tol, k, s->opts.max_cycles)) {
                    bs[b].done = true;
                    changed = true;
                } else {
                    any = true;
                }
            }
            if (changed && any) CKS(upload_active(s, bs, stream));
        }
    }

    // solution out (every wall Neumann: the zero-mean solution)
    if (s->singular) CK(launch_remove_mean(H.fine, 1, s->partials, s->dmean, stream));
    for (int b = 0; b < nbox; ++b) s->hside[b] = side[b];
    CK(cudaMemcpyAsync(s->dside, s->hside, sizeof(int) * nbox, cudaMemcpyHostToDevice, stream));
    // max-norm statistics: max |f - A phi| / max |f| of the returned solution
    const bool want_max = s->opts.max_norm && st;
    if (want_max) {
        if (s->pcg) CK(launch_pack(H.fine, s->doff, fd, 1, stream));  // f held CG's residual
        if (s->xmode)
            CK(launch_exchange(H.fine, nullptr, s->xrec[0], s->nxrec[0], s->xmax[0], stream));
        CK(launch_max_norm(H.fine, s->dside, 0, s->partials, s->dmean, stream));
        CK(launch_max_norm(H.fine, s->dside, 1, s->partials, s->dinv, stream));
        CK(cudaMemcpyAsync(s->hnorm, s->dmean, sizeof(double) * nbox, cudaMemcpyDeviceToHost,
                           stream));
        CK(cudaMemcpyAsync(s->hnorm + nbox, s->dinv, sizeof(double) * nbox,
                           cudaMemcpyDeviceToHost, stream));
    }
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
    CK(cudaMemcpyAsync(s->hside + nbox, s->derr, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    s->stage_clean = true;
    (void)fst;
    (void)pst;
    s->kernels += (launch_counter() - k0) - (s->cap_kernels - c0);
    if (s->hside[nbox]) {
        // a kernel's bounded wait gave up: the iterate is not trustworthy
        CK(cudaMemsetAsync(s->derr, 0, sizeof(int), stream));
        CK(cudaStreamSynchronize(stream));
        for (int b = 0; b < nbox; ++b) bs[b].status = MG_ERR_TIMEOUT;
    }

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
            if (want_max && s->hnorm[b] > 0.0) o.rel_resid_max = s->hnorm[nbox + b] / s->hnorm[b];
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
    if (s->singular)
        return set_error(MG_ERR_UNSUPPORTED,
                         "no adjoint when A is singular (no Dirichlet wall)");
    if (s->bc >> 6)
        return set_error(MG_ERR_UNSUPPORTED, "no adjoint with periodic axes");
    DeviceGuard gd(s->dev);
    cudaGetLastError();  // drop a stale non-sticky error of an earlier call
    int worst = MG_OK;
    // with shared weights every box is a right-hand side of box 0: one beta,
    // one beta gradient (its first off[1] values)
    const long long nbeta = s->shared ? s->off[1] : s->total;
    const double *dbd = nullptr;
    bool dbst = false;
    CKS(device_view(s, dLdbeta, 2, true, stream, &dbd, &dbst, nbeta));
    double *db = const_cast<double *>(dbd);
    for (int r = 0; r < nrhs; ++r) {
        const size_t o = (size_t)r * s->total;
        int rc = solver_solve(s, g + o, dLdf + o, tol, st ? st + (size_t)r * s->nbox : nullptr,
                              stream, true, false);
        s->stage_clean = false;  // the gradient below still reads staging buffers
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
            const long long ob = s->shared ? 0 : s->off[b];
            s->kernels += 1;
            CK(launch_beta_grad(d[0], d[1], d[2], 1.0 / (s->dx[b] * s->dx[b]), s->bc,
                                s->beta + ob, pd + s->off[b], s->stage_b + s->off[b], db + ob,
                                stream));
        }
    }
    if (dbst)
        CK(cudaMemcpyAsync(dLdbeta, db, sizeof(double) * nbeta, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    s->stage_clean = true;
    if (worst != MG_OK) set_error(worst, "adjoint solve status %d", worst);
    return worst;
}

}  // namespace mg

// ================================================================ C ABI ====

using namespace mg;

struct mg_ctx {
    Solver *s;
    Solver *multi = nullptr;     // nrhs right-hand sides as one shared-weight batch
    int multi_n = 0;
    long long beta_version = 0;  // bumped by every mg_set_beta
    long long multi_version = -1;
};

// The shared-weight batch for nrhs right-hand sides, created on first use and
// given the context's current beta.
static int multi_solver(mg_ctx *ctx, int nrhs, cudaStream_t st, Solver **out)
{
    Solver *s = ctx->s;
    if (!s->beta_set) return set_error(MG_ERR_INVALID_ARG, "mg_set_beta was not called");
    if (ctx->multi && ctx->multi_n != nrhs) {
        solver_destroy(ctx->multi);
        ctx->multi = nullptr;
    }
    if (!ctx->multi) {
        std::vector<std::array<int, 3>> n(nrhs, s->n[0]);
        std::vector<double> dx(nrhs, s->dx[0]);
        int rc = solver_create(&ctx->multi, nrhs, reinterpret_cast<const int(*)[3]>(n.data()),
                               dx.data(), s->bc, &s->opts, true);
        if (rc != MG_OK) {
            ctx->multi = nullptr;
            return rc;
        }
        ctx->multi_n = nrhs;
        ctx->multi_version = -1;
    }
    if (ctx->multi_version != ctx->beta_version) {
        int rc = solver_set_beta(ctx->multi, s->beta, st);
        if (rc != MG_OK) return rc;
        ctx->multi_version = ctx->beta_version;
    }
    ctx->multi->prof = s->prof;
    *out = ctx->multi;
    return MG_OK;
}
struct mg_batch {
    Solver *s;
};
struct mg_level {
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
    ++ctx->beta_version;
    return solver_set_beta(ctx->s, beta, (cudaStream_t)stream);
}

int mg_solve(mg_ctx *ctx, const double *f, double *phi, double tol, mg_stats *st, void *stream)
{
    if (!ctx) return set_error(MG_ERR_INVALID_ARG, "NULL context");
    return solver_solve(ctx->s, f, phi, tol, st, (cudaStream_t)stream, false);
}

int mg_solve_ex(mg_ctx *ctx, int nrhs, const double *f, double *phi, double tol, int flags,
                mg_stats *st, void *stream)
{
    if (!ctx || nrhs < 1 || !f || !phi)
        return set_error(MG_ERR_INVALID_ARG, "NULL argument or nrhs < 1");
    if (flags & ~MG_ZERO_GUESS) return set_error(MG_ERR_INVALID_ARG, "unknown flags");
    const bool zero = (flags & MG_ZERO_GUESS) != 0;
    if (nrhs == 1) return solver_solve(ctx->s, f, phi, tol, st, (cudaStream_t)stream, zero);
    Solver *m = nullptr;
    CKS(multi_solver(ctx, nrhs, (cudaStream_t)stream, &m));
    return solver_solve(m, f, phi, tol, st, (cudaStream_t)stream, zero);
}
int mg_solve_multi(mg_ctx *ctx, int nrhs, const double *f, double *phi, double tol, mg_stats *st,
                   void *stream)
{
    if (!ctx || nrhs < 1 || !f || !phi)
        return set_error(MG_ERR_INVALID_ARG, "NULL argument or nrhs < 1");
    if (nrhs == 1) return solver_solve(ctx->s, f, phi, tol, st, (cudaStream_t)stream, false);
    Solver *m = nullptr;
    CKS(multi_solver(ctx, nrhs, (cudaStream_t)stream, &m));
    return solver_solve(m, f, phi, tol, st, (cudaStream_t)stream, false);
}

int mg_adjoint(mg_ctx *ctx, int nrhs, const double *phi, const double *g, double *dLdf,
               double *dLdbeta, double tol, mg_stats *st, void *stream)
{
    if (!ctx) return set_error(MG_ERR_INVALID_ARG, "NULL context");
    if (nrhs <= 1)
        return solver_adjoint(ctx->s, nrhs, phi, g, dLdf, dLdbeta, tol, st, (cudaStream_t)stream);
    Solver *m = nullptr;
    CKS(multi_solver(ctx, nrhs, (cudaStream_t)stream, &m));
    return solver_adjoint(m, 1, phi, g, dLdf, dLdbeta, tol, st, (cudaStream_t)stream);
}

int mg_project_rhs(mg_ctx *ctx, const double *u, const double *v, const double *w,
                   const double *S, double *f, void *stream)
{
    if (!ctx || !u || !v || !w || !f) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    Solver *s = ctx->s;
    DeviceGuard g(s->dev);
    cudaGetLastError();
    const auto &n = s->n[0];
    CK(launch_project_rhs(n[0], n[1], n[2], s->dx[0], u, v, w, S, f, (cudaStream_t)stream));
    s->kernels += 1;
    return MG_OK;
}

int mg_project_correct(mg_ctx *ctx, const double *phi, double *u, double *v, double *w,
                       void *stream)
{
    if (!ctx || !phi || !u || !v || !w) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    Solver *s = ctx->s;
    if (!s->beta_set) return set_error(MG_ERR_INVALID_ARG, "mg_set_beta was not called");
    DeviceGuard g(s->dev);
    cudaGetLastError();
    const auto &n = s->n[0];
    const LevelBufs<double> &L = s->h64.lv[0][0];
    if (s->bc >> 6)
        return set_error(MG_ERR_UNSUPPORTED, "projection with periodic axes is not implemented");
    CK(launch_project_correct(n[0], n[1], n[2], s->dx[0], L.wx, L.wy, L.wz, phi, u, v, w,
                              (cudaStream_t)stream, s->wide));
    s->kernels += 1;
    return MG_OK;
}

int mg_bc_lift(mg_ctx *ctx, const double *vals, const double *f, double *f_out, void *stream)
{
    if (!ctx || !vals || !f || !f_out) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    Solver *s = ctx->s;
    if (!s->beta_set) return set_error(MG_ERR_INVALID_ARG, "mg_set_beta was not called");
    DeviceGuard g(s->dev);
    cudaGetLastError();
    const auto &n = s->n[0];
    const LevelBufs<double> &L = s->h64.lv[0][0];
    CK(launch_bc_lift(n[0], n[1], n[2], 1.0 / s->dx[0], s->bc, L.wx, L.wy, L.wz, vals, f, f_out,
                      (cudaStream_t)stream, s->wide));
    s->kernels += 1;
    return MG_OK;
}

int mg_smoother_kind(const mg_ctx *ctx, int level, int *kind)
{
    if (!ctx || !kind) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    const Solver *s = ctx->s;
    if (level < 0 || level >= s->nlev[0])
        return set_error(MG_ERR_INVALID_ARG, "level %d outside 0..%d", level, s->nlev[0] - 1);
    *kind = 0;
    auto of = [&](const auto &H) {
        if (level < (int)H.fused.size() && H.fused[level] && H.smooth[level].nbox > 0)
            *kind = H.maps[level] ? 2 : 1;
    };
    if (s->has32) of(s->h32);
    else of(s->h64);
    return MG_OK;
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
    solver_destroy(ctx->multi);
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
int mg_solve_batched_ex(mg_batch *b, const double *f, double *phi, double tol, int flags,
                        mg_stats *st, void *stream)
{
    if (!b) return set_error(MG_ERR_INVALID_ARG, "NULL batch");
    if (flags & ~MG_ZERO_GUESS) return set_error(MG_ERR_INVALID_ARG, "unknown flags");
    return solver_solve(b->s, f, phi, tol, st, (cudaStream_t)stream, (flags & MG_ZERO_GUESS) != 0);
}

void mg_batch_destroy(mg_batch *b)
{
    if (!b) return;
    solver_destroy(b->s);
    delete b;
}

int mg_level_create(mg_level **out, int nbox, const int (*lo)[3], const int (*n)[3], double dx,
                    int bc, const mg_opts *opts)
{
    if (!out || !lo || !n || nbox < 1) return set_error(MG_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    if (!(dx > 0.0) || !std::isfinite(dx)) return set_error(MG_ERR_INVALID_ARG, "dx must be > 0");
    std::vector<double> dxs(nbox, dx);
    Solver *s = nullptr;
    int rc = solver_create(&s, nbox, n, dxs.data(), bc, opts, false, lo);
    if (rc != MG_OK) return rc;
    *out = new mg_level{s};
    return MG_OK;
}

int mg_level_set_beta(mg_level *lv, const double *beta, void *stream)
{
    if (!lv) return set_error(MG_ERR_INVALID_ARG, "NULL level");
    return solver_set_beta(lv->s, beta, (cudaStream_t)stream);
}

int mg_level_solve(mg_level *lv, const double *f, double *phi, double tol, mg_stats *st,
                   void *stream)
{
    if (!lv) return set_error(MG_ERR_INVALID_ARG, "NULL level");
    return solver_solve(lv->s, f, phi, tol, st, (cudaStream_t)stream, false);
}
int mg_level_solve_ex(mg_level *lv, const double *f, double *phi, double tol, int flags,
                      mg_stats *st, void *stream)
{
    if (!lv) return set_error(MG_ERR_INVALID_ARG, "NULL level");
    if (flags & ~MG_ZERO_GUESS) return set_error(MG_ERR_INVALID_ARG, "unknown flags");
    return solver_solve(lv->s, f, phi, tol, st, (cudaStream_t)stream, (flags & MG_ZERO_GUESS) != 0);
}

int mg_level_levels(const mg_level *lv, int *nlev)
{
    if (!lv || !nlev) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    *nlev = lv->s->nlev[0];
    return MG_OK;
}

void mg_level_destroy(mg_level *lv)
{
    if (!lv) return;
    solver_destroy(lv->s);
    delete lv;
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
    int rc = profile_read(ctx->s, out, reset);
    if (rc == MG_OK && ctx->multi) {
        // the shared-weight batch's kernels belong to this context too
        mg_profile m;
        profile_read(ctx->multi, &m, reset);
        out->kernels += m.kernels;
        for (int k = 0; k < MG_PROF_NKIND; ++k) {
            out->ms[k] += m.ms[k];
            out->launches[k] += m.launches[k];
        }
    }
    return rc;
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
int mg_level_profile_enable(mg_level *lv, int on)
{
    if (!lv) return set_error(MG_ERR_INVALID_ARG, "NULL level");
    return profile_enable(lv->s, on);
}
int mg_level_profile_read(mg_level *lv, mg_profile *out, int reset)
{
    if (!lv) return set_error(MG_ERR_INVALID_ARG, "NULL level");
    return profile_read(lv->s, out, reset);
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
