// slab.cu -- one box split in z into slabs, each slab on its own GPU
// (mg_slab_*, include/mg.h).
//
// The paper's codes distribute the grids of a level over MPI ranks and fill
// their ghost cells from the neighbouring grids before every stencil (paper
// Sec. 2); MAESTRO's linear solves are what limits its scaling (Sec. 3).
// Here the analogue for one large box on several GPUs: slab r holds planes
// z0[r] .. z0[r+1]-1 on its own device, in the wide level layout (a guard
// plane below and above).  Every level down to the gather level is smoothed
// slab-parallel: before each single-colour pass and each residual, each slab
// pulls its neighbours' boundary planes of phi into its guard planes (one
// copy per interface and direction, cudaMemcpyPeerAsync: peer copies into a
// local halo buffer).  At the gather level the whole box is small (at most
// 32^3 cells, or the slabs cannot halve further): the slabs' restriction
// writes straight into the level-0 arrays of one coarse context on the first
// device, which runs the rest of the V-cycle alone, and the slabs'
// prolongation reads its correction back from there.  The residual norm is
// the sum of the slabs' squared norms, taken on the host once per cycle.
//
// Each slab is a one-box coupled-level context (solver.cu) cut at the
// gather level; its descriptors for that level are re-pointed at the coarse
// context's arrays.  The interfaces' face weights are harmonic means over
// the two slabs' cells (the slabs exchange their boundary planes of beta
// before the face step), and both slabs of an interface compute its coarse
// faces from the same values, so the slab solve is the single-box solve of
// the same operator.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "solver.h"

namespace mg {
namespace {

constexpr long long kGatherCells = 32768;   // a level of at most 32^3 cells is gathered

#define SCK(call)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return set_error(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,        \
                             "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,         \
                             __LINE__);                                                         \
    } while (0)
#define SCKS(expr)                   \
    do {                             \
        int s_ = (expr);             \
        if (s_ != MG_OK) return s_;  \
    } while (0)

struct DevSwitch {
    int prev = -1;
    DevSwitch() { cudaGetDevice(&prev); }
    ~DevSwitch()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct SlabPlan {
    int n[3] = {0, 0, 0};
    int nslab = 0;
    int gather = 0;        // level solved by the coarse context
    std::vector<int> z0;   // [nslab + 1] first plane of each slab, level 0
};

// Equal slabs of nz / nslab planes.  Levels halve (all dims) while the
// level has more than 32^3 cells, its dims are even and >= 4 (the one-box
// rule) and every slab keeps an even thickness; the level where that stops is
// gathered.
int make_plan(const int n[3], int nslab, SlabPlan *p)
{
    if (!n || n[0] < 1 || n[1] < 1 || n[2] < 1)
        return set_error(MG_ERR_INVALID_ARG, "slab plan: need n >= 1");
    if (nslab < 1 || nslab > 64)
        return set_error(MG_ERR_INVALID_ARG, "slab plan: nslab must be in 1..64");
    if (n[2] % nslab)
        return set_error(MG_ERR_UNSUPPORTED, "slab plan: nz = %d is not a multiple of %d slabs",
                         n[2], nslab);
    p->n[0] = n[0];
    p->n[1] = n[1];
    p->n[2] = n[2];
    p->nslab = nslab;
    p->z0.resize(nslab + 1);
    const int t0 = n[2] / nslab;
    for (int r = 0; r <= nslab; ++r) p->z0[r] = r * t0;
    int d[3] = {n[0], n[1], n[2]}, t = t0, L = 0;
    while ((long long)d[0] * d[1] * d[2] > kGatherCells) {
        bool ok = t % 2 == 0 && t >= 2;
        for (int q = 0; q < 3; ++q) ok = ok && d[q] % 2 == 0 && d[q] >= 4;
        if (!ok) break;
        for (int q = 0; q < 3; ++q) d[q] /= 2;
        t /= 2;
        ++L;
    }
    if (L == 0)
        return set_error(MG_ERR_UNSUPPORTED,
                         "slab plan: no level to smooth slab by slab (the box has at most 32^3 "
                         "cells, or its dims or slab thickness do not halve)");
    p->gather = L;
    return MG_OK;
}

// Halo copies of one level: slab r's top plane into slab r+1's lower guard
// plane, slab r+1's bottom plane into slab r's upper guard plane.
struct HaloRec {
    int src, src_k, dst, dst_k;
};
std::vector<HaloRec> halo_records(const SlabPlan &p, int level)
{
    std::vector<HaloRec> out;
    const int t = (p.z0[1] - p.z0[0]) >> level;
    for (int r = 0; r + 1 < p.nslab; ++r) {
        out.push_back({r, t - 1, r + 1, -1});
        out.push_back({r + 1, 0, r, t});
    }
    return out;
}

}  // namespace

struct SlabCtx {
    SlabPlan plan;
    mg_opts opts{};
    std::vector<int> dev;             // [slab]
    std::vector<Solver *> sl;         // [slab] one-box coupled contexts cut at the gather level
    Solver *coarse = nullptr;         // the gather level and below, on dev[0]
    std::vector<cudaStream_t> st;     // [slab]
    cudaStream_t cst = nullptr;       // coarse context's stream
    std::vector<cudaEvent_t> ev_a, ev_b;  // [slab]
    cudaEvent_t ev_c = nullptr;
    double *hnorm = nullptr;          // pinned [slab]
    bool beta_set = false;
};

namespace {

// Level arrays of slab r at level l.
struct SlabLevel {
    double *phi, *f, *wx, *wy, *wz;
    int nx, ny, nz, P;
    long long Q;
};
SlabLevel slab_level(const SlabCtx *c, int r, int l)
{
    const Solver *s = c->sl[r];
    const LevelBufs<double> &L = s->h64.lv[0][l];
    const auto &d = s->dims[0][l];
    SlabLevel o;
    o.phi = L.phi;
    o.f = L.f;
    o.wx = L.wx;
    o.wy = L.wy;
    o.wz = L.wz;
    o.nx = d[0];
    o.ny = d[1];
    o.nz = d[2];
    o.P = (int)pitch_row(d[0], true);
    o.Q = pitch_plane(d[0], d[1], true);
    return o;
}

// Ghost exchange of level l's phi between neighbouring slabs.  Each slab
// first waits until its neighbours have finished the stage before (their
// boundary planes are final), pulls those planes into its guard planes on
// its own stream, and then every slab waits until its neighbours have
// pulled its boundary planes before it may change them again.
int exchange(SlabCtx *c, int l)
{
    const int R = c->plan.nslab;
    if (R < 2) return MG_OK;
    for (int r = 0; r < R; ++r) {
        SCK(cudaSetDevice(c->dev[r]));
        SCK(cudaEventRecord(c->ev_a[r], c->st[r]));
    }
    for (const HaloRec &h : halo_records(c->plan, l)) {
        const SlabLevel S = slab_level(c, h.src, l), D = slab_level(c, h.dst, l);
        SCK(cudaSetDevice(c->dev[h.dst]));
        SCK(cudaStreamWaitEvent(c->st[h.dst], c->ev_a[h.src], 0));
        const size_t bytes = sizeof(double) * ((size_t)(D.ny - 1) * D.P + D.nx);
        SCK(cudaMemcpyPeerAsync(D.phi + (long long)h.dst_k * D.Q, c->dev[h.dst],
                                S.phi + (long long)h.src_k * S.Q, c->dev[h.src], bytes,
                                c->st[h.dst]));
    }
    for (int r = 0; r < R; ++r) {
        SCK(cudaSetDevice(c->dev[r]));
        SCK(cudaEventRecord(c->ev_b[r], c->st[r]));
    }
    for (int r = 0; r < R; ++r) {
        SCK(cudaSetDevice(c->dev[r]));
        if (r > 0) SCK(cudaStreamWaitEvent(c->st[r], c->ev_b[r - 1], 0));
        if (r + 1 < R) SCK(cudaStreamWaitEvent(c->st[r], c->ev_b[r + 1], 0));
    }
    return MG_OK;
}

// The coarse context's stream waits for every slab (join), or every slab
// for the coarse context (fork).
int join(SlabCtx *c)
{
    for (int r = 0; r < c->plan.nslab; ++r) {
        SCK(cudaSetDevice(c->dev[r]));
        SCK(cudaEventRecord(c->ev_a[r], c->st[r]));
        SCK(cudaSetDevice(c->dev[0]));
        SCK(cudaStreamWaitEvent(c->cst, c->ev_a[r], 0));
    }
    return MG_OK;
}
int fork_out(SlabCtx *c)
{
    SCK(cudaSetDevice(c->dev[0]));
    SCK(cudaEventRecord(c->ev_c, c->cst));
    for (int r = 0; r < c->plan.nslab; ++r) {
        SCK(cudaSetDevice(c->dev[r]));
        SCK(cudaStreamWaitEvent(c->st[r], c->ev_c, 0));
    }
    return MG_OK;
}

// Re-point slab r's last smoothed level (gather - 1) at the coarse
// context's level-0 arrays: its restriction writes the coarse right-hand
// side (and zeroes the coarse guess) there, its prolongation reads the
// coarse correction from there, its set-up coarsening writes the coarse
// face weights there.  Cell (I, J, K) of the slab's coarse range is cell
// (I, J, K + zc) of the coarse box.
int link_coarse(SlabCtx *c, int r)
{
    Solver *s = c->sl[r];
    const int g = c->plan.gather;
    const int zc = c->plan.z0[r] >> g;
    const LevelBufs<double> &C = c->coarse->h64.lv[0][0];
    const auto &cd = c->coarse->dims[0][0];
    const int cP = (int)pitch_row(cd[0]);
    const long long cQ = pitch_plane(cd[0], cd[1]);
    SCK(cudaSetDevice(c->dev[r]));
    Box<double> B;
    Box<double> *bp = const_cast<Box<double> *>(s->h64.smooth[g - 1].boxes);
    SCK(cudaMemcpy(&B, bp, sizeof B, cudaMemcpyDeviceToHost));
    B.phic = C.phi + (long long)zc * cQ;
    B.fc = C.f + (long long)zc * cQ;
    B.cP = cP;
    B.cQ = cQ;
    B.cpar = zc & 1;
    SCK(cudaMemcpy(bp, &B, sizeof B, cudaMemcpyHostToDevice));
    SetupBox U;
    SetupBox *up = const_cast<SetupBox *>(s->setup_coarsen[g - 1].boxes);
    SCK(cudaMemcpy(&U, up, sizeof U, cudaMemcpyDeviceToHost));
    U.cwx = C.wx + (long long)zc * cQ;
    U.cwy = C.wy + (long long)zc * cQ;
    U.cwz = C.wz + (long long)zc * cQ;
    U.cP = cP;
    U.cQ = cQ;
    SCK(cudaMemcpy(up, &U, sizeof U, cudaMemcpyHostToDevice));
    return MG_OK;
}

void destroy(SlabCtx *c)
{
    if (!c) return;
    DevSwitch keep;
    for (size_t r = 0; r < c->sl.size(); ++r) {
        cudaSetDevice(c->dev[r]);
        if (r < c->st.size() && c->st[r]) cudaStreamSynchronize(c->st[r]);
    }
    if (c->cst) {
        cudaSetDevice(c->dev[0]);
        cudaStreamSynchronize(c->cst);
    }
    for (size_t r = 0; r < c->sl.size(); ++r) {
        cudaSetDevice(c->dev[r]);
        if (c->sl[r]) solver_destroy(c->sl[r]);
        if (r < c->st.size() && c->st[r]) cudaStreamDestroy(c->st[r]);
        if (r < c->ev_a.size() && c->ev_a[r]) cudaEventDestroy(c->ev_a[r]);
        if (r < c->ev_b.size() && c->ev_b[r]) cudaEventDestroy(c->ev_b[r]);
    }
    if (!c->dev.empty()) cudaSetDevice(c->dev[0]);
    if (c->coarse) solver_destroy(c->coarse);
    if (c->cst) cudaStreamDestroy(c->cst);
    if (c->ev_c) cudaEventDestroy(c->ev_c);
    if (c->hnorm) cudaFreeHost(c->hnorm);
    delete c;
}

// One V-cycle: slab-parallel levels down to the gather level, the coarse
// context's V-cycle there, slab-parallel levels up again.
int vcycle(SlabCtx *c)
{
    const int R = c->plan.nslab, g = c->plan.gather;
    const mg_opts &o = c->opts;
    const bool red = o.nu1 > 0 && !o.full_residual;
    for (int l = 0; l < g; ++l) {
        for (int sw = 0; sw < o.nu1; ++sw)
            for (int color = 0; color < 2; ++color) {
                SCKS(exchange(c, l));
                for (int r = 0; r < R; ++r) {
                    SCK(cudaSetDevice(c->dev[r]));
                    SCK(launch_rbgs_pass(c->sl[r]->h64.smooth[l], c->sl[r]->active, color,
                                         c->st[r]));
                }
            }
        SCKS(exchange(c, l));
        for (int r = 0; r < R; ++r) {
            SCK(cudaSetDevice(c->dev[r]));
            const BoxSet<double> &S = c->sl[r]->h64.smooth[l];
            SCK(red ? launch_resid_restrict_red(S, c->sl[r]->active, c->st[r])
                    : launch_resid_restrict(S, c->sl[r]->active, c->st[r]));
        }
    }
    SCKS(join(c));
    SCK(cudaSetDevice(c->dev[0]));
    SCK(solver_enqueue_vcycle64(c->coarse, c->cst));
    SCKS(fork_out(c));
    for (int l = g - 1; l >= 0; --l) {
        for (int r = 0; r < R; ++r) {
            SCK(cudaSetDevice(c->dev[r]));
            SCK(launch_prolong(c->sl[r]->h64.smooth[l], c->sl[r]->active, c->st[r]));
        }
        for (int sw = 0; sw < o.nu2; ++sw)
            for (int color = 0; color < 2; ++color) {
                SCKS(exchange(c, l));
                for (int r = 0; r < R; ++r) {
                    SCK(cudaSetDevice(c->dev[r]));
                    SCK(launch_rbgs_pass(c->sl[r]->h64.smooth[l], c->sl[r]->active, color,
                                         c->st[r]));
                }
            }
    }
    return MG_OK;
}

// ||f||^2 (field 1) or ||f - A phi||^2 (field 0) of every slab into hnorm,
// and their sum.
int norm2(SlabCtx *c, int field, double *sum)
{
    const int R = c->plan.nslab;
    if (field == 0) SCKS(exchange(c, 0));
    for (int r = 0; r < R; ++r) {
        Solver *s = c->sl[r];
        SCK(cudaSetDevice(c->dev[r]));
        SCK(launch_norm_partials(s->h64.fine, nullptr, field == 0 ? 0 : 1, s->partials,
                                 c->st[r]));
        SCK(launch_norm_finish(s->h64.fine, nullptr, s->partials, s->dnorm, nullptr, nullptr,
                               c->st[r]));
        SCK(cudaMemcpyAsync(c->hnorm + r, s->dnorm, sizeof(double), cudaMemcpyDeviceToHost,
                            c->st[r]));
    }
    double t = 0.0;
    for (int r = 0; r < R; ++r) {
        SCK(cudaSetDevice(c->dev[r]));
        SCK(cudaStreamSynchronize(c->st[r]));
        t += c->hnorm[r] * c->hnorm[r];   // fixed slab order
    }
    *sum = t;
    return MG_OK;
}

bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace mg

using namespace mg;

struct mg_slab {
    SlabCtx *c;
};

extern "C" {

int mg_slab_plan(const int n[3], int nslab, int *z0, int *gather_level)
{
    SlabPlan p;
    SCKS(make_plan(n, nslab, &p));
    if (z0)
        for (int r = 0; r <= nslab; ++r) z0[r] = p.z0[r];
    if (gather_level) *gather_level = p.gather;
    return MG_OK;
}

int mg_slab_halo(const int n[3], int nslab, int level, int *nrec, int *out, int cap)
{
    SlabPlan p;
    SCKS(make_plan(n, nslab, &p));
    if (!nrec) return set_error(MG_ERR_INVALID_ARG, "nrec is NULL");
    if (level < 0 || level >= p.gather)
        return set_error(MG_ERR_INVALID_ARG, "level %d outside the slab levels 0..%d", level,
                         p.gather - 1);
    const std::vector<HaloRec> recs = halo_records(p, level);
    *nrec = (int)recs.size();
    if (out)
        for (int i = 0; i < (int)recs.size() && i < cap; ++i) {
            out[4 * i] = recs[i].src;
            out[4 * i + 1] = recs[i].src_k;
            out[4 * i + 2] = recs[i].dst;
            out[4 * i + 3] = recs[i].dst_k;
        }
    return MG_OK;
}

int mg_slab_create(mg_slab **out, const int n[3], double dx, int nslab, const int *devices,
                   const mg_opts *opts)
{
    if (!out) return set_error(MG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!(dx > 0.0) || !std::isfinite(dx)) return set_error(MG_ERR_INVALID_ARG, "need dx > 0");
    SlabPlan plan;
    SCKS(make_plan(n, nslab, &plan));
    mg_opts o;
    mg_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != MG_FP64 || o.krylov || o.persistent)
        return set_error(MG_ERR_UNSUPPORTED,
                         "slab-decomposed boxes run FP64 V-cycles (no mixed precision, krylov "
                         "or persistent launches)");
    int ndev = 0;
    SCK(cudaGetDeviceCount(&ndev));
    DevSwitch keep;
    SlabCtx *c = new SlabCtx();
    c->plan = plan;
    c->opts = o;
    c->dev.resize(nslab);
    for (int r = 0; r < nslab; ++r) {
        int d = 0;
        if (devices) d = devices[r];
        else cudaGetDevice(&d);
        if (d < 0 || d >= ndev) {
            destroy(c);
            return set_error(MG_ERR_INVALID_ARG, "slab %d: device %d of %d", r, d, ndev);
        }
        c->dev[r] = d;
    }
    // slabs on other devices reach the coarse context's arrays directly
    for (int r = 0; r < nslab; ++r) {
        if (c->dev[r] == c->dev[0]) continue;
        int can = 0;
        cudaDeviceCanAccessPeer(&can, c->dev[r], c->dev[0]);
        int back = 0;
        cudaDeviceCanAccessPeer(&back, c->dev[0], c->dev[r]);
        if (!can || !back) {
            destroy(c);
            return set_error(MG_ERR_UNSUPPORTED, "devices %d and %d have no peer access",
                             c->dev[r], c->dev[0]);
        }
        for (int k = 0; k < 2; ++k) {
            cudaSetDevice(k ? c->dev[0] : c->dev[r]);
            cudaError_t e = cudaDeviceEnablePeerAccess(k ? c->dev[r] : c->dev[0], 0);
            if (e != cudaSuccess && e != cudaErrorPeerAccessAlreadyEnabled) {
                destroy(c);
                return set_error(MG_ERR_CUDA, "cudaDeviceEnablePeerAccess: %s",
                                 cudaGetErrorString(e));
            }
            cudaGetLastError();
        }
    }
    mg_opts so = o;
    so.use_graph = 0;
    const int t = plan.z0[1] - plan.z0[0];
    c->sl.assign(nslab, nullptr);
    c->st.assign(nslab, nullptr);
    c->ev_a.assign(nslab, nullptr);
    c->ev_b.assign(nslab, nullptr);
    for (int r = 0; r < nslab; ++r) {
        cudaSetDevice(c->dev[r]);
        const int nn[1][3] = {{n[0], n[1], t}};
        const int lo[1][3] = {{0, 0, plan.z0[r]}};
        int rc = solver_create(&c->sl[r], 1, nn, &dx, 0, &so, false, lo, plan.gather + 1);
        if (rc != MG_OK) {
            destroy(c);
            return rc;
        }
        if (cudaStreamCreateWithFlags(&c->st[r], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_a[r], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_b[r], cudaEventDisableTiming) != cudaSuccess) {
            destroy(c);
            return set_error(MG_ERR_CUDA, "slab streams / events: %s",
                             cudaGetErrorString(cudaGetLastError()));
        }
    }
    cudaSetDevice(c->dev[0]);
    const int g = plan.gather;
    const int cn[1][3] = {{n[0] >> g, n[1] >> g, n[2] >> g}};
    const double cdx = std::ldexp(dx, g);
    int rc = solver_create(&c->coarse, 1, cn, &cdx, 0, &so);
    if (rc != MG_OK) {
        destroy(c);
        return rc;
    }
    if (cudaStreamCreateWithFlags(&c->cst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_c, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&c->hnorm, sizeof(double) * nslab) != cudaSuccess) {
        destroy(c);
        return set_error(MG_ERR_CUDA, "coarse stream / host buffer: %s",
                         cudaGetErrorString(cudaGetLastError()));
    }
    for (int r = 0; r < nslab; ++r) {
        rc = link_coarse(c, r);
        if (rc != MG_OK) {
            destroy(c);
            return rc;
        }
    }
    *out = new mg_slab{c};
    return MG_OK;
}

int mg_slab_set_beta(mg_slab *sb, const double *const *beta)
{
    if (!sb || !beta) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    SlabCtx *c = sb->c;
    const int R = c->plan.nslab, g = c->plan.gather;
    for (int r = 0; r < R; ++r)
        if (!beta[r] || !on_device(beta[r], c->dev[r]))
            return set_error(MG_ERR_INVALID_ARG, "beta of slab %d is not memory of device %d", r,
                             c->dev[r]);
    DevSwitch keep;
    // each slab's beta into its level-0 layout (staged in phi), guard cells
    // -1 (walls), then the neighbours' boundary planes of beta into the
    // interface guards, so that the face step forms the harmonic mean there
    for (int r = 0; r < R; ++r) {
        Solver *s = c->sl[r];
        SCK(cudaSetDevice(c->dev[r]));
        SCK(cudaMemcpyAsync(s->beta, beta[r], sizeof(double) * s->total,
                            cudaMemcpyDeviceToDevice, c->st[r]));
        SCK(launch_guard_fill(s->h64.fine, -1.0, c->st[r]));
        SCK(launch_pack(s->h64.fine, s->doff, s->beta, 0, c->st[r]));
    }
    SCKS(exchange(c, 0));
    for (int r = 0; r < R; ++r) {
        Solver *s = c->sl[r];
        SCK(cudaSetDevice(c->dev[r]));
        SCK(launch_setup(s->setup_lv[0], 4, c->st[r]));
        for (int l = 0; l + 1 < g; ++l) SCK(launch_setup(s->setup_coarsen[l], 1, c->st[r]));
        for (int l = 0; l < g; ++l) SCK(launch_setup(s->setup_lv[l], 2, c->st[r]));
        SCK(launch_guard_fill(s->h64.fine, 0.0, c->st[r]));
    }
    // the last coarsening writes the coarse context's level-0 weights; two
    // neighbouring slabs write the same values on their shared face plane,
    // so they take turns
    for (int r = 0; r < R; ++r) {
        SCK(cudaSetDevice(c->dev[r]));
        if (r > 0) SCK(cudaStreamWaitEvent(c->st[r], c->ev_a[r - 1], 0));
        SCK(launch_setup(c->sl[r]->setup_coarsen[g - 1], 1, c->st[r]));
        SCK(cudaEventRecord(c->ev_a[r], c->st[r]));
    }
    SCKS(join(c));
    SCK(cudaSetDevice(c->dev[0]));
    SCKS(solver_setup_from_weights(c->coarse, c->cst));
    SCKS(fork_out(c));
    for (int r = 0; r < R; ++r) {
        SCK(cudaSetDevice(c->dev[r]));
        SCK(cudaStreamSynchronize(c->st[r]));
    }
    SCK(cudaSetDevice(c->dev[0]));
    SCK(cudaStreamSynchronize(c->cst));
    c->beta_set = true;
    return MG_OK;
}

int mg_slab_solve(mg_slab *sb, const double *const *f, double *const *phi, double tol, int flags,
                  mg_stats *st)
{
    if (!sb || !f || !phi) return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    if (!(tol > 0.0)) return set_error(MG_ERR_INVALID_ARG, "tol must be > 0");
    SlabCtx *c = sb->c;
    if (!c->beta_set) return set_error(MG_ERR_INVALID_ARG, "mg_slab_set_beta was not called");
    const int R = c->plan.nslab;
    for (int r = 0; r < R; ++r)
        if (!f[r] || !phi[r] || !on_device(f[r], c->dev[r]) || !on_device(phi[r], c->dev[r]))
            return set_error(MG_ERR_INVALID_ARG, "f or phi of slab %d is not memory of device %d",
                             r, c->dev[r]);
    DevSwitch keep;
    const auto t0 = std::chrono::steady_clock::now();
    const bool zero = (flags & MG_ZERO_GUESS) != 0;
    const int one = 1;
    for (int r = 0; r < R; ++r) {
        Solver *s = c->sl[r];
        SCK(cudaSetDevice(c->dev[r]));
        SCK(cudaMemcpyAsync(s->active, &one, sizeof(int), cudaMemcpyHostToDevice, c->st[r]));
        SCK(launch_pack(s->h64.fine, s->doff, f[r], 1, c->st[r]));
        if (zero) SCK(launch_zero(s->h64.fine, nullptr, c->st[r]));
        else SCK(launch_pack(s->h64.fine, s->doff, phi[r], 0, c->st[r]));
    }
    SCK(cudaSetDevice(c->dev[0]));
    SCK(cudaMemcpyAsync(c->coarse->active, &one, sizeof(int), cudaMemcpyHostToDevice, c->cst));
    double nf2 = 0.0, r2 = 0.0;
    SCKS(norm2(c, 1, &nf2));
    const double nf = std::sqrt(nf2);
    if (zero) r2 = nf2;
    else SCKS(norm2(c, 0, &r2));
    int status = MG_ERR_NOT_CONVERGED, cycles = 0, stall = 0, nh = 0;
    double hist[MG_MAX_HIST];
    const double rel0 = nf > 0.0 ? std::sqrt(r2) / nf : 0.0;
    double best = rel0, rel = rel0;
    hist[nh++] = rel0;
    if (!std::isfinite(nf) || !std::isfinite(rel0)) status = MG_ERR_NONFINITE;
    else if (nf == 0.0 || rel0 <= tol) status = MG_OK;
    if (nf == 0.0)
        for (int r = 0; r < R; ++r) {
            SCK(cudaSetDevice(c->dev[r]));
            SCK(launch_zero(c->sl[r]->h64.fine, nullptr, c->st[r]));
        }
    while (status == MG_ERR_NOT_CONVERGED) {
        SCKS(vcycle(c));
        ++cycles;
        SCKS(norm2(c, 0, &r2));
        rel = std::sqrt(r2) / nf;
        if (nh < MG_MAX_HIST) hist[nh++] = rel;
        if (!std::isfinite(rel)) status = MG_ERR_NONFINITE;
        else if (rel <= tol) status = MG_OK;
        else if (rel > 1e3 * std::max(rel0, tol)) status = MG_ERR_DIVERGED;
        else {
            stall = rel > 0.9 * best ? stall + 1 : 0;
            best = std::min(best, rel);
            if (stall >= 5 || cycles >= c->opts.max_cycles) break;
        }
    }
    for (int r = 0; r < R; ++r) {
        Solver *s = c->sl[r];
        SCK(cudaSetDevice(c->dev[r]));
        SCK(launch_unpack(s->h64.fine, s->doff, phi[r], nullptr, c->st[r]));
        SCK(cudaStreamSynchronize(c->st[r]));
    }
    if (st) {
        memset(st, 0, sizeof *st);
        st->cycles = cycles;
        st->status = status;
        st->norm_f = nf;
        st->rel_resid0 = rel0;
        st->rel_resid = rel;
        for (int i = 0; i < nh; ++i) st->hist[i] = hist[i];
        st->t_solve_ms =
            std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0)
                .count();
    }
    if (status != MG_OK)
        set_error(status, "slab solve finished with status %d (%s)", status,
                  mg_error_string(status));
    return status;
}

void mg_slab_destroy(mg_slab *sb)
{
    if (!sb) return;
    destroy(sb->c);
    delete sb;
}

}  // extern "C"
