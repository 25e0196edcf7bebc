// solver.h -- host-side hierarchy and cycle driver shared by mg_ctx (one box)
// and mg_batch (many boxes).
#pragma once

#include <array>
#include <string>
#include <vector>

#include "kernels.h"
#include "level.h"
#include "mg.h"

namespace mg {

int set_error(int code, const char *fmt, ...);

// Arrays of one box at one level, in one precision.
template <class T>
struct LevelBufs {
    T *phi = nullptr, *phi2 = nullptr, *f = nullptr;
    T *wx = nullptr, *wy = nullptr, *wz = nullptr, *invD = nullptr;
    T *D = nullptr;  // FP64 levels only: sum of the six weights
};

// All levels of all boxes in one precision, plus the launch sets.
template <class T>
struct Hier {
    std::vector<std::vector<LevelBufs<T>>> lv;  // [box][level]
    std::vector<T *> ainv;                      // [box] dense coarsest-level inverse
    std::vector<BoxSet<T>> smooth;              // [level]: boxes not yet at their bottom
    std::vector<char> fused;                    // [level]: smooth with fused sweeps
    std::vector<const SweepMaps *> maps;        // [level]: TMA maps of the level's boxes (or null)
    std::vector<char> prol;                     // [level]: the maps hold the coarse phi (fused
                                                //   prolongation in the first post-smoothing sweep)
    BoxSet<T> fine{};                           // level 0 of every box
    BoxSet<T> bottom{};                         // coarsest level of every box
    std::vector<int> lc;                        // [box] first level run by the coarse kernel
    const CoarseJob<T> *jobs = nullptr;         // [box] device
    int njobs = 0;
    cudaGraphExec_t graph = nullptr;            // captured V-cycle (+ fine norm for FP64)
    cudaGraphExec_t head = nullptr;             // look-ahead: first red pass + norm
    cudaGraphExec_t down0 = nullptr;            // host-judged inner cycles: finest level's down leg
    cudaGraphExec_t rest = nullptr;             // ... and the rest of the cycle
    T *uinv = nullptr;                          // coupled level: dense inverse of the union bottom
    int pgrid = 0;                              // resident CTAs of the persistent level kernels
    T *cgp = nullptr, *cgq = nullptr;           // CG coarsest level: p and q (level arrays)
    int cggrid = 0;                             // CG coarsest level: CTAs of its launch
};

// A timed stretch of one stage class: events recorded before and after it.
struct ProfSlot {
    int kind;
    cudaEvent_t b, e;
    int launches;   // launches of the stage class the stretch holds
};

struct Solver {
    int dev = 0;
    int nbox = 0;
    bool shared = false;  // all boxes are one box's right-hand sides: one weight set
    mg_opts opts{};
    std::vector<std::array<int, 3>> n;              // [box] fine dims (nx, ny, nz)
    std::vector<double> dx;                          // [box]
    std::vector<std::vector<std::array<int, 3>>> dims;  // [box][level]
    std::vector<int> nlev;                           // [box]
    int maxlev = 0;
    int max_bottom = 0;                              // most cells on a coarsest level
    int sms = 0;                                     // multiprocessors of the device
    std::vector<long long> off;                      // [box+1] packed cell offsets
    long long total = 0;                             // packed cells

    char *arena = nullptr;                           // every level array, zero-filled
    char *desc = nullptr;                            // launch-set descriptors
    Hier<double> h64;
    Hier<float> h32;
    bool has32 = false;

    double *beta = nullptr;        // packed copy of cell beta
    double *work = nullptr;        // coarsest-level inverse scratch
    double *partials = nullptr;    // per-tile partial sums
    double *dnorm = nullptr;       // [nbox] last residual norm
    double *dnormf = nullptr;      // [nbox] ||f||
    double *dinv = nullptr;        // [nbox] scratch reciprocal
    double *se = nullptr, *sr = nullptr, *sr_inv = nullptr;  // mixed scales
    int *active = nullptr;         // [nbox] device flags
    int *active32 = nullptr;       // [nbox] device flags of a refinement step's inner FP32 cycles
    bool inner_adapt = false;      // mixed: inner cycles end per box on the inner residual
    bool inner_norm = false;       // enqueueing inner cycles: restriction with norm + exit test
    bool inner_while = false;      // enqueueing the device loop's body: inner cycles as a WHILE node
    int *icount = nullptr;         // [2] device: inner cycles run in this step, in this solve
    double *ipart = nullptr;       // device: per-warp sums of the finest FP32 restriction
    double *ichunk = nullptr;      // device: their sums over chunks of tiles of one box
    const int *icstart = nullptr;  // device [nbox + 1]: first chunk of each box of that set
    int inner_chunks = 0;
    long long inner_cycle_kernels = 0;  // launches of one inner cycle in the WHILE form
    const long long *doff = nullptr;  // [nbox + 1] device copy of off
    int *dside = nullptr;          // [nbox] device: 1 if the solution ended in phi2
    double *hnorm = nullptr;       // pinned [2 * nbox]
    int *hactive = nullptr;        // pinned [nbox]
    int *hflags = nullptr;         // pinned [nbox]: inner flags read by the host-judged loop
    int *hside = nullptr;          // pinned [nbox + 1]; the last is the error word's copy
    double *stage_a = nullptr, *stage_b = nullptr, *stage_c = nullptr;  // packed staging
    cudaStream_t cap = nullptr;    // capture stream
    cudaStream_t cap2 = nullptr;   // capture stream of a nested conditional body
    // host inputs of a solve are copied in on this stream, concurrently with
    // work already queued on the caller's stream (e.g. mg_set_beta's set-up)
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_in = nullptr;   // the copy-in is done
    // the set-up's coarsest inverses run on this stream, concurrently with the
    // diagonal and FP32 steps of the finer levels (fork / join events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // a one-box host beta is copied in by slabs of planes on the copy stream,
    // the face-weight step of each slab starting as soon as it has landed
    static constexpr int kBetaSlabs = 8;
    cudaEvent_t ev_slab[kBetaSlabs] = {};
    bool stage_clean = false;      // the staging buffers are idle (last staged call returned OK)
    cudaEvent_t ev_setup0 = nullptr, ev_setup1 = nullptr;
    bool beta_set = false;
    float t_setup_ms = 0.f;
    bool setup_pending = false;
    // mixed precision on independent boxes (mg_opts.fp32_setup = 0): the
    // levels below the finest are FP32 only, averaged from the finer FP32
    // weights (the finest level's are the rounded FP64 ones)
    bool coarse32 = false;

    // measurement (mg_profile_*)
    bool prof = false;                    // record stage events
    bool graph_prof = false;              // graphs were captured with events
    std::vector<ProfSlot> slots64, slots32;  // event slots inside the graphs
    std::vector<ProfSlot> direct;         // slots of direct launches since the last collect
    std::vector<const std::vector<ProfSlot> *> pending;  // graph slot lists to collect
    std::vector<cudaEvent_t> ev_free;     // reusable events
    std::vector<ProfSlot> *rec = nullptr; // where begin/end append (capture or direct)
    bool capturing = false;
    double prof_ms[MG_PROF_NKIND] = {};
    long long prof_n[MG_PROF_NKIND] = {};
    long long kernels = 0;                // kernels launched by this solver
    long long cap_kernels = 0;            // kernels enqueued into graph captures
    long long graph_kernels64 = 0, graph_kernels32 = 0, graph_kernels_head = 0;
    std::vector<ProfSlot> slots_head;     // event slots of the look-ahead head graph
    std::vector<ProfSlot> slots_down0, slots_rest;  // ... of the host-judged inner cycle parts
    long long graph_kernels_down0 = 0, graph_kernels_rest = 0;
    // FP64 look-ahead: each cycle starts with an out-of-place red pass that
    // also yields the previous iterate's residual norm, judged before the
    // rest of the cycle (no separate norm pass)
    bool lookahead = false;
    // coupled level (the boxes solved as one domain; mg_level)
    bool coupled = false;                            // one norm for all boxes (mg_level)
    int cut = 0;                                     // levels kept when the coarsest is solved
                                                     // elsewhere (slab-decomposed box), else 0
    bool xmode = false;                              // ghost exchanges: coupled level or periodic axes
    bool wide = false;                               // wide-guard layout (xmode)
    std::vector<std::vector<std::array<int, 3>>> lo;  // [box][level] lower corners (coupled)
    std::vector<const ExchRec *> xrec;               // [level] device exchange records
    std::vector<int> nxrec;                          // [level]
    std::vector<int> xmax;                           // [level] cells of the largest record
    UnionBottom ub{};                                // union of the coarsest levels

    // set-up launch sets
    std::vector<SetupSet> setup_lv;       // [level] every box that has the level
    std::vector<SetupSet> setup_coarsen;  // [level] boxes that have level + 1
    SetupSet setup_bottom{};              // coarsest level of every box
    int bottom_packed = 0;                // dynamic shared memory of k_setup_bottom (packed matrices)

    int *derr = nullptr;                  // device error word (bounded waits that gave up)
    unsigned *gbar = nullptr;             // device grid-barrier word of the persistent launches
    // one box whose coarsest level is too large for a dense inverse: solved
    // there by conjugate gradients (p, q in the hierarchies; partial sums)
    bool cg_bottom = false;
    double *cgpart = nullptr;
    int bc = 0;                           // wall mask: bit w set = wall w Neumann
    bool singular = false;                // every wall Neumann: A has the constants as null space
    double *dmean = nullptr;              // [nbox] scratch: removed means
    bool tma = false;                     // FP32 fused sweeps use the TMA kernel

    // conjugate gradients preconditioned by a symmetric V-cycle (krylov = 1):
    // level-0 FP64 x in phi2, r in f, z in phi; p and q per box
    bool pcg = false;
    double **pcg_p = nullptr, **pcg_q = nullptr;  // device [nbox] arrays of level-0 pointers
    PcgScalars sc{};
    cudaGraphExec_t loop_pcg = nullptr;
    long long loop_kernels_pcg = 0;

    // on-device convergence loop (conditional CUDA graph)
    char *jblock = nullptr;               // device: judge state block
    char *hjblock = nullptr;              // pinned host mirror
    size_t jbytes = 0;
    JudgeState J{};
    cudaGraphExec_t loop64 = nullptr, loop32 = nullptr;
    long long loop_kernels64 = 0, loop_kernels32 = 0;  // kernels per loop iteration
};

// shared_weights: the nbox boxes are right-hand sides of one box (same dims,
// dx and beta); weights, diagonals and the coarsest inverse exist once.
// lo (nullable): lower corners of the boxes of a coupled level (one domain;
// all dx equal, bc 0); NULL: independent boxes.
// cut > 0 (coupled levels only): keep levels 0 .. cut - 1; the last of them
// has no dense inverse of its own (its problem is solved by another context,
// as the coarse end of a slab-decomposed box).
int solver_create(Solver **out, int nbox, const int (*n)[3], const double *dx, int bc,
                  const mg_opts *opts, bool shared_weights = false,
                  const int (*lo)[3] = nullptr, int cut = 0);
// Set-up of a one-box FP64 context whose level-0 face weights were written
// into its arrays by the caller: coarse weights, diagonals and the dense
// coarsest inverse, on st.
int solver_setup_from_weights(Solver *s, cudaStream_t st);
// One FP64 V-cycle of every active box from its level-0 f and phi (phi is the
// initial guess), enqueued on st.
cudaError_t solver_enqueue_vcycle64(Solver *s, cudaStream_t st);
void solver_destroy(Solver *s);
int solver_set_beta(Solver *s, const double *beta_packed, cudaStream_t st);
// Solve every box; f/phi packed.  zero_guess ignores phi's input.
// side_copy: host inputs may be copied in on the solver's copy stream
// (false when the caller still has stage-buffer work queued on stream).
int solver_solve(Solver *s, const double *f, double *phi, double tol, mg_stats *st,
                 cudaStream_t stream, bool zero_guess, bool side_copy = true);
int solver_adjoint(Solver *s, int nrhs, const double *phi, const double *g, double *dLdf,
                   double *dLdbeta, double tol, mg_stats *st, cudaStream_t stream);

}  // namespace mg
