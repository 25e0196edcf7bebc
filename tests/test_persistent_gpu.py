"""Persistent level sweeps (mg_opts.persistent = 1) against the per-stage
launches and the oracle (GPU).

A level smoothed with single-colour passes runs as one launch going down
(pre-smoothing passes, residual, restriction) and one coming up
(prolongation, post-smoothing passes), with a bounded grid barrier between
stages.  Within one colour a Gauss-Seidel pass updates cells that do not
depend on each other, and every stage does the same arithmetic per cell as
its own kernel, so the solutions must be bitwise those of the per-stage
launches; they are also held to the oracle's solution.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import BatchSolver, LevelSolver, MGError, Solver, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _dev(a, dev):
    return torch.from_numpy(np.array(a, order="C", copy=True)).to(dev)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batched_persistent_is_bitwise_the_per_stage_solve(cuda_device, precision, use_graph):
    d = inputs.batched(12, 41, sizes=(8, 12, 16, 24, 32, 48), dx=1 / 48)
    shapes = [tuple(int(v) for v in dims[::-1]) for dims in d["dims"]]
    beta = _dev(np.concatenate([b.ravel() for b in d["beta"]]), cuda_device)
    f = _dev(np.concatenate([x.ravel() for x in d["f"]]), cuda_device)
    out = {}
    for persistent in (False, "small", True):
        bs = BatchSolver(shapes, d["dx"], precision=precision, device=cuda_device,
                         persistent=persistent, use_graph=use_graph, smoother="passes")
        bs.set_beta(beta)
        phi, sts = bs.solve(f, tol=TOL)
        assert all(s["status"] == "ok" for s in sts)
        out[persistent] = (phi.cpu(), [s["cycles"] for s in sts])
        bs.close()
    for mode in ("small", True):
        assert out[mode][1] == out[False][1]
        assert torch.equal(out[mode][0], out[False][0])
    flat = out[True][0].numpy()
    o = 0
    for b, sh in enumerate(shapes):
        n = sh[0] * sh[1] * sh[2]
        got = flat[o:o + n].reshape(sh)
        o += n
        ref, _ = O.solve(d["beta"][b], d["f"][b], d["dx"], tol=1e-13)
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision,smoother", [("fp64", "auto"), ("mixed", "passes"),
                                                ("mixed", "fused")])
def test_single_box_persistent_matches(cuda_device, precision, smoother):
    # the finest level too (FP64: after the look-ahead red pass the first
    # sweep's black pass runs out of place inside the persistent launch);
    # levels smoothed with fused FP32 sweeps keep their own launches
    d = inputs.stellar((64, 48, 40), 12)
    beta, f = _dev(d["beta"], cuda_device), _dev(d["f"], cuda_device)
    out = {}
    for persistent in (False, True):
        with Solver(f.shape, d["dx"], precision=precision, device=cuda_device,
                    persistent=persistent, smoother=smoother) as s:
            s.set_beta(beta)
            phi, st = s.solve(f, tol=TOL)
            assert st["status"] == "ok"
            out[persistent] = phi
    assert torch.equal(out[True], out[False])
    ref, _ = O.solve(d["beta"], d["f"], d["dx"], tol=1e-13)
    assert np.linalg.norm(out[True].cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)


def test_persistent_with_symmetric_cycles_and_odd_sweeps(cuda_device):
    d = inputs.stellar((32, 40, 24), 13)
    beta, f = _dev(d["beta"], cuda_device), _dev(d["f"], cuda_device)
    for kw in ({"krylov": True}, {"nu1": 3, "nu2": 1}, {"nu1": 0, "nu2": 2},
               {"full_residual": True}):
        out = {}
        for persistent in (False, True):
            with Solver(f.shape, d["dx"], device=cuda_device, persistent=persistent,
                        **kw) as s:
                s.set_beta(beta)
                phi, st = s.solve(f, tol=TOL)
                assert st["status"] == "ok", (kw, st)
                out[persistent] = phi
        assert torch.equal(out[True], out[False]), kw


def test_coupled_level_persistent(cuda_device):
    # exchanges run as stages of the persistent launch
    d = inputs.stellar(32, 14)
    m = 16
    los = [(i * m, j * m, k * m) for k in range(2) for j in range(2) for i in range(2)]
    sl = [(slice(k, k + m), slice(j, j + m), slice(i, i + m)) for (i, j, k) in los]
    bp = _dev(np.concatenate([d["beta"][q].ravel() for q in sl]), cuda_device)
    fp = _dev(np.concatenate([d["f"][q].ravel() for q in sl]), cuda_device)
    out = {}
    for persistent in (False, True):
        lv = LevelSolver(los, [(m, m, m)] * len(los), d["dx"], device=cuda_device,
                         persistent=persistent)
        lv.set_beta(bp)
        phi, st = lv.solve(fp, tol=TOL)
        assert st["status"] == "ok"
        out[persistent] = phi
        lv.close()
    assert torch.equal(out[True], out[False])
    ref, _ = O.solve(d["beta"], d["f"], d["dx"], tol=1e-13)
    got = np.zeros_like(ref)
    parts = out[True].cpu().numpy()
    o = 0
    for q in sl:
        got[q] = parts[o:o + m ** 3].reshape(m, m, m)
        o += m ** 3
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_persistent_profile_counts_one_launch_per_level_and_direction(cuda_device):
    d = inputs.stellar((64, 64, 64), 15)
    beta, f = _dev(d["beta"], cuda_device), _dev(d["f"], cuda_device)
    with Solver(f.shape, d["dx"], device=cuda_device, persistent=True, coarse_cells=-1) as s:
        s.set_beta(beta)
        s.profile(True)
        _, st = s.solve(f, tol=TOL)
        prof = s.read_profile(reset=True)
        cycles = st["cycles"]
        nlev = len(s.levels())
    # finest level: a down and an up launch per cycle, and outside them
    # only the look-ahead red pass that starts each cycle (and judges the
    # last one)
    assert prof["level"]["launches"] == 2 * cycles
    assert prof["pass"]["launches"] == cycles + 1
    for k in ("sweep", "restrict", "prolong"):
        assert prof[k]["launches"] == 0, k
    # every level above the coarsest: 2 launches; the coarsest one solve
    with Solver(f.shape, d["dx"], device=cuda_device, persistent=True, coarse_cells=-1,
                use_graph=False) as s:
        s.set_beta(beta)
        s.read_profile(reset=True)
        _, st = s.solve(f, tol=TOL)
        k_total = s.read_profile(reset=True)["kernels"]
    with Solver(f.shape, d["dx"], device=cuda_device, persistent=False, coarse_cells=-1,
                use_graph=False) as s:
        s.set_beta(beta)
        s.read_profile(reset=True)
        _, st2 = s.solve(f, tol=TOL)
        k_stage = s.read_profile(reset=True)["kernels"]
    assert st["cycles"] == st2["cycles"]
    # per cycle and level: 2 launches instead of 2 nu1 + 1 + 1 + 2 nu2 = 10
    # (one fewer on the finest level of an FP64 cycle: the look-ahead red
    # pass stays outside)
    assert k_stage - k_total == st["cycles"] * (nlev - 1) * 8 - st["cycles"]


def test_persistent_barrier_that_gives_up_returns_timeout(cuda_device):
    d = inputs.batched(6, 42, sizes=(16, 24, 32), dx=1 / 32)
    shapes = [tuple(int(v) for v in dims[::-1]) for dims in d["dims"]]
    beta = _dev(np.concatenate([b.ravel() for b in d["beta"]]), cuda_device)
    f = _dev(np.concatenate([x.ravel() for x in d["f"]]), cuda_device)
    bs = BatchSolver(shapes, d["dx"], device=cuda_device, persistent=True, wait_limit=-1,
                     max_cycles=3)
    bs.set_beta(beta)
    with pytest.raises(MGError) as ei:
        bs.solve(f, tol=TOL)
    assert ei.value.name == "timeout"
    bs.close()
    torch.cuda.synchronize(cuda_device)   # the context is intact
    bs = BatchSolver(shapes, d["dx"], device=cuda_device, persistent=True)
    bs.set_beta(beta)
    _, sts = bs.solve(f, tol=TOL)
    assert all(s["status"] == "ok" for s in sts)
    bs.close()
