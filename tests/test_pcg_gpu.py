"""V-cycle-preconditioned conjugate gradients on the GPU (krylov = 1) against
the oracle.  Parity bar as for the V-cycle solves: relative L2 difference
<= 1e-9 from the oracle's converged solution, the oracle's own residual of
the GPU solution <= 1.01 x the tolerance; the iteration count matches the
oracle's preconditioned CG within one iteration or 5% (same preconditioner,
FP64 on both sides, different rounding order)."""
import numpy as np
import pytest
import torch

import oracle as O
from bounds import residual_slack
from paper_1008_2801_gb300 import BatchSolver, MGError, Solver, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _case(shape, seed, contrast=None):
    nz, ny, nx = shape
    if contrast is None:
        d = inputs.stellar((nx, ny, nz), seed)
    else:
        d = inputs.inclusions((nx, ny, nz), seed, contrast=contrast)
    return d["beta"], d["f"], d["dx"]


def _solve(beta, f, h, dev, bc=0, **kw):
    kw.setdefault("max_cycles", 400)
    with Solver(f.shape, h, device=dev, bc=bc, krylov=True, **kw) as s:
        s.set_beta(_t(beta, dev))
        phi, st = s.solve(_t(f, dev), tol=TOL)
        return phi.cpu().numpy(), st


def _check(beta, f, h, phi, st, bc=0):
    assert st["status"] == "ok", st
    ref, info = O.pcg_solve(beta, f, h, tol=1e-13, maxit=400, bc=bc)
    assert info["status"] == "ok"
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)
    r = O.residual(O.face_beta(beta, bc), h, f, phi)
    assert O.norm2(r) <= TOL * 1.01 * O.norm2(f)
    _, info = O.pcg_solve(beta, f, h, tol=TOL, maxit=400, bc=bc)
    # finite-precision CG at high contrast: the iteration count moves with
    # rounding (a few ulp in the weights shift it by one or two at ~100)
    assert abs(st["cycles"] - info["cycles"]) <= max(1, info["cycles"] // 20), \
        (st["cycles"], info["cycles"])


@pytest.mark.parametrize("contrast", [None, 1e2, 1e4, 1e6])
@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 40, 64)])
def test_matches_the_oracle(cuda_device, shape, contrast):
    beta, f, h = _case(shape, 30, contrast)
    phi, st = _solve(beta, f, h, cuda_device)
    _check(beta, f, h, phi, st)


@pytest.mark.parametrize("bc", [0b000011, 0b110100, 0b011111])
def test_neumann_walls(cuda_device, bc):
    beta, f, h = _case((16, 32, 24), 31, 1e3)
    phi, st = _solve(beta, f, h, cuda_device, bc=bc)
    _check(beta, f, h, phi, st, bc)


def test_residual_history_follows_the_oracle(cuda_device):
    beta, f, h = _case((32, 32, 32), 32, 1e4)
    phi, st = _solve(beta, f, h, cuda_device)
    _, info = O.pcg_solve(beta, f, h, tol=TOL, maxit=400)
    n = min(len(st["hist"]), len(info["hist"]), 20)
    np.testing.assert_allclose(st["hist"][:n], info["hist"][:n], rtol=1e-6)


def test_converges_where_vcycles_stall(cuda_device):
    beta, f, h = _case((64, 64, 64), 33, 1e4)
    phi, st = _solve(beta, f, h, cuda_device)
    assert st["status"] == "ok" and st["cycles"] < 150
    with Solver(f.shape, h, device=cuda_device, max_cycles=150) as s:
        s.set_beta(_t(beta, cuda_device))
        _, sv = s.solve(_t(f, cuda_device), tol=TOL)
    assert sv["status"] == "not_converged"        # stalled or out of cycles


def test_initial_guess_and_zero_rhs(cuda_device):
    beta, f, h = _case((16, 16, 16), 34, 1e2)
    with Solver(f.shape, h, device=cuda_device, krylov=True) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, st = s.solve(_t(f, cuda_device), tol=1e-13)
        again, st2 = s.solve(_t(f, cuda_device), phi.clone(), tol=1e-10)
        assert st2["cycles"] == 0 and torch.equal(again, phi)
        zero, st3 = s.solve(torch.zeros_like(phi), tol=1e-10)
        assert st3["status"] == "ok" and not zero.any()


def test_device_loop_matches_host_loop(cuda_device):
    beta, f, h = _case((32, 32, 32), 35, 1e4)
    res = []
    for use_graph in (True, False):
        phi, st = _solve(beta, f, h, cuda_device, use_graph=use_graph)
        res.append((phi, st["cycles"], list(st["hist"])))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1:] == res[1][1:]


def test_batched_uneven_boxes(cuda_device):
    shapes = [(16, 32, 24), (32, 32, 32), (8, 16, 64), (24, 24, 24)]
    cases = [_case(s, 40 + i, 1e4) for i, s in enumerate(shapes)]
    h = cases[0][2]
    with BatchSolver(shapes, h, device=cuda_device, krylov=True) as b:
        b.set_beta(b.pack([_t(c[0], cuda_device) for c in cases]))
        phi, st = b.solve(b.pack([_t(c[1], cuda_device) for c in cases]), tol=TOL)
        parts = [p.cpu().numpy() for p in b.unpack(phi)]
    for (beta, f, _), p, s in zip(cases, parts, st):
        _check(beta, f, h, p, s)


def test_several_right_hand_sides(cuda_device):
    beta, f, h = _case((16, 32, 32), 36, 1e3)
    rng = np.random.default_rng(37)
    fs = np.stack([f, rng.uniform(-1, 1, f.shape), rng.uniform(-1, 1, f.shape)])
    with Solver(f.shape, h, device=cuda_device, krylov=True) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, sts = s.solve(_t(fs, cuda_device), tol=TOL)
        phi = phi.cpu().numpy()
    for k in range(3):
        _check(beta, fs[k], h, phi[k], sts[k])


@pytest.mark.parametrize("contrast", [None, 1e4, 1e6])
def test_mixed_precision_preconditioner(cuda_device, contrast):
    # CG and its vectors in FP64, the symmetric V-cycle in FP32 on r / ||r||:
    # the same solution in at most half again as many iterations
    beta, f, h = _case((32, 32, 64), 50, contrast)
    phi, st = _solve(beta, f, h, cuda_device, precision="mixed")
    assert st["status"] == "ok", st
    ref, info = O.pcg_solve(beta, f, h, tol=1e-13, maxit=400)
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)
    faces = O.face_beta(beta)
    r = O.residual(faces, h, f, phi)
    # the solve stopped on its own FP64 residual of phi (<= tol); this
    # evaluation differs from it by rounding only, which a 1e6 contrast makes
    # a few per cent of tol
    assert O.norm2(r) <= TOL * O.norm2(f) + residual_slack(faces, h, f, phi)
    _, st64 = _solve(beta, f, h, cuda_device)
    # an FP32 cycle is symmetric and linear only to FP32 rounding, which CG
    # feels more as beta's contrast grows (1e6: about a third more iterations)
    assert st["cycles"] <= st64["cycles"] * 1.5 + 2, (st["cycles"], st64["cycles"])


def test_mixed_batched_boxes(cuda_device):
    shapes = [(16, 32, 24), (32, 32, 32), (8, 16, 64)]
    cases = [_case(s, 60 + i, 1e3) for i, s in enumerate(shapes)]
    h = cases[0][2]
    with BatchSolver(shapes, h, device=cuda_device, krylov=True, precision="mixed",
                     max_cycles=400) as b:
        b.set_beta(b.pack([_t(c[0], cuda_device) for c in cases]))
        phi, st = b.solve(b.pack([_t(c[1], cuda_device) for c in cases]), tol=TOL)
        parts = [p.cpu().numpy() for p in b.unpack(phi)]
    for (beta, f, _), p, s in zip(cases, parts, st):
        assert s["status"] == "ok", s
        ref, _ = O.pcg_solve(beta, f, h, tol=1e-13, maxit=400)
        assert np.linalg.norm(p - ref) <= 1e-9 * np.linalg.norm(ref)


def test_unsupported_uses(cuda_device):
    shape = (8, 8, 8)
    for kw in ({"bc": 63}, {"bc": 64}, {"nu1": 2, "nu2": 1}):
        with pytest.raises(MGError) as e:
            Solver(shape, 0.1, device=cuda_device, krylov=True, **kw)
        assert e.value.name == "unsupported", kw


def test_adjoint_with_krylov_matches_the_oracle(cuda_device):
    beta, f, h = _case((16, 16, 32), 38, 1e3)
    rng = np.random.default_rng(39)
    tgt = rng.uniform(-1, 1, f.shape)
    with Solver(f.shape, h, device=cuda_device, krylov=True) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, _ = s.solve(_t(f, cuda_device), tol=1e-12)
        lam, dbeta = s.adjoint(phi, phi - _t(tgt, cuda_device), tol=1e-12)
        phi, lam, dbeta = phi.cpu().numpy(), lam.cpu().numpy(), dbeta.cpu().numpy()
    lam_ref, db_ref, infos = O.adjoint(beta, h, phi, phi - tgt, tol=1e-13, max_cycles=400)
    assert np.linalg.norm(lam - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    assert np.linalg.norm(dbeta - db_ref) <= 1e-8 * np.linalg.norm(db_ref)
