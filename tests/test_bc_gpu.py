"""Wall conditions on the GPU against the CPU oracle: Dirichlet / Neumann
masks, lifted wall values and the singular all-Neumann solve (GPU).

Tolerances: face weights and the beta gradient to 1e-13 relative (same
arithmetic up to rounding order; a Neumann wall face is exactly 0); the lift
to 1e-14 relative; whole solves to 1e-9 relative L2 against the oracle at a
1e-13 relative residual, as for the Dirichlet solves.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import BatchSolver, MGError, Solver, inputs, wall_shapes
from paper_1008_2801_gb300 import ops as K

pytestmark = pytest.mark.gpu

TOL = 1e-10
MASKS = [1, 0b010110, 0b100100, 63]


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _case(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    return d["beta"], d["f"], d["dx"]


def _walls(shape, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1, 1, s) for s in wall_shapes(shape)]


@pytest.mark.parametrize("bc", [0, 1, 2, 4, 8, 16, 32, 63, 0b101010])
def test_face_weights_follow_the_mask(cuda_device, bc):
    shape = (9, 6, 13)
    beta, _, h = _case(shape, 40)
    w = K.face_weights(_t(beta, cuda_device), h, bc=bc)
    for wt, fo, kind in zip(w, O.face_beta(beta, bc), "xyz"):
        got = K.get(wt, shape, kind).cpu().numpy()
        want = fo / h ** 2
        zero = want == 0.0
        assert np.array_equal(got[zero], want[zero])
        assert np.max(np.abs(got[~zero] - want[~zero]) / want[~zero]) <= 1e-15


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 4, 5), (4, 16, 16)])
def test_singular_coarsest_inverse(cuda_device, shape):
    beta, f, h = _case(shape, 41)
    w = K.face_weights(_t(beta, cuda_device), h, bc=63)
    ainv = K.bottom_inverse(w, shape, singular=True).cpu().numpy()
    A = O.dense_matrix(O.face_beta(beta, 63), h, shape)
    r = np.random.default_rng(42).uniform(-1, 1, A.shape[0]) + 0.5   # any mean
    x = ainv @ r
    np.testing.assert_allclose(A @ x, r - r.mean(), atol=1e-10 * np.abs(r).max())
    r0 = r - r.mean()                                  # zero mean: the zero-mean solution
    x0 = ainv @ r0
    assert abs(x0.mean()) <= 1e-12 * np.abs(x0).max()
    want = np.linalg.lstsq(A, r0, rcond=None)[0]
    np.testing.assert_allclose(x0, want, atol=1e-10 * np.abs(want).max())


@pytest.mark.parametrize("bc", [0, 0b100110, 63])
def test_beta_gradient_with_neumann_walls(cuda_device, bc):
    shape = (5, 7, 9)
    beta, _, h = _case(shape, 43)
    rng = np.random.default_rng(44)
    phi, lam = rng.uniform(-1, 1, shape), rng.uniform(-1, 1, shape)
    got = K.beta_grad(_t(beta, cuda_device), _t(phi, cuda_device), _t(lam, cuda_device), h,
                      bc=bc).cpu().numpy()
    want = O.beta_grad(beta, h, phi, lam, bc=bc)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("bc", [0, 0b010110, 63])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 4), (7, 9, 13), (20, 12, 40)])
def test_lift_of_wall_values(cuda_device, bc, shape):
    beta, f, h = _case(shape, 45)
    vals = O.wall_values(_walls(shape, 46))
    with Solver(shape, h, device=cuda_device, bc=bc) as s:
        s.set_beta(_t(beta, cuda_device))
        got = s.bc_lift(_t(vals, cuda_device), _t(f, cuda_device)).cpu().numpy()
        # in place gives the same
        ft = _t(f, cuda_device)
        s.bc_lift(_t(vals, cuda_device), ft, out=ft)
        assert np.array_equal(ft.cpu().numpy(), got)
    want = O.bc_lift(beta, h, f, vals, bc)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-14 * scale


def _solve(beta, f, h, dev, bc, precision="fp64", tol=TOL, **kw):
    with Solver(f.shape, h, precision=precision, device=dev, bc=bc, **kw) as s:
        s.set_beta(_t(beta, dev))
        phi, st = s.solve(_t(f, dev), tol=tol)
        return phi.cpu().numpy(), st


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bc", MASKS)
@pytest.mark.parametrize("shape", [(24, 16, 20), (40, 24, 56), (64, 64, 64)])
def test_solve_matches_the_oracle(cuda_device, shape, bc, precision):
    beta, f, h = _case(shape, 47)
    f = f + 0.3                                       # a mean, removed when bc = 63
    phi, st = _solve(beta, f, h, cuda_device, bc, precision)
    assert st["status"] == "ok", st
    ref, info = O.solve(beta, f, h, tol=1e-13, bc=bc)
    assert info["status"] == "ok"
    # every wall Neumann in mixed precision: each refinement step's residual
    # goes to the FP32 cycles rounded to FP32, which leaves an error in the
    # smoothest non-constant modes that the residual barely sees (A scales
    # them by its smallest nonzero eigenvalue); at 64^3 the error comes out up
    # to about 30 times the relative residual (FP64 V-cycles: about 6)
    bar = 3e-9 if (precision == "mixed" and bc == 63) else 1e-9
    assert np.linalg.norm(phi - ref) <= bar * np.linalg.norm(ref)
    fr = f - f.mean() if bc == 63 else f
    r = O.residual(O.face_beta(beta, bc), h, fr, phi)
    assert O.norm2(r) <= TOL * 1.01 * O.norm2(fr)
    if bc == 63:
        assert abs(phi.mean()) <= 1e-13 * np.abs(phi).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_inhomogeneous_walls_manufactured(cuda_device, precision):
    # phi = cos(1.3x + 0.2) sin(2y + 0.5) cos z + x y with its wall values and
    # fluxes: the GPU solve of the lifted problem equals the oracle's, and
    # both carry the same discretisation error.
    n, bc = 32, 0b010110
    shape = (n, n, n)
    h = 1.0 / n
    zc, yc, xc = np.meshgrid(*(((np.arange(n) + 0.5) * h),) * 3, indexing="ij")
    b = lambda x, y, z: 1 + np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z) / 2
    p = lambda x, y, z: np.cos(1.3 * x + 0.2) * np.sin(2 * y + 0.5) * np.cos(z) + x * y
    grads = (lambda x, y, z: -1.3 * np.sin(1.3 * x + 0.2) * np.sin(2 * y + 0.5) * np.cos(z) + y,
             lambda x, y, z: 2 * np.cos(1.3 * x + 0.2) * np.cos(2 * y + 0.5) * np.cos(z) + x,
             lambda x, y, z: -np.cos(1.3 * x + 0.2) * np.sin(2 * y + 0.5) * np.sin(z))
    # f = div(beta grad phi) by a fine central difference of the exact flux
    e = 1e-5
    f = np.zeros(shape)
    for a, g in enumerate(grads):
        d = [0.0, 0.0, 0.0]
        d[a] = e
        up = b(xc + d[0], yc + d[1], zc + d[2]) * g(xc + d[0], yc + d[1], zc + d[2])
        dn = b(xc - d[0], yc - d[1], zc - d[2]) * g(xc - d[0], yc - d[1], zc - d[2])
        f += (up - dn) / (2 * e)
    beta = b(xc, yc, zc)
    walls = []
    L = n * h
    cc = (np.arange(n) + 0.5) * h
    for w in range(6):
        hi = w & 1
        if w < 2:
            Z, Y = np.meshgrid(cc, cc, indexing="ij")
            X = np.full_like(Z, L if hi else 0.0)
        elif w < 4:
            Z, X = np.meshgrid(cc, cc, indexing="ij")
            Y = np.full_like(Z, L if hi else 0.0)
        else:
            Y, X = np.meshgrid(cc, cc, indexing="ij")
            Z = np.full_like(Y, L if hi else 0.0)
        if (bc >> w) & 1:
            walls.append((1 if hi else -1) * b(X, Y, Z) * grads[w // 2](X, Y, Z))
        else:
            walls.append(p(X, Y, Z))
    vals = O.wall_values(walls)
    with Solver(shape, h, precision=precision, device=cuda_device, bc=bc) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, st = s.solve(_t(f, cuda_device), tol=TOL, bc_values=_t(vals, cuda_device))
        phi = phi.cpu().numpy()
    assert st["status"] == "ok"
    ref, _ = O.solve(beta, O.bc_lift(beta, h, f, vals, bc), h, tol=1e-13, bc=bc)
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)
    exact = p(xc, yc, zc)
    assert np.abs(phi - exact).max() < 2e-3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bc", [0b000011, 63])
def test_batched_boxes_with_walls(cuda_device, precision, bc):
    shapes = [(16, 24, 32), (32, 16, 16), (8, 8, 24)]
    h = 1.0 / 32
    cases = [_case(s, 50 + i) for i, s in enumerate(shapes)]
    bs = BatchSolver(shapes, h, precision=precision, device=cuda_device, bc=bc)
    try:
        bs.set_beta(_t(np.concatenate([c[0].ravel() for c in cases]), cuda_device))
        fs = [c[1] + 0.2 for c in cases]
        phi, st = bs.solve(_t(np.concatenate([f.ravel() for f in fs]), cuda_device), tol=TOL)
        outs = bs.unpack(phi.cpu())
    finally:
        bs.close()
    for (beta, _, _), f, got, s in zip(cases, fs, outs, st):
        assert s["status"] == "ok"
        ref, _ = O.solve(beta, f, h, tol=1e-13, bc=bc)
        assert np.linalg.norm(got.numpy() - ref) <= 1e-9 * np.linalg.norm(ref)


def test_multi_rhs_keeps_the_walls(cuda_device):
    shape, bc = (16, 24, 32), 0b110001
    beta, f, h = _case(shape, 55)
    fs = np.stack([f, np.random.default_rng(56).uniform(-1, 1, shape)])
    with Solver(shape, h, device=cuda_device, bc=bc) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, st = s.solve(_t(fs, cuda_device), tol=TOL)
        phi = phi.cpu().numpy()
    for r in range(2):
        ref, _ = O.solve(beta, fs[r], h, tol=1e-13, bc=bc)
        assert np.linalg.norm(phi[r] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_adjoint_with_neumann_walls(cuda_device):
    shape, bc = (16, 16, 24), 0b100110
    beta, f, h = _case(shape, 57)
    t = np.random.default_rng(58).uniform(-1, 1, shape)
    with Solver(shape, h, device=cuda_device, bc=bc) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, _ = s.solve(_t(f, cuda_device), tol=1e-12)
        lam, dbeta = s.adjoint(phi, phi - _t(t, cuda_device), tol=1e-12)
        phi, lam, dbeta = (a.cpu().numpy() for a in (phi, lam, dbeta))
    lam_o, db_o, _ = O.adjoint(beta, h, phi, phi - t, bc=bc)
    assert np.linalg.norm(lam - lam_o) <= 1e-9 * np.linalg.norm(lam_o)
    assert np.linalg.norm(dbeta - db_o) <= 1e-8 * np.linalg.norm(db_o)


def test_adjoint_of_the_singular_solve_is_unsupported(cuda_device):
    shape = (8, 8, 8)
    beta, f, h = _case(shape, 59)
    with Solver(shape, h, device=cuda_device, bc=63) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, _ = s.solve(_t(f, cuda_device))
        with pytest.raises(MGError) as e:
            s.adjoint(phi, phi)
        assert e.value.name == "unsupported"


@pytest.mark.parametrize("bc", [0b001001, 63])
def test_projection_with_neumann_walls(cuda_device, bc):
    shape = (12, 10, 14)
    nz, ny, nx = shape
    beta, _, h = _case(shape, 60)
    rng = np.random.default_rng(61)
    u = rng.uniform(-1, 1, (nz, ny, nx + 1))
    v = rng.uniform(-1, 1, (nz, ny + 1, nx))
    w = rng.uniform(-1, 1, (nz + 1, ny, nx))
    phi = rng.uniform(-1, 1, shape)
    with Solver(shape, h, device=cuda_device, bc=bc) as s:
        s.set_beta(_t(beta, cuda_device))
        ut, vt, wt = (_t(a, cuda_device) for a in (u, v, w))
        s.project_correct(_t(phi, cuda_device), ut, vt, wt)
        got = [a.cpu().numpy() for a in (ut, vt, wt)]
    want = O.correct(beta, h, phi, u, v, w, bc=bc)
    for g, wn in zip(got, want):
        assert np.max(np.abs(g - wn)) <= 1e-13 * np.max(np.abs(wn))
