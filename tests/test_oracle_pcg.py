"""CPU pins of the oracle's V-cycle-preconditioned conjugate gradients (a
variant the paper does not describe: CG on -A with the symmetric V-cycle as
preconditioner, for high-contrast beta).

Checked against: symmetry and definiteness of the preconditioner (and the
asymmetry of the cycle whose post-smoother is not the adjoint, so that the
symmetry test is sensitive to the colour order), a dense solve of a matrix
built here from cell adjacency (not from the oracle's faces), the
monotone decrease of the error's energy norm over the iterations (the
minimisation property of CG, which a wrong alpha, beta or sign breaks), one
iteration when the cycle is the exact inverse (a single-level box), and
convergence where the V-cycle iteration stalls."""
import numpy as np
import pytest

import oracle as O
from paper_1008_2801_gb300 import inputs


def _dense(beta, h, bc):
    """-A from cell adjacency: Dirichlet walls add 2 beta, Neumann walls
    nothing, inner faces the harmonic mean."""
    nz, ny, nx = beta.shape
    n = beta.size
    M = np.zeros((n, n))
    idx = np.arange(n).reshape(beta.shape)
    dims = (nx, ny, nz)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx[k, j, i]
                for d, step in ((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)):
                    p = [i, j, k]
                    p[d] += step
                    w = 2 * d + (step > 0)
                    if 0 <= p[d] < dims[d]:
                        a, b = beta[k, j, i], beta[p[2], p[1], p[0]]
                        hm = 2 * a * b / (a + b)
                        M[r, r] += hm
                        M[r, idx[p[2], p[1], p[0]]] -= hm
                    elif not (bc >> w) & 1:
                        M[r, r] += 2 * beta[k, j, i]
    return M / h ** 2


def _case(shape, seed, contrast=None):
    nz, ny, nx = shape
    if contrast is None:
        d = inputs.stellar((nx, ny, nz), seed)
    else:
        d = inputs.inclusions((nx, ny, nz), seed, contrast=contrast, count=4)
    return d["beta"], d["f"], d["dx"]


@pytest.mark.parametrize("bc", [0, 0b010110])
@pytest.mark.parametrize("contrast", [None, 1e4])
def test_symmetric_cycle_is_symmetric_and_negative_definite(bc, contrast):
    beta, _, h = _case((8, 16, 16), 1, contrast)
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal((2,) + beta.shape)
    Vu = O.vcycle_apply(beta, h, u, bc=bc)
    Vv = O.vcycle_apply(beta, h, v, bc=bc)
    a, b = np.vdot(u, Vv), np.vdot(Vu, v)
    assert abs(a - b) <= 1e-12 * np.sqrt(np.vdot(u, -Vu) * np.vdot(v, -Vv))
    for w in (u, v, rng.standard_normal(beta.shape)):
        assert np.vdot(w, O.vcycle_apply(beta, h, w, bc=bc)) < 0
    # linear in its right-hand side (zero start)
    np.testing.assert_allclose(O.vcycle_apply(beta, h, 2 * u - v, bc=bc), 2 * Vu - Vv,
                               atol=1e-12 * np.abs(Vu).max())


def test_the_solve_cycle_is_not_symmetric():
    # red-then-black post-smoothing is not the adjoint of the pre-smoother:
    # the symmetry check above would catch a colour-order mistake
    beta, _, h = _case((8, 16, 16), 3)
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal((2,) + beta.shape)
    a = np.vdot(u, O.vcycle_apply(beta, h, v, sym=False))
    b = np.vdot(O.vcycle_apply(beta, h, u, sym=False), v)
    assert abs(a - b) > 1e-6 * abs(a)


@pytest.mark.parametrize("bc", [0, 0b100011])
@pytest.mark.parametrize("contrast", [1e2, 1e6])
def test_pcg_matches_a_dense_solve(bc, contrast):
    beta, f, h = _case((8, 8, 8), 5, contrast)
    want = np.linalg.solve(-_dense(beta, h, bc), f.ravel()).reshape(f.shape)
    got, info = O.pcg_solve(beta, f, h, tol=1e-14, bc=bc)
    assert info["status"] == "ok"
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


def test_energy_norm_of_the_error_decreases_every_iteration():
    beta, f, h = _case((8, 8, 16), 6, 1e4)
    B = _dense(beta, h, 0)
    x = np.linalg.solve(B, -f.ravel())
    errs = []
    for k in range(1, 9):
        got, info = O.pcg_solve(beta, f, h, tol=1e-300, maxit=k)
        assert info["cycles"] == k
        e = got.ravel() - x
        errs.append(e @ B @ e)
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3 * errs[0]


def test_exact_preconditioner_converges_in_one_iteration():
    # odd dims: a single level, solved by the dense bottom solver, so the
    # "V-cycle" is -(-A)^{-1} itself
    beta, f, h = _case((7, 5, 3), 7, 1e3)
    assert O.levels(beta.shape[::-1]) == [(3, 5, 7)]
    got, info = O.pcg_solve(beta, f, h, tol=1e-12)
    assert info["status"] == "ok" and info["cycles"] == 1
    want = np.linalg.solve(-_dense(beta, h, 0), f.ravel()).reshape(f.shape)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_pcg_converges_where_vcycles_stall():
    beta, f, h = _case((32, 32, 32), 1, 1e4)
    phi, info = O.pcg_solve(beta, f, h, tol=1e-10, maxit=200)
    assert info["status"] == "ok" and info["cycles"] < 120
    _, vi = O.solve(beta, f, h, tol=1e-10, max_cycles=200)
    assert vi["status"] == "not_converged"
    r = O.residual(O.face_beta(beta), h, f, phi)
    assert O.norm2(r) <= 1.01e-10 * O.norm2(f)


def test_initial_guess_and_zero_rhs():
    beta, f, h = _case((8, 8, 8), 8, 1e2)
    ref, _ = O.pcg_solve(beta, f, h, tol=1e-14)
    again, info = O.pcg_solve(beta, f, h, tol=1e-10, phi0=ref)
    assert info["status"] == "ok" and info["cycles"] == 0
    np.testing.assert_array_equal(again, ref)
    zero, info = O.pcg_solve(beta, np.zeros_like(f), h, phi0=ref)
    assert info["status"] == "ok" and not zero.any()
    _, info = O.pcg_solve(beta, f, h, bc=63)
    assert info["status"] == "bad_hierarchy"          # every wall Neumann: not offered
