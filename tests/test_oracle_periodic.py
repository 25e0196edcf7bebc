"""CPU pins of the oracle's periodic axes (wall-mask bits 6, 7, 8 = x, y, z).

Checked against: Fourier modes (exact eigenvectors of the periodic discrete
operator for constant beta) combined with the sine modes of Dirichlet walls,
invariance under cyclic shifts of beta and f, and a dense operator built
here from cell adjacency with wrap-around (not from the oracle's faces).
"""
import numpy as np
import pytest

import oracle as O
from paper_1008_2801_gb300 import inputs

PX, PY, PZ = 64, 128, 256


def _dense(beta, h, bc):
    """-A from cell adjacency: periodic axes wrap, Dirichlet walls add 2 beta,
    Neumann walls nothing."""
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
                    if 0 <= p[d] < dims[d] or (bc >> (6 + d)) & 1:
                        p[d] %= dims[d]
                        a, b = beta[k, j, i], beta[p[2], p[1], p[0]]
                        hm = 2 * a * b / (a + b)
                        M[r, r] += hm
                        M[r, idx[p[2], p[1], p[0]]] -= hm
                    elif not (bc >> w) & 1:
                        M[r, r] += 2 * beta[k, j, i]
    return M / h ** 2


def _grid(shape, h):
    nz, ny, nx = shape
    return np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")


def test_fourier_and_sine_modes_are_exact():
    # periodic x with two Dirichlet axes, constant beta: cos(2 pi m i / nx)
    # times the lowest sine modes in y and z
    shape = (12, 10, 16)
    nz, ny, nx = shape
    h = 1.0 / 16
    b = 1.7
    K, J, I = _grid(shape, h)
    phi = np.cos(2 * np.pi * 3 * I / nx + 0.4) * np.sin(np.pi * (J + 0.5) / ny) * \
        np.sin(np.pi * (K + 0.5) / nz)
    lam = -4 * b / h ** 2 * (np.sin(np.pi * 3 / nx) ** 2 + np.sin(np.pi / (2 * ny)) ** 2 +
                             np.sin(np.pi / (2 * nz)) ** 2)
    beta = np.full(shape, b)
    np.testing.assert_allclose(O.apply_periodic(O.face_beta_periodic(beta, PX), h, phi, PX),
                               lam * phi, atol=1e-9 * abs(lam))
    got, info = O.periodic_solve(beta, lam * phi, h, PX, tol=1e-14)
    assert info["status"] == "ok"
    np.testing.assert_allclose(got, phi, atol=1e-11)


def test_triply_periodic_mode_and_zero_mean():
    shape = (8, 12, 10)
    nz, ny, nx = shape
    h = 0.1
    b = 2.3
    K, J, I = _grid(shape, h)
    m = (2, 3, 1)
    phi = np.cos(2 * np.pi * (m[0] * I / nx + m[1] * J / ny + m[2] * K / nz) + 0.9)
    lam = -4 * b / h ** 2 * (np.sin(np.pi * m[0] / nx) ** 2 + np.sin(np.pi * m[1] / ny) ** 2 +
                             np.sin(np.pi * m[2] / nz) ** 2)
    bc = PX | PY | PZ
    f = lam * phi + 0.5                       # a constant part, not in the range of A
    got, info = O.periodic_solve(np.full(shape, b), f, h, bc, tol=1e-14)
    assert info["status"] == "ok"
    np.testing.assert_allclose(got, phi - phi.mean(), atol=1e-11)
    assert abs(got.mean()) < 1e-14


@pytest.mark.parametrize("bc", [PX, PY | PZ, PX | PY | PZ, PX | 0b110000, PZ | 0b000011])
def test_cyclic_shifts_commute_with_the_solve(bc):
    shape = (8, 10, 12)
    d = inputs.stellar(shape[::-1], 21)
    beta, f, h = d["beta"], d["f"], d["dx"]
    shift = tuple(s if (bc >> (6 + (2 - a))) & 1 else 0 for a, s in enumerate((3, 4, 5)))
    phi, info = O.periodic_solve(beta, f, h, bc, tol=1e-13)
    assert info["status"] == "ok"
    phs, _ = O.periodic_solve(np.roll(beta, shift, (0, 1, 2)), np.roll(f, shift, (0, 1, 2)), h,
                              bc, tol=1e-13)
    np.testing.assert_allclose(phs, np.roll(phi, shift, (0, 1, 2)), atol=1e-10 * np.abs(phi).max())


@pytest.mark.parametrize("bc", [PX, PX | PY, PX | PY | PZ, PY | 0b110011])
def test_periodic_operator_matches_a_dense_adjacency_matrix(bc):
    shape = (4, 3, 5)
    d = inputs.stellar(shape[::-1], 22)
    beta, f, h = d["beta"], d["f"], d["dx"]
    M = _dense(beta, h, bc)
    # A phi from the oracle, column by column
    cols = []
    for c in range(beta.size):
        e = np.zeros(beta.size)
        e[c] = 1
        cols.append(O.apply_periodic(O.face_beta_periodic(beta, bc), h, e.reshape(shape), bc).ravel())
    A = np.array(cols).T
    np.testing.assert_allclose(-A, M, atol=1e-10 * np.abs(M).max())
    np.testing.assert_allclose(M, M.T, atol=1e-10 * np.abs(M).max())
    singular = all(((bc >> (6 + a)) & 1) or ((bc >> (2 * a)) & 3) == 3 for a in range(3))
    ev = np.linalg.eigvalsh(M)
    if singular:
        assert abs(ev[0]) < 1e-8 * ev[-1] and ev[1] > 1e-6 * ev[-1]
        want = np.linalg.lstsq(-M, (f - f.mean()).ravel(), rcond=None)[0]
    else:
        assert ev[0] > 0
        want = np.linalg.solve(-M, f.ravel())
    got, info = O.periodic_solve(beta, f, h, bc, tol=1e-14)
    assert info["status"] == "ok"
    np.testing.assert_allclose(got.ravel(), want, atol=1e-10 * np.abs(want).max())
