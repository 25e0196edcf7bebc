"""CPU pins of the oracle's wall conditions (Dirichlet / Neumann mask, lifted
wall values, the singular all-Neumann solve).

The paper only names the equation the solve enforces (Sec. 1); the wall
conditions are the standard cell-centred ones: a Dirichlet wall holds phi at
the wall h/2 from the cell centre, a Neumann wall prescribes the outward flux
beta dphi/dn.  Each test below checks the oracle against something other than
itself: the textbook ghost-cell form of the same stencil, a pseudo-inverse of
the dense matrix, fields the scheme differentiates exactly, second-order
convergence to a manufactured solution, and finite differences.
"""
import numpy as np
import pytest

import oracle as O

sympy = pytest.importorskip("sympy")

WALLS = ("x-", "x+", "y-", "y+", "z-", "z+")


def centres(shape, h):
    nz, ny, nx = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h,
                          (np.arange(nx) + 0.5) * h, indexing="ij")
    return x, y, z


def wall_points(shape, h):
    """Face-centre coordinates of the six walls, as (x, y, z) arrays shaped
    like the packed wall arrays."""
    nz, ny, nx = shape
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    cx, cy, cz = ((np.arange(n) + 0.5) * h for n in (nx, ny, nz))
    pts = []
    for w in range(6):
        hi = w & 1
        if w < 2:
            z, y = np.meshgrid(cz, cy, indexing="ij")
            x = np.full_like(z, Lx if hi else 0.0)
        elif w < 4:
            z, x = np.meshgrid(cz, cx, indexing="ij")
            y = np.full_like(z, Ly if hi else 0.0)
        else:
            y, x = np.meshgrid(cy, cx, indexing="ij")
            z = np.full_like(y, Lz if hi else 0.0)
        pts.append((x, y, z))
    return pts


def ghost_apply(beta, h, phi, vals, bc):
    """A phi with the wall values in ghost cells (the ghost-cell method):
    the box is padded by one cell; a Dirichlet ghost holds 2 g - phi_c (so
    the wall midpoint holds g), a Neumann ghost phi_c + q h / beta_c (so the
    wall flux is q); ghost beta = the adjacent cell's beta; every face uses
    the harmonic mean; the 7-point flux sum is taken on the interior."""
    nz, ny, nx = beta.shape
    shapes = O.wall_shapes(beta.shape)
    split = np.split(np.asarray(vals), np.cumsum([a * b for a, b in shapes])[:-1])
    walls = [s.reshape(sh) for s, sh in zip(split, shapes)]
    P = np.zeros((nz + 2, ny + 2, nx + 2))
    B = np.ones((nz + 2, ny + 2, nx + 2))
    P[1:-1, 1:-1, 1:-1] = phi
    B[1:-1, 1:-1, 1:-1] = beta
    sl = {0: (slice(1, -1), slice(1, -1), 0), 1: (slice(1, -1), slice(1, -1), -1),
          2: (slice(1, -1), 0, slice(1, -1)), 3: (slice(1, -1), -1, slice(1, -1)),
          4: (0, slice(1, -1), slice(1, -1)), 5: (-1, slice(1, -1), slice(1, -1))}
    inner = {0: (slice(None), slice(None), 0), 1: (slice(None), slice(None), -1),
             2: (slice(None), 0, slice(None)), 3: (slice(None), -1, slice(None)),
             4: (0, slice(None), slice(None)), 5: (-1, slice(None), slice(None))}
    for w in range(6):
        pc, bcell = phi[inner[w]], beta[inner[w]]
        if (bc >> w) & 1:
            P[sl[w]] = pc + walls[w] * h / bcell
        else:
            P[sl[w]] = 2.0 * walls[w] - pc
        B[sl[w]] = bcell
    c = P[1:-1, 1:-1, 1:-1]
    bcen = B[1:-1, 1:-1, 1:-1]
    out = np.zeros_like(phi)
    for ax in range(3):
        for d in (-1, 1):
            idx = [slice(1, -1)] * 3
            idx[2 - ax] = slice(1 + d, P.shape[2 - ax] - 1 + d)
            pn, bn = P[tuple(idx)], B[tuple(idx)]
            out += 2.0 * bcen * bn / (bcen + bn) * (pn - c)
    return out / h**2


@pytest.mark.parametrize("bc", [0, 1, 2, 4, 8, 16, 32, 21, 42, 36, 63])
def test_lift_and_faces_match_the_ghost_cell_form(bc):
    rng = np.random.default_rng(100 + bc)
    shape = (5, 4, 6)
    h = 0.37
    beta = rng.uniform(0.5, 3.0, shape)
    phi = rng.standard_normal(shape)
    vals = rng.standard_normal(sum(a * b for a, b in O.wall_shapes(shape)))
    want = ghost_apply(beta, h, phi, vals, bc)
    f = rng.standard_normal(shape)
    lift = f - O.bc_lift(beta, h, f, vals, bc)          # the wall terms of A phi
    got = O.apply(O.face_beta(beta, bc), h, phi) + lift
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_wall_faces_follow_the_mask():
    rng = np.random.default_rng(7)
    beta = rng.uniform(1, 2, (3, 4, 5))
    for bc in range(64):
        bx, by, bz = O.face_beta(beta, bc)
        ends = [bx[:, :, 0], bx[:, :, -1], by[:, 0, :], by[:, -1, :], bz[0], bz[-1]]
        cells = [beta[:, :, 0], beta[:, :, -1], beta[:, 0, :], beta[:, -1, :], beta[0], beta[-1]]
        for w in range(6):
            want = 0.0 * cells[w] if (bc >> w) & 1 else 2.0 * cells[w]
            assert np.array_equal(ends[w], want), (bc, WALLS[w])


def test_all_neumann_operator_is_singular_on_constants_only():
    rng = np.random.default_rng(8)
    shape = (4, 3, 5)
    beta = rng.uniform(0.5, 2.0, shape)
    h = 0.25
    A = O.dense_matrix(O.face_beta(beta, 63), h, shape)
    np.testing.assert_allclose(A, A.T, atol=1e-12)
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-12 / h**2
    ev = np.linalg.eigvalsh(A)
    assert ev.max() < 1e-10 and abs(ev[-1]) < 1e-10 and ev[-2] < -1e-3
    for bc in (0, 31, 62, 21):
        Ab = O.dense_matrix(O.face_beta(beta, bc), h, shape)
        assert np.linalg.eigvalsh(Ab).max() < -1e-6
        assert np.abs(Ab @ np.ones(Ab.shape[0])).max() > 1e-3


@pytest.mark.parametrize("shape", [(8, 6, 4), (9, 13, 11)])
def test_singular_solve_is_the_pseudoinverse_solution(shape):
    # (8, 6, 4) coarsens once to a dense bottom; (9, 13, 11) is one level of
    # 1287 cells, solved by the conjugate-gradient bottom.
    rng = np.random.default_rng(sum(shape))
    h = 1.0 / 16
    beta = rng.uniform(0.5, 4.0, shape)
    f = rng.standard_normal(shape)                          # not mean-free
    phi, info = O.solve(beta, f, h, tol=1e-12, bc=63)
    assert info["status"] == "ok"
    A = O.dense_matrix(O.face_beta(beta, 63), h, shape)
    want = np.linalg.lstsq(A, (f - f.mean()).ravel(), rcond=None)[0]
    assert abs(want.mean()) < 1e-10 * np.abs(want).max()
    assert abs(phi.mean()) < 1e-13 * np.abs(phi).max()
    np.testing.assert_allclose(phi.ravel(), want, atol=1e-9 * np.abs(want).max())


def _packed(shape, h, fn):
    return O.wall_values([fn(w, *p) for w, p in enumerate(wall_points(shape, h))])


def test_quadratic_field_is_exact_with_neumann_walls():
    # Second differences and face-centred first differences of a quadratic
    # are exact, so with constant beta and exact wall fluxes the discrete
    # solution equals the field (minus its mean: all walls Neumann).
    shape = (12, 8, 16)
    h = 1.0 / 16
    b = 2.5
    x, y, z = centres(shape, h)
    phi_e = x**2 + 2 * y**2 - z**2 + 0.3 * x * y
    f = np.full(shape, b * (2 + 4 - 2))
    grad = (lambda x, y, z: 2 * x + 0.3 * y, lambda x, y, z: 4 * y + 0.3 * x,
            lambda x, y, z: -2 * z)
    q = _packed(shape, h, lambda w, x, y, z: (1 if w & 1 else -1) * b * grad[w // 2](x, y, z))
    beta = np.full(shape, b)
    fl = O.bc_lift(beta, h, f, q, 63)
    assert abs(fl.sum()) < 1e-9 * np.abs(fl).sum()         # compatible
    phi, info = O.solve(beta, fl, h, tol=1e-13, bc=63)
    assert info["status"] == "ok"
    want = phi_e - phi_e.mean()
    np.testing.assert_allclose(phi, want, atol=1e-10 * np.abs(want).max())


def test_linear_field_is_exact_with_mixed_walls():
    shape = (8, 12, 10)
    h = 0.1
    b = 1.7
    bc = (1 << 2) | (1 << 5)          # y- and z+ Neumann, the rest Dirichlet
    x, y, z = centres(shape, h)
    lin = lambda x, y, z: 1 + 2 * x - y + 0.5 * z
    slope = (2.0, -1.0, 0.5)

    def wall(w, x, y, z):
        if (bc >> w) & 1:
            return (1 if w & 1 else -1) * b * slope[w // 2] * np.ones_like(x)
        return lin(x, y, z)

    beta = np.full(shape, b)
    fl = O.bc_lift(beta, h, np.zeros(shape), _packed(shape, h, wall), bc)
    phi, info = O.solve(beta, fl, h, tol=1e-13, bc=bc)
    assert info["status"] == "ok"
    np.testing.assert_allclose(phi, lin(x, y, z), atol=1e-11)


def _manufactured(bc):
    X, Y, Z = sympy.symbols("x y z")
    s = sympy.sin
    beta = 1 + s(2 * sympy.pi * X) * s(2 * sympy.pi * Y) * s(2 * sympy.pi * Z) / 2
    phi = sympy.cos(1.3 * X + 0.2) * s(2 * Y + 0.5) * sympy.cos(Z) + X * Y
    f = sum(sympy.diff(beta * sympy.diff(phi, v), v) for v in (X, Y, Z))
    dphi = [sympy.diff(phi, v) for v in (X, Y, Z)]
    L = lambda e: sympy.lambdify((X, Y, Z), e, "numpy")
    return L(beta), L(phi), L(f), [L(d) for d in dphi]


def _error(n, bc):
    beta_f, phi_f, f_f, dphi = _manufactured(bc)
    shape = (n, n, n)
    h = 1.0 / n
    x, y, z = centres(shape, h)
    beta = beta_f(x, y, z) * np.ones(shape)

    def wall(w, x, y, z):
        if (bc >> w) & 1:
            return (1 if w & 1 else -1) * beta_f(x, y, z) * dphi[w // 2](x, y, z)
        return phi_f(x, y, z)

    fl = O.bc_lift(beta, h, f_f(x, y, z), _packed(shape, h, wall), bc)
    phi, info = O.solve(beta, fl, h, tol=1e-13, bc=bc)
    assert info["status"] == "ok"
    e = phi_f(x, y, z)
    if bc == 63:
        e = e - e.mean()
    return np.abs(phi - e).max()


@pytest.mark.parametrize("bc", [0, 0b010110, 63])
def test_manufactured_solution_converges_at_second_order(bc):
    e16, e32 = _error(16, bc), _error(32, bc)
    assert e32 < 0.02
    assert e16 / e32 > 3.3, (e16, e32)


def _dense_solve(beta, h, f, bc):
    A = O.dense_matrix(O.face_beta(beta, bc), h, beta.shape)
    return np.linalg.solve(A, f.ravel()).reshape(beta.shape)


def test_beta_gradient_with_neumann_walls_matches_finite_differences():
    rng = np.random.default_rng(11)
    shape = (4, 4, 6)
    h = 0.2
    bc = 0b100110
    beta = rng.uniform(0.5, 2.0, shape)
    f = rng.standard_normal(shape)
    t = rng.standard_normal(shape)
    phi = _dense_solve(beta, h, f, bc)
    lam, dbeta, infos = O.adjoint(beta, h, phi, phi - t, bc=bc)
    assert infos[0]["status"] == "ok"
    loss = lambda b: 0.5 * np.sum((_dense_solve(b, h, f, bc) - t) ** 2)
    for idx in [(0, 0, 0), (3, 3, 5), (1, 2, 3), (0, 3, 2), (2, 0, 5)]:
        e = np.zeros(shape)
        e[idx] = 1e-5 * beta[idx]
        fd = (loss(beta + e) - loss(beta - e)) / (2 * e[idx])
        assert abs(dbeta[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), idx
    np.testing.assert_allclose(lam, _dense_solve(beta, h, phi - t, bc), atol=1e-9)


def test_adjoint_of_the_singular_solve_is_rejected():
    beta = np.ones((4, 4, 4))
    _, _, infos = O.adjoint(beta, 0.25, np.zeros_like(beta), np.ones_like(beta), bc=63)
    assert infos[0]["status"] == "bad_hierarchy"


@pytest.mark.parametrize("bc", [0b001001, 63])
def test_velocity_correction_with_neumann_walls(bc):
    rng = np.random.default_rng(bc)
    shape = (5, 6, 7)
    nz, ny, nx = shape
    h = 0.3
    beta = rng.uniform(0.5, 2.0, shape)
    phi = rng.standard_normal(shape)
    u = rng.standard_normal((nz, ny, nx + 1))
    v = rng.standard_normal((nz, ny + 1, nx))
    w = rng.standard_normal((nz + 1, ny, nx))
    u2, v2, w2 = O.correct(beta, h, phi, u, v, w, bc=bc)
    d0, d1 = O.divergence(u, v, w, h), O.divergence(u2, v2, w2, h)
    Aphi = O.apply(O.face_beta(beta, bc), h, phi)
    np.testing.assert_allclose(d1, d0 - Aphi, atol=1e-10 * np.abs(Aphi).max())
    ends = [(u, u2, (slice(None), slice(None), 0)), (u, u2, (slice(None), slice(None), -1)),
            (v, v2, (slice(None), 0, slice(None))), (v, v2, (slice(None), -1, slice(None))),
            (w, w2, (0,)), (w, w2, (-1,))]
    for k, (a, b, sl) in enumerate(ends):
        if (bc >> k) & 1:
            assert np.array_equal(a[sl], b[sl]), WALLS[k]
        else:
            assert not np.array_equal(a[sl], b[sl]), WALLS[k]
