"""CPU pins of the oracle's multi-box level: the operator on the union of
disjoint boxes (paper Sec. 2: a MultiFAB level is the union of disjoint
rectangular grids), taken as a mask over the bounding box and solved by
conjugate gradients.

Checked against: the single-box multigrid oracle when the union is one
rectangle; independent single-box solves when the boxes do not share a face;
a dense operator built here from cell adjacency (not from the oracle's face
arrays) and solved directly.
"""
import numpy as np
import pytest

import oracle as O
from paper_1008_2801_gb300 import inputs


def _case(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    return d["beta"], d["f"], d["dx"]


def test_full_mask_is_the_single_box_solve():
    beta, f, h = _case((10, 12, 14), 1)
    mask = np.ones(beta.shape, dtype=np.int32)
    phi, info = O.masked_solve(beta, mask, f, h, tol=1e-13)
    assert info["status"] == "ok"
    ref, _ = O.solve(beta, f, h, tol=1e-13)
    np.testing.assert_allclose(phi, ref, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("gap", [1, 2])
def test_boxes_without_a_shared_face_are_independent(gap):
    # two boxes along x separated by `gap` outside cells
    nz, ny = 6, 5
    beta, f, h = _case((nz + 4, ny + 4, 8 + gap + 7), 2)
    los, ns = [(0, 0, 0), (8 + gap, 0, 0)], [(8, ny, nz), (7, ny, nz)]
    shape = beta.shape
    mask = O.level_mask(los, ns, shape)
    phi, info = O.masked_solve(beta, mask, f, h, tol=1e-13)
    assert info["status"] == "ok"
    for (i, j, k), (a, b, c) in zip(los, ns):
        sl = (slice(k, k + c), slice(j, j + b), slice(i, i + a))
        ref, _ = O.solve(beta[sl], f[sl], h, tol=1e-13)
        np.testing.assert_allclose(phi[sl], ref, atol=1e-10 * np.abs(ref).max())
    assert np.all(phi[mask == 0] == 0.0)


def test_edge_contact_does_not_couple():
    nz, ny, nx = 8, 8, 8
    beta, f, h = _case((nz, ny, nx), 3)
    los, ns = [(0, 0, 0), (4, 4, 0)], [(4, 4, 8), (4, 4, 8)]   # share only the edge x=4, y=4
    mask = O.level_mask(los, ns, beta.shape)
    phi, _ = O.masked_solve(beta, mask, f, h, tol=1e-13)
    for (i, j, k), (a, b, c) in zip(los, ns):
        sl = (slice(k, k + c), slice(j, j + b), slice(i, i + a))
        ref, _ = O.solve(beta[sl], f[sl], h, tol=1e-13)
        np.testing.assert_allclose(phi[sl], ref, atol=1e-10 * np.abs(ref).max())


def _adjacency_matrix(beta, mask, h):
    """-A on the domain cells, built from cell adjacency: each pair of domain
    cells sharing a face couples with the harmonic mean of their beta; each
    face from a domain cell to a non-domain cell (or the box wall) adds 2 beta
    of the cell to its diagonal."""
    nz, ny, nx = beta.shape
    idx = -np.ones(beta.shape, dtype=np.int64)
    cells = np.argwhere(mask != 0)
    idx[tuple(cells.T)] = np.arange(len(cells))
    M = np.zeros((len(cells), len(cells)))
    for r, (k, j, i) in enumerate(cells):
        for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            kk, jj, ii = k + dk, j + dj, i + di
            inside = 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx and mask[kk, jj, ii]
            if inside:
                a, b = beta[k, j, i], beta[kk, jj, ii]
                w = 2 * a * b / (a + b)
                M[r, r] += w
                M[r, idx[kk, jj, ii]] -= w
            else:
                M[r, r] += 2 * beta[k, j, i]
    return M / h ** 2, cells


def test_l_shaped_level_matches_a_dense_solve():
    # three boxes forming an L in x-y, two planes thick
    beta, f, h = _case((2, 6, 6), 4)
    los, ns = [(0, 0, 0), (3, 0, 0), (0, 3, 0)], [(3, 3, 2), (3, 3, 2), (3, 3, 2)]
    mask = O.level_mask(los, ns, beta.shape)
    M, cells = _adjacency_matrix(beta, mask, h)
    np.testing.assert_allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() > 0
    # the oracle's face arrays give the same operator on the domain
    A = O.dense_matrix(O.masked_face_beta(beta, mask), h, beta.shape)
    flat = np.ravel_multi_index(tuple(cells.T), beta.shape)
    np.testing.assert_allclose(-A[np.ix_(flat, flat)], M, atol=1e-10 * np.abs(M).max())
    phi, info = O.masked_solve(beta, mask, f, h, tol=1e-14)
    assert info["status"] == "ok"
    want = np.linalg.solve(-M, f[tuple(cells.T)])
    np.testing.assert_allclose(phi[tuple(cells.T)], want, atol=1e-11 * np.abs(want).max())
    assert np.all(phi[mask == 0] == 0.0)
