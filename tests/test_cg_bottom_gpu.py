"""Boxes whose halving stops at a coarsest level too large for a dense
inverse (more than MG_MAX_BOTTOM = 1024 cells) solve that level by
diagonally preconditioned conjugate gradients on the GPU (GPU).

The oracle solves such a level by conjugate gradients as well; the bottom
solve's accuracy sets only the cycle count, so the GPU solution is held to
the oracle's solution at 1e-9 and to a residual of 1e-10 by the oracle's
own operator.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import Solver, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _dev(a, dev):
    return torch.from_numpy(np.array(a, order="C", copy=True)).to(dev)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(33, 33, 33), (36, 52, 44), (100, 100, 100), (5, 7, 301)])
def test_large_coarsest_level_matches_the_oracle(cuda_device, shape, precision):
    # (nz, ny, nx): 33^3 does not halve at all (the CG solves the whole box);
    # 44 x 52 x 36 stops at 11 x 13 x 9 = 1287 cells; 100^3 at 25^3; the
    # thin odd box at 301 x 7 x 5
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), 60)
    with Solver(shape, d["dx"], precision=precision, device=cuda_device) as s:
        lv = s.levels()
        assert np.prod(lv[-1]) > 1024
        s.set_beta(_dev(d["beta"], cuda_device))
        phi, st = s.solve(_dev(d["f"], cuda_device), tol=TOL)
    assert st["status"] == "ok", st
    got = phi.cpu().numpy()
    r = O.residual(O.face_beta(d["beta"]), d["dx"], d["f"], got)
    assert O.norm2(r) <= 1.01 * TOL * O.norm2(d["f"])
    ref, info = O.solve(d["beta"], d["f"], d["dx"], tol=1e-13)
    assert info["status"] == "ok"
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_large_coarsest_level_with_neumann_walls_krylov_and_no_graph(cuda_device):
    d = inputs.stellar((36, 52, 44), 61)
    shape = d["f"].shape
    beta, f = _dev(d["beta"], cuda_device), _dev(d["f"], cuda_device)
    bc = 1 | 8 | 32     # Neumann x-, y+, z+; the other walls Dirichlet
    ref, _ = O.solve(d["beta"], d["f"], d["dx"], tol=1e-13, bc=bc)
    for kw in ({"use_graph": False}, {"krylov": True}, {"persistent": True}):
        with Solver(shape, d["dx"], bc=bc, device=cuda_device, **kw) as s:
            s.set_beta(beta)
            phi, st = s.solve(f, tol=TOL)
        assert st["status"] == "ok", (kw, st)
        assert np.linalg.norm(phi.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref), kw


def test_large_coarsest_level_is_deterministic(cuda_device):
    d = inputs.stellar(33, 62)
    beta, f = _dev(d["beta"], cuda_device), _dev(d["f"], cuda_device)
    with Solver((33, 33, 33), d["dx"], device=cuda_device) as s:
        s.set_beta(beta)
        a, _ = s.solve(f, tol=TOL)
        b, _ = s.solve(f, tol=TOL)
    assert torch.equal(a, b)
