"""Degenerate and ragged shapes through the whole solve, against the oracle:
single cells, single rows and columns, odd sizes that cannot be halved
(one-level hierarchies solved by the dense coarsest inverse alone), shapes
that halve along some levels only, and batches mixing all of them.  Parity
bar as elsewhere: relative L2 difference <= 1e-9 from the oracle at a 1e-13
relative residual."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import BatchSolver, MGError, Solver, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10
SHAPES = [(1, 1, 1), (1, 1, 9), (1, 8, 1), (7, 1, 1), (2, 2, 2), (3, 5, 7), (1, 16, 16),
          (4, 4, 32), (6, 10, 3), (9, 9, 9)]


def _case(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    return d["beta"], d["f"] + 0.3, d["dx"]      # a non-zero mean: one cell is not 0


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("krylov", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", SHAPES)
def test_degenerate_shapes(cuda_device, shape, precision, krylov):
    beta, f, h = _case(shape, 50)
    with Solver(shape, h, precision=precision, device=cuda_device, krylov=krylov) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, st = s.solve(_t(f, cuda_device), tol=TOL)
    assert st["status"] == "ok", st
    ref, info = O.solve(beta, f, h, tol=1e-13)
    assert info["status"] == "ok"
    assert np.linalg.norm(phi.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_of_degenerate_and_regular_boxes(cuda_device, precision):
    shapes = SHAPES + [(16, 32, 24)]
    cases = [_case(s, 60 + i) for i, s in enumerate(shapes)]
    h = 1.0 / 32
    with BatchSolver(shapes, h, precision=precision, device=cuda_device) as b:
        b.set_beta(b.pack([_t(c[0], cuda_device) for c in cases]))
        phi, sts = b.solve(b.pack([_t(c[1], cuda_device) for c in cases]), tol=TOL)
        parts = [p.cpu().numpy() for p in b.unpack(phi)]
    for (beta, f, _), p, st in zip(cases, parts, sts):
        assert st["status"] == "ok", st
        ref, _ = O.solve(beta, f, h, tol=1e-13)
        assert np.linalg.norm(p - ref) <= 1e-9 * np.linalg.norm(ref)


def test_single_cell_is_one_division(cuda_device):
    # one cell with Dirichlet walls: (A phi) = -6 * 2 beta / h^2 phi
    beta, f, h = np.full((1, 1, 1), 3.0), np.full((1, 1, 1), 5.0), 0.5
    with Solver((1, 1, 1), h, device=cuda_device) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, st = s.solve(_t(f, cuda_device), tol=1e-14)
    assert st["status"] == "ok"
    assert phi.item() == pytest.approx(5.0 / (-12 * 3.0 / 0.25), rel=1e-15)


def test_invalid_shapes_are_rejected(cuda_device):
    for shape in ((0, 4, 4), (4, -1, 4)):
        with pytest.raises(MGError) as e:
            Solver(shape, 0.1, device=cuda_device)
        assert e.value.name == "invalid_arg"
    with pytest.raises(MGError) as e:
        BatchSolver([], 0.1, device=cuda_device)
    assert e.value.name == "invalid_arg"
    with pytest.raises(MGError) as e:
        # 35937-cell coarsest levels in a batch (one box at a time solves them by CG)
        BatchSolver([(33, 33, 33), (8, 8, 8)], 0.1, device=cuda_device)
    assert e.value.name == "unsupported"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(15, 5, 3), (11, 7, 3), (9, 7, 5), (13, 5, 5)])
def test_coarsest_inverse_either_side_of_shared_memory(cuda_device, shape, precision):
    # one-level boxes (odd sides) whose dense inverse is packed in shared
    # memory or kept in global scratch: 225 and 231 cells straddle the FP64
    # limit (n <= 225), 315 and 325 the FP32 one (n <= 319)
    beta, f, h = _case(shape, 70)
    with Solver(shape, h, precision=precision, device=cuda_device) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, st = s.solve(_t(f, cuda_device), tol=TOL)
    assert st["status"] == "ok", st
    ref, info = O.solve(beta, f, h, tol=1e-13)
    assert info["status"] == "ok"
    assert np.linalg.norm(phi.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
