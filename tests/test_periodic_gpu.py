"""Periodic axes on the GPU against the oracle's periodic CG solve (wall-mask
bits 6, 7, 8).  Parity bar as for the other solves: relative L2 difference
<= 1e-9 from the oracle at a 1e-13 relative residual; singular cases
(every axis periodic or Neumann on both walls) return the zero-mean
solution."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import BatchSolver, MGError, Solver, inputs, wall_shapes

pytestmark = pytest.mark.gpu

TOL = 1e-10
PX, PY, PZ = 64, 128, 256


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _case(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    return d["beta"], d["f"], d["dx"]


def _solve(beta, f, h, dev, bc, precision="fp64"):
    with Solver(f.shape, h, precision=precision, device=dev, bc=bc) as s:
        s.set_beta(_t(beta, dev))
        phi, st = s.solve(_t(f, dev), tol=TOL)
        return phi.cpu().numpy(), st


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bc", [PX, PY | PZ, PX | PY | PZ, PX | 0b110000, PY | PZ | 0b000011,
                                PZ | 0b000100])
@pytest.mark.parametrize("shape", [(16, 24, 32), (40, 32, 24)])
def test_solve_matches_the_oracle(cuda_device, shape, bc, precision):
    beta, f, h = _case(shape, 60)
    f = f + 0.2
    phi, st = _solve(beta, f, h, cuda_device, bc, precision)
    assert st["status"] == "ok", st
    ref, info = O.periodic_solve(beta, f, h, bc, tol=1e-13)
    assert info["status"] == "ok"
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)
    singular = all(((bc >> (6 + a)) & 1) or ((bc >> (2 * a)) & 3) == 3 for a in range(3))
    if singular:
        assert abs(phi.mean()) <= 1e-13 * np.abs(phi).max()


def test_cyclic_shift_commutes_with_the_gpu_solve(cuda_device):
    shape, bc = (16, 24, 32), PX | PY
    beta, f, h = _case(shape, 61)
    a, _ = _solve(beta, f, h, cuda_device, bc)
    b, _ = _solve(np.roll(beta, (5, 3), (1, 2)), np.roll(f, (5, 3), (1, 2)), h, cuda_device, bc)
    assert np.linalg.norm(b - np.roll(a, (5, 3), (1, 2))) <= 1e-9 * np.linalg.norm(a)


def test_lift_skips_periodic_walls(cuda_device):
    shape, bc = (8, 6, 10), PX | 0b100000
    beta, f, h = _case(shape, 62)
    rng = np.random.default_rng(63)
    walls = [rng.uniform(-1, 1, s) for s in wall_shapes(shape)]
    with Solver(shape, h, device=cuda_device, bc=bc) as s:
        s.set_beta(_t(beta, cuda_device))
        got = s.bc_lift(_t(O.wall_values(walls), cuda_device), _t(f, cuda_device)).cpu().numpy()
    walls[0] = walls[0] * 0
    walls[1] = walls[1] * 0                   # x walls are periodic: nothing lifted
    want = O.bc_lift(beta, h, f, O.wall_values(walls), bc & 63)
    assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))


def test_unsupported_periodic_uses(cuda_device):
    shape = (8, 8, 8)
    beta, f, h = _case(shape, 64)
    with Solver(shape, h, device=cuda_device, bc=PX) as s:
        s.set_beta(_t(beta, cuda_device))
        phi, _ = s.solve(_t(f, cuda_device))
        with pytest.raises(MGError) as e:
            s.adjoint(phi, phi)
        assert e.value.name == "unsupported"
        with pytest.raises(MGError) as e:
            s.solve(_t(np.stack([f, f]), cuda_device))         # several right-hand sides
        assert e.value.name == "unsupported"
        u = torch.zeros((8, 8, 9), dtype=torch.float64, device=cuda_device)
        v = torch.zeros((8, 9, 8), dtype=torch.float64, device=cuda_device)
        w = torch.zeros((9, 8, 8), dtype=torch.float64, device=cuda_device)
        with pytest.raises(MGError) as e:
            s.project_correct(phi, u, v, w)
        assert e.value.name == "unsupported"
    with pytest.raises(MGError) as e:
        BatchSolver([shape, shape], h, device=cuda_device, bc=PX)
    assert e.value.name == "unsupported"
