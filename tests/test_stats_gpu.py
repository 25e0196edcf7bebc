"""The max-norm residual statistic (opts.max_norm): max |f - A phi| / max |f|
of the returned solution, against the same quantity formed by the oracle's
residual of that solution."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import BatchSolver, Solver, inputs

pytestmark = pytest.mark.gpu


def _case(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    return d["beta"], d["f"], d["dx"]


def _rel_max(beta, f, h, phi, bc=0):
    singular = all(((bc >> (6 + a)) & 1) or ((bc >> (2 * a)) & 3) == 3 for a in range(3))
    fe = f - f.mean() if singular else f          # the solve takes the compatible part
    if bc >> 6:
        r = fe - O.apply_periodic(O.face_beta_periodic(beta, bc), h, phi, bc)
    else:
        r = O.residual(O.face_beta(beta, bc), h, fe, phi)
    return np.abs(r).max() / np.abs(fe).max()


@pytest.mark.parametrize("kw", [{}, {"precision": "mixed"}, {"krylov": True},
                                {"bc": 0b000011}, {"bc": 64 | 128}])
def test_max_norm_matches_the_oracle_residual(cuda_device, kw):
    shape = (16, 24, 32)
    beta, f, h = _case(shape, 70)
    bc = kw.get("bc", 0)
    with Solver(shape, h, device=cuda_device, max_norm=True, **kw) as s:
        s.set_beta(torch.from_numpy(beta).to(cuda_device))
        phi, st = s.solve(torch.from_numpy(f).to(cuda_device), tol=1e-8)
    phi = phi.cpu().numpy()
    want = _rel_max(beta, f, h, phi, bc)
    assert st["rel_resid_max"] > 0
    assert abs(st["rel_resid_max"] - want) <= 1e-6 * want + 1e-15


def test_off_by_default_and_batched(cuda_device):
    shapes = [(16, 16, 16), (8, 24, 32)]
    cases = [_case(sh, 71 + i) for i, sh in enumerate(shapes)]
    h = cases[0][2]
    with Solver(shapes[0], h, device=cuda_device) as s:
        s.set_beta(torch.from_numpy(cases[0][0]).to(cuda_device))
        _, st = s.solve(torch.from_numpy(cases[0][1]).to(cuda_device))
        assert st["rel_resid_max"] == 0.0
    with BatchSolver(shapes, h, device=cuda_device, max_norm=True) as b:
        b.set_beta(b.pack([torch.from_numpy(c[0]) for c in cases]).to(cuda_device))
        phi, sts = b.solve(b.pack([torch.from_numpy(c[1]) for c in cases]).to(cuda_device),
                           tol=1e-8)
        parts = [p.cpu().numpy() for p in b.unpack(phi)]
    for (beta, f, _), p, st in zip(cases, parts, sts):
        assert abs(st["rel_resid_max"] - _rel_max(beta, f, h, p)) <= 1e-6 * st["rel_resid_max"]
