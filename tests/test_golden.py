"""Stored oracle values (tests/golden/) reproduced by the oracle here (CPU)
and by the CUDA solver (GPU)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1008_2801_gb300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden():
    vals = np.loadtxt(os.path.join(HERE, "stellar_12x4x8.txt"))
    return vals.reshape(8, 4, 12), inputs.stellar((12, 4, 8), 77)


def test_oracle_reproduces_the_stored_solution():
    want, d = _golden()
    phi, info = O.solve(d["beta"], d["f"], d["dx"], tol=1e-14)
    assert info["status"] == "ok"
    assert np.max(np.abs(phi - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gpu_reproduces_the_stored_solution(cuda_device, precision):
    import torch
    from paper_1008_2801_gb300 import Solver
    want, d = _golden()
    with Solver((8, 4, 12), d["dx"], precision=precision, device=cuda_device) as s:
        s.set_beta(torch.from_numpy(d["beta"]).to(cuda_device))
        phi, st = s.solve(torch.from_numpy(d["f"]).to(cuda_device), tol=1e-12)
    assert st["status"] == "ok"
    assert np.linalg.norm(phi.cpu().numpy() - want) <= 1e-9 * np.linalg.norm(want)
