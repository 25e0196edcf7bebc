"""Projection steps around the solve (GPU) against the oracle: the divergence
right-hand side, the velocity correction, and the constraint div(u') = S
after a projection.  Tolerance: each output sums at most 6 differences, so
1e-13 of the term scale (100x the FP64 rounding bound)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import Solver, inputs

pytestmark = pytest.mark.gpu

SHAPES = [(6, 10, 14), (24, 40, 56), (40, 24, 56)]


def _case(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    r = np.random.default_rng(seed + 7)
    u = r.standard_normal((nz, ny, nx + 1))
    v = r.standard_normal((nz, ny + 1, nx))
    w = r.standard_normal((nz + 1, ny, nx))
    S = r.standard_normal(shape)
    return d, u, v, w, S


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("shape", SHAPES)
def test_divergence_rhs(cuda_device, shape):
    d, u, v, w, S = _case(shape, 1)
    with Solver(shape, d["dx"], device=cuda_device) as s:
        for src in (S, None):
            f = s.project_rhs(_t(u, cuda_device), _t(v, cuda_device), _t(w, cuda_device),
                              None if src is None else _t(src, cuda_device))
            want = O.divergence(u, v, w, d["dx"], src)
            scale = 6 * max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max()) / d["dx"] + 1
            assert np.max(np.abs(f.cpu().numpy() - want)) <= 1e-13 * scale


@pytest.mark.parametrize("shape", SHAPES)
def test_velocity_correction(cuda_device, shape):
    d, u, v, w, _ = _case(shape, 2)
    phi = np.random.default_rng(3).uniform(-1, 1, shape)
    with Solver(shape, d["dx"], device=cuda_device) as s:
        s.set_beta(_t(d["beta"], cuda_device))
        tu, tv, tw = _t(u, cuda_device), _t(v, cuda_device), _t(w, cuda_device)
        s.project_correct(_t(phi, cuda_device), tu, tv, tw)
        want = O.correct(d["beta"], d["dx"], phi, u, v, w)
        for got, ref in zip((tu, tv, tw), want):
            scale = np.abs(ref).max() + 2 * d["beta"].max() / d["dx"]
            assert np.max(np.abs(got.cpu().numpy() - ref)) <= 1e-13 * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_projection_enforces_the_constraint(cuda_device, precision):
    shape = (48, 32, 40)
    d, u, v, w, S = _case(shape, 4)
    with Solver(shape, d["dx"], precision=precision, device=cuda_device) as s:
        s.set_beta(_t(d["beta"], cuda_device))
        tu, tv, tw = _t(u, cuda_device), _t(v, cuda_device), _t(w, cuda_device)
        phi, st = s.project(tu, tv, tw, _t(S, cuda_device), tol=1e-10)
        assert st["status"] == "ok"
    f = O.divergence(u, v, w, d["dx"], S)
    div = O.divergence(tu.cpu().numpy(), tv.cpu().numpy(), tw.cpu().numpy(), d["dx"])
    assert np.linalg.norm(div - S) <= 1.01e-10 * np.linalg.norm(f)
