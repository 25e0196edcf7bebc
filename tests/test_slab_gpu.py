"""The slab-decomposed box (mg_slab_*) against the oracle (GPU).

This run has one GPU, so the slabs are placed on the same device: each has
its own context and stream, and their halo planes move by peer copies
(device-to-device here) exactly as between two GPUs, ordered by events.
The solution must match the oracle's solution of the whole box to 1e-9 at
a relative residual of 1e-10 (by the oracle's operator), whatever the
number of slabs.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import MGError, SlabSolver, Solver, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _dev(a, dev):
    return torch.from_numpy(np.array(a, order="C", copy=True)).to(dev)


def _rel_resid(beta, f, phi, h):
    r = O.residual(O.face_beta(beta), h, f, phi)
    return O.norm2(r) / O.norm2(f)


@pytest.mark.parametrize("shape,nslab", [((64, 64, 64), 2), ((128, 48, 40), 4),
                                         ((96, 64, 64), 3), ((64, 40, 56), 1),
                                         ((256, 32, 32), 8)])
def test_slab_solve_matches_the_oracle(cuda_device, shape, nslab):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), 20 + nslab)
    with SlabSolver(shape, d["dx"], nslab, devices=[cuda_device.index] * nslab) as s:
        assert s.gather >= 1
        s.set_beta(_dev(d["beta"], cuda_device))
        phi, st = s.solve(_dev(d["f"], cuda_device), tol=TOL)
        assert st["status"] == "ok", st
    got = phi.cpu().numpy()
    assert _rel_resid(d["beta"], d["f"], got, d["dx"]) <= TOL * 1.01
    ref, _ = O.solve(d["beta"], d["f"], d["dx"], tol=1e-13)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_slab_solve_tracks_the_single_box_solve(cuda_device):
    # same operator, same V(2,2) cycle structure: the iteration counts agree
    # and the two solutions differ only at the level of the tolerance
    d = inputs.manufactured(64)
    beta, f = _dev(d["beta"], cuda_device), _dev(d["f"], cuda_device)
    with Solver((64, 64, 64), d["dx"], device=cuda_device) as s:
        s.set_beta(beta)
        one, st1 = s.solve(f, tol=TOL)
    with SlabSolver((64, 64, 64), d["dx"], 2) as s:
        s.set_beta(beta)
        two, st2 = s.solve(f, tol=TOL)
    assert st1["status"] == st2["status"] == "ok"
    assert abs(st1["cycles"] - st2["cycles"]) <= 1
    assert (one - two).norm() <= 1e-9 * one.norm()
    # the discretisation error against the exact solution is the same
    e1 = (one.cpu().numpy() - d["phi_exact"])
    e2 = (two.cpu().numpy() - d["phi_exact"])
    assert abs(np.abs(e1).max() - np.abs(e2).max()) <= 1e-6 * np.abs(e1).max()


def test_slab_initial_guess_zero_rhs_and_errors(cuda_device):
    d = inputs.stellar(64, 31)
    beta, f = _dev(d["beta"], cuda_device), _dev(d["f"], cuda_device)
    with SlabSolver((64, 64, 64), d["dx"], 2) as s:
        with pytest.raises(MGError):
            s.solve(f)                      # no beta yet
        s.set_beta(beta)
        phi, st = s.solve(f, tol=TOL)
        again, st2 = s.solve(f, phi=phi.clone(), tol=TOL)   # from the solution
        assert st2["cycles"] == 0 and torch.equal(again, phi)
        z, st3 = s.solve(torch.zeros_like(f), phi=torch.ones_like(f))
        assert st3["status"] == "ok" and not z.any()
    with SlabSolver((64, 64, 64), d["dx"], 2, max_cycles=1) as s:
        s.set_beta(beta)
        _, st4 = s.solve(f, tol=TOL)
        assert st4["status"] == "not_converged" and st4["cycles"] == 1
    with pytest.raises(MGError) as ei:
        SlabSolver((64, 64, 64), 1 / 64, 3)   # 64 planes do not split in 3
    assert ei.value.name == "unsupported"
