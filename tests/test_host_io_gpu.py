"""Host buffers and the zero initial guess (MG_ZERO_GUESS) through the C ABI:
the solution is the device-buffer solution bit for bit, phi's input is not
read with the flag (it may hold NaN), and host inputs copied in on the
context's copy stream (overlapping the set-up queued by mg_set_beta) are the
ones of this call, also when calls follow each other with different data."""
import numpy as np
import pytest
import torch

from paper_1008_2801_gb300 import BatchSolver, LevelSolver, Solver, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _case(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    return torch.from_numpy(d["beta"]), torch.from_numpy(d["f"]), d["dx"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_buffers_match_device_buffers(cuda_device, precision):
    beta, f, h = _case((32, 48, 64), 1)
    with Solver(tuple(f.shape), h, precision=precision, device=cuda_device) as s:
        s.set_beta(beta.to(cuda_device))
        want, _ = s.solve(f.to(cuda_device), tol=TOL)
        want = want.cpu()
        bh, fh = beta.pin_memory(), f.pin_memory()
        ph = torch.full(f.shape, float("nan"), dtype=torch.float64).pin_memory()
        for _ in range(2):
            s.set_beta(bh)
            got, st = s.solve(fh, phi=ph, tol=TOL, zero_guess=True)
            assert st["status"] == "ok"
            assert got.data_ptr() == ph.data_ptr()
            assert torch.equal(got, want)
            ph.fill_(float("nan"))


def test_consecutive_host_solves_read_their_own_inputs(cuda_device):
    beta, f, h = _case((32, 32, 32), 2)
    rng = np.random.default_rng(3)
    fs = [torch.from_numpy(rng.uniform(-1, 1, f.shape)) for _ in range(4)]
    with Solver(tuple(f.shape), h, device=cuda_device) as s:
        s.set_beta(beta.to(cuda_device))
        want = [s.solve(g.to(cuda_device), tol=TOL)[0].cpu() for g in fs]
        hs = [g.pin_memory() for g in fs]
        for g, w in zip(hs, want):
            s.set_beta(beta.pin_memory())            # a set-up queued before each solve
            got, _ = s.solve(g, tol=TOL)
            assert torch.equal(got, w)
        # with an initial guess from the host (copied in, not ignored)
        got, st = s.solve(hs[0], phi=want[0].clone().pin_memory(), tol=TOL)
        assert st["cycles"] == 0 and torch.equal(got, want[0])


def test_adjoint_after_host_solves(cuda_device):
    beta, f, h = _case((16, 32, 32), 4)
    tgt = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, (2,) + tuple(f.shape)))
    fb = torch.stack([f, -0.5 * f])
    with Solver(tuple(f.shape), h, device=cuda_device) as s:
        s.set_beta(beta.to(cuda_device))
        phi_d, _ = s.solve(fb.to(cuda_device), tol=TOL)
        lam_d, db_d = s.adjoint(phi_d, phi_d - tgt.to(cuda_device), tol=TOL)
        phi_h, _ = s.solve(fb.pin_memory(), tol=TOL)
        lam_h, db_h = s.adjoint(phi_h, (phi_h - tgt).contiguous(), tol=TOL)
        phi_h2, _ = s.solve(fb.pin_memory(), tol=TOL)
    assert torch.equal(phi_h, phi_d.cpu()) and torch.equal(phi_h2, phi_h)
    assert torch.equal(lam_h, lam_d.cpu()) and torch.equal(db_h, db_d.cpu())


def test_batched_and_level_zero_guess_ignore_phi(cuda_device):
    shapes = [(16, 16, 32), (32, 32, 32)]
    cases = [_case(s, 6 + i) for i, s in enumerate(shapes)]
    h = cases[0][2]
    with BatchSolver(shapes, h, device=cuda_device) as b:
        b.set_beta(b.pack([c[0] for c in cases]).to(cuda_device))
        fp = b.pack([c[1] for c in cases]).to(cuda_device)
        want, _ = b.solve(fp, tol=TOL)
        got, st = b.solve(fp, torch.full_like(fp, float("nan")), tol=TOL, zero_guess=True)
        assert all(x["status"] == "ok" for x in st) and torch.equal(got, want)
    beta, f, h = _case((16, 16, 32), 8)
    los, ns = [(0, 0, 0), (16, 0, 0)], [(16, 16, 16)] * 2
    with LevelSolver(los, ns, h, device=cuda_device) as lv:
        lv.set_beta(lv.pack([beta[:, :, :16], beta[:, :, 16:]]).to(cuda_device))
        fp = lv.pack([f[:, :, :16], f[:, :, 16:]]).to(cuda_device)
        want, _ = lv.solve(fp, tol=TOL)
        got, st = lv.solve(fp, torch.full_like(fp, float("nan")), tol=TOL, zero_guess=True)
        assert st["status"] == "ok" and torch.equal(got, want)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(112, 128, 128), (96, 128, 128), (128, 128, 192)])
def test_host_beta_by_slabs_matches_device_beta(cuda_device, shape, precision):
    # a pinned host beta of 4 MiB or more is copied in by slabs of planes,
    # each slab's face weights starting when it has landed (3 slabs of 38,
    # 38 and 36 planes in the first shape, 6 in the last): the set-up, and so
    # the solution, is the device beta's bit for bit, also when a second
    # set-up follows
    beta, f, h = _case(shape, 9)
    assert beta.numel() * 8 >= 2 << 22
    with Solver(tuple(f.shape), h, precision=precision, device=cuda_device) as s:
        s.set_beta(beta.to(cuda_device))
        want, _ = s.solve(f.to(cuda_device), tol=TOL)
        bh = beta.pin_memory()
        for _ in range(2):
            s.set_beta(bh)
            got, st = s.solve(f.to(cuda_device), tol=TOL)
            assert st["status"] == "ok"
            assert torch.equal(got, want)
