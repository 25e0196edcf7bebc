"""Adjoint / autograd of the solve (GPU) against finite differences and the
CPU oracle's adjoint.  Loss L = 0.5 * sum (phi - phi_target)^2 over all
right-hand sides; dL/df = lambda with A lambda = phi - phi_target and
dL/dbeta from the face products chained through the harmonic face mean."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import MGSolve, Solver, inputs, solve

pytestmark = pytest.mark.gpu


def _dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _grads(case, dev, tol, precision="fp64"):
    beta = _dev(case["beta"], dev).requires_grad_(True)
    f = _dev(case["f"], dev).requires_grad_(True)
    tgt = _dev(case["phi_target"], dev)
    with Solver(tuple(beta.shape), case["dx"], precision=precision, device=dev) as s:
        phi = MGSolve.apply(f, beta, s, tol)
        loss = 0.5 * ((phi - tgt) ** 2).sum()
        loss.backward()
    return phi.detach(), f.grad, beta.grad


def test_adjoint_vs_central_differences_16(cuda_device):
    case = inputs.adjoint_case(16, 2, 5)
    phi, df, dbeta = _grads(case, cuda_device, 1e-13)
    beta, f, tgt, h = case["beta"], case["f"], case["phi_target"], case["dx"]

    def phis(b, ff):
        with Solver(b.shape, h, device=cuda_device) as s:
            s.set_beta(_dev(b, cuda_device))
            p, _ = s.solve(_dev(ff, cuda_device), tol=1e-13)
            return p.cpu().numpy()

    def central(bp, bm, fp, fm, eps):
        pp, pm = phis(bp, fp), phis(bm, fm)
        return np.sum((pp - pm) * (0.5 * (pp + pm) - tgt)) / (2 * eps)

    r = np.random.default_rng(1)
    dbn, dfn = dbeta.cpu().numpy(), df.cpu().numpy()
    for _ in range(5):
        c = tuple(r.integers(0, 16, 3))
        eps = 1e-4 * beta[c]
        bp, bm = beta.copy(), beta.copy()
        bp[c] += eps
        bm[c] -= eps
        fd = central(bp, bm, f, f, eps)
        assert abs(fd - dbn[c]) <= 1e-6 * np.abs(dbn).max()
        b = int(r.integers(0, 2))
        fp, fm = f.copy(), f.copy()
        fp[(b,) + c] += 0.1
        fm[(b,) + c] -= 0.1
        fd = central(beta, beta, fp, fm, 0.1)
        assert abs(fd - dfn[(b,) + c]) <= 1e-6 * np.abs(dfn).max()


@pytest.mark.parametrize("n", [32, 128])
def test_adjoint_vs_oracle(cuda_device, n):
    case = inputs.adjoint_case(n, 8 if n == 128 else 3, 5)
    phi, df, dbeta = _grads(case, cuda_device, 1e-12)
    g = phi.cpu().numpy() - case["phi_target"]
    lam, dbo, infos = O.adjoint(case["beta"], case["dx"], phi.cpu().numpy(), g, tol=1e-13)
    assert all(i["status"] == "ok" for i in infos)
    assert np.linalg.norm(df.cpu().numpy() - lam) <= 1e-9 * np.linalg.norm(lam)
    assert np.linalg.norm(dbeta.cpu().numpy() - dbo) <= 1e-9 * np.linalg.norm(dbo)


def test_euler_identity_on_gpu(cuda_device):
    case = inputs.adjoint_case(24, 2, 6)
    phi, df, dbeta = _grads(case, cuda_device, 1e-13)
    g = phi - _dev(case["phi_target"], cuda_device)
    lhs = (dbeta * _dev(case["beta"], cuda_device)).sum().item()
    rhs = -(g * phi).sum().item()
    assert abs(lhs - rhs) <= 1e-9 * abs(rhs)


def test_functional_solve_is_differentiable(cuda_device):
    case = inputs.adjoint_case(16, 1, 7)
    beta = _dev(case["beta"], cuda_device).requires_grad_(True)
    f = _dev(case["f"][0], cuda_device).requires_grad_(True)
    phi = solve(f, beta, case["dx"], tol=1e-12)
    (phi * phi).sum().backward()
    assert torch.isfinite(beta.grad).all() and torch.isfinite(f.grad).all()
    # d/df of sum(phi^2) = 2 A^-1 phi
    with Solver((16, 16, 16), case["dx"], device=cuda_device) as s:
        s.set_beta(beta.detach())
        want, _ = s.solve((2 * phi).detach(), tol=1e-12)
    assert torch.allclose(f.grad, want, rtol=1e-8, atol=1e-12 * want.abs().max().item())
