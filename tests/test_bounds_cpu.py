"""The rounding allowance the GPU tests use when they re-evaluate a result's
residual with the oracle: |A| |phi| is what it says, and the allowance
covers the gap between two FP64 evaluations of f - A phi that sum in
different orders (here the oracle's stencil loop and a dense product)."""
import numpy as np
import pytest

import oracle as O
from bounds import abs_stencil, residual_slack


@pytest.mark.parametrize("bc", [0, 63, 0b010110])
@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 2, 6)])
def test_abs_stencil_is_abs_A_times_abs_phi(shape, bc):
    rng = np.random.default_rng(11)
    h = 0.25
    beta = rng.uniform(0.5, 2.0, shape)
    phi = rng.uniform(-1.0, 1.0, shape)
    faces = O.face_beta(beta, bc)
    A = O.dense_matrix(faces, h, shape)
    want = (np.abs(A) @ np.abs(phi).ravel()).reshape(shape)
    got = abs_stencil(faces, h, phi)
    assert np.max(np.abs(got - want)) <= 1e-14 * np.max(want)


@pytest.mark.parametrize("contrast", [1.0, 1e4, 1e6])
def test_slack_covers_two_evaluation_orders(contrast):
    # a near-solution phi (so that f - A phi cancels, where rounding shows)
    # of a problem with beta spread over `contrast`
    rng = np.random.default_rng(12)
    shape = (6, 7, 8)
    h = 1.0 / 8
    beta = 10.0 ** rng.uniform(0.0, np.log10(contrast) if contrast > 1 else 0.0, shape)
    faces = O.face_beta(beta)
    A = O.dense_matrix(faces, h, shape)
    phi = rng.uniform(-1.0, 1.0, shape)
    f = (A @ phi.ravel()).reshape(shape) * (1 + 1e-12 * rng.uniform(-1, 1, shape))
    r_loop = O.residual(faces, h, f, phi)
    r_dense = f - (A @ phi.ravel()).reshape(shape)
    gap = float(np.linalg.norm(r_loop - r_dense))
    slack = residual_slack(faces, h, f, phi)
    assert gap <= slack
    # and the allowance is a rounding allowance: far below the residual of a
    # cruder iterate
    assert slack <= 1e-12 * float(np.linalg.norm(np.abs(f) + abs_stencil(faces, h, phi)))
