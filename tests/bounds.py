"""Rounding bounds the tests allow when they re-evaluate a GPU result with
the oracle's operator (test infrastructure, not the solver)."""
import numpy as np


def abs_stencil(faces, h, phi):
    """|A| |phi|: per cell, the sum over its faces of b (|phi_neighbour| +
    |phi_cell|) / h^2 (the neighbour outside the box is 0)."""
    bx, by, bz = faces
    a = np.abs(phi)
    p = np.pad(a, 1)
    s = (bx[:, :, :-1] * (p[1:-1, 1:-1, :-2] + a) + bx[:, :, 1:] * (p[1:-1, 1:-1, 2:] + a) +
         by[:, :-1, :] * (p[1:-1, :-2, 1:-1] + a) + by[:, 1:, :] * (p[1:-1, 2:, 1:-1] + a) +
         bz[:-1] * (p[:-2, 1:-1, 1:-1] + a) + bz[1:] * (p[2:, 1:-1, 1:-1] + a))
    return s / (h * h)


def residual_slack(faces, h, f, phi):
    """Bound on the difference of two FP64 evaluations of f - A phi that
    round differently: each cell's 7-term sum carries at most about 9 units
    of 2^-53 of |f| + |A| |phi| on either side."""
    return 20 * 2.0 ** -53 * float(np.sqrt(np.sum((np.abs(f) + abs_stencil(faces, h, phi)) ** 2)))
