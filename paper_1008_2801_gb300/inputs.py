"""Seeded synthetic inputs for the variable-coefficient Poisson solve.

This module only *generates inputs*: cell-centred coefficient fields beta,
right-hand sides f and targets.  It holds none of the solver's arithmetic
(no face coefficients, no discrete operator, no smoother), so both the CPU
oracle and the CUDA path can be fed from it without sharing method code.

The problem is the one of the paper's Sec. 1: a MAESTRO time step solves a
variable-coefficient Poisson equation div(beta grad phi) = f that follows from
the low-Mach velocity constraint.  The paper prints no workload for it, so the
recipes below are synthetic stand-ins shaped like a white-dwarf convection
run (a centrally condensed stellar density profile, beta = 1/rho):

* ``manufactured``: smooth beta = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z)
  and f = div(beta grad phi_exact) for phi_exact = sin(pi x) sin(pi y) sin(pi z),
  evaluated pointwise at cell centres from the continuous formula.
* ``stellar``: rho(r) = (1 + (r / r_c)^2)^(-3/2) about a centre, multiplied by
  (1 + 0.01 N(0,1)) per-cell noise, beta = 1 / rho; f ~ U[-1, 1] with its mean
  removed.  Draw order from ``numpy.random.default_rng(seed)``: noise, then f,
  then (where used) targets, each in C order (nz, ny, nx).
* ``batched``: many boxes of uneven size, each with its own stellar profile.
* ``inclusions``: high-contrast beta, 1 in a background with random balls
  where beta = contrast (centres ~ U[0.1, 0.9]^3, radii ~ U[0.04, 0.1] of the
  box's x extent), f ~ U[-1, 1]; draw order centres, radii, f.  The
  coefficient jumps are not aligned with coarse cells, the case where a
  V-cycle iteration slows down and CG with a V-cycle preconditioner does not.

Arrays are float64 numpy arrays in C order with shape (nz, ny, nx), x fastest;
cell centres are at x_i = (i + 1/2) dx.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "cell_centres",
    "manufactured",
    "stellar",
    "batched",
    "adjoint_case",
    "inclusions",
    "config",
    "BATCH_SIZES",
]

BATCH_SIZES = (32, 48, 64, 96, 128)


def cell_centres(n, dx):
    """Return broadcastable coordinate arrays (z, y, x) of cell centres."""
    nx, ny, nz = n
    x = (np.arange(nx, dtype=np.float64) + 0.5) * dx
    y = (np.arange(ny, dtype=np.float64) + 0.5) * dx
    z = (np.arange(nz, dtype=np.float64) + 0.5) * dx
    return z[:, None, None], y[None, :, None], x[None, None, :]


def manufactured(n: int):
    """Smooth-coefficient case on the unit cube with n^3 cells (dx = 1/n).

    Returns dict(beta, f, phi_exact, dx).  f is the continuous operator applied
    to phi_exact: grad(beta) . grad(phi) + beta * laplacian(phi).
    """
    dx = 1.0 / n
    z, y, x = cell_centres((n, n, n), dx)
    pi = np.pi
    sx, sy, sz = np.sin(pi * x), np.sin(pi * y), np.sin(pi * z)
    cx, cy, cz = np.cos(pi * x), np.cos(pi * y), np.cos(pi * z)
    Sx, Sy, Sz = np.sin(2 * pi * x), np.sin(2 * pi * y), np.sin(2 * pi * z)
    Cx, Cy, Cz = np.cos(2 * pi * x), np.cos(2 * pi * y), np.cos(2 * pi * z)
    beta = 1.0 + 0.5 * Sx * Sy * Sz
    phi = sx * sy * sz
    # grad beta = pi * (Cx Sy Sz, Sx Cy Sz, Sx Sy Cz); grad phi = pi * (cx sy sz, ...)
    gbgp = pi * pi * (Cx * Sy * Sz * cx * sy * sz
                      + Sx * Cy * Sz * sx * cy * sz
                      + Sx * Sy * Cz * sx * sy * cz)
    f = gbgp - 3.0 * pi * pi * beta * phi
    return {
        "beta": np.ascontiguousarray(np.broadcast_to(beta, (n, n, n))),
        "f": np.ascontiguousarray(np.broadcast_to(f, (n, n, n))),
        "phi_exact": np.ascontiguousarray(np.broadcast_to(phi, (n, n, n))),
        "dx": dx,
    }


def _stellar_beta(n, dx, centre, rc, noise):
    z, y, x = cell_centres(n, dx)
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    rho = (1.0 + r2 / (rc * rc)) ** (-1.5)
    rho = rho * (1.0 + 0.01 * noise)
    return 1.0 / rho


def stellar(n, seed: int, dx: float | None = None, nrhs: int = 0):
    """Stellar-profile beta and random f on an (nx, ny, nz) box.

    ``n`` is an int (cube) or a 3-tuple (nx, ny, nz).  dx defaults to 1/nx so
    the cube spans [0, 1]^3; the profile is centred at (1/2, 1/2, 1/2) with
    core radius 0.3.  With ``nrhs`` > 0 the result also carries ``f_batch``
    (nrhs, nz, ny, nx) drawn after ``f`` and targets ``phi_target`` of the same
    shape drawn after that.
    """
    if isinstance(n, int):
        n = (n, n, n)
    nx, ny, nz = n
    if dx is None:
        dx = 1.0 / nx
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((nz, ny, nx))
    beta = _stellar_beta(n, dx, (0.5, 0.5, 0.5), 0.3, noise)
    del noise
    f = rng.uniform(-1.0, 1.0, (nz, ny, nx))
    f -= f.mean()
    out = {"beta": beta, "f": f, "dx": dx}
    if nrhs:
        fb = rng.uniform(-1.0, 1.0, (nrhs, nz, ny, nx))
        tgt = rng.uniform(-1.0, 1.0, (nrhs, nz, ny, nx))
        out["f_batch"] = fb
        out["phi_target"] = tgt
    return out


def inclusions(n, seed: int, contrast: float = 1e4, count: int = 24,
               dx: float | None = None):
    """High-contrast beta (1 outside, ``contrast`` inside random balls) and
    random f on an (nx, ny, nz) box (``n`` an int for a cube); dx defaults to
    1/nx.  Returns dict(beta, f, dx)."""
    if isinstance(n, int):
        n = (n, n, n)
    nx, ny, nz = n
    if dx is None:
        dx = 1.0 / nx
    rng = np.random.default_rng(seed)
    ext = np.array([nx, ny, nz], dtype=np.float64) * dx
    centres = rng.uniform(0.1, 0.9, (count, 3)) * ext
    radii = rng.uniform(0.04, 0.1, count) * ext[0]
    z, y, x = cell_centres(n, dx)
    inside = np.zeros((nz, ny, nx), dtype=bool)
    for c, r in zip(centres, radii):
        inside |= (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r
    beta = np.where(inside, float(contrast), 1.0)
    f = rng.uniform(-1.0, 1.0, (nz, ny, nx))
    return {"beta": beta, "f": f, "dx": dx}


def batched(nbox: int = 64, seed: int = 4, sizes=BATCH_SIZES, dx: float = 1.0 / 128):
    """Many independent boxes of uneven size, each with its own stellar profile.

    Per-dimension sizes are drawn i.i.d. from ``sizes`` (array (nbox, 3) of
    (nx, ny, nz)), then per box: centre ~ U(0, n_d dx) per dimension, core
    radius ~ U[0.1, 0.4], per-cell noise, f ~ U[-1, 1] minus its mean.
    Returns dict(dims, beta (list), f (list), dx, centres, radii).
    """
    rng = np.random.default_rng(seed)
    dims = rng.choice(np.asarray(sizes, dtype=np.int64), size=(nbox, 3))
    betas, fs, centres, radii = [], [], [], []
    for b in range(nbox):
        nx, ny, nz = (int(v) for v in dims[b])
        centre = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz]) * dx
        rc = rng.uniform(0.1, 0.4)
        noise = rng.standard_normal((nz, ny, nx))
        betas.append(_stellar_beta((nx, ny, nz), dx, centre, rc, noise))
        f = rng.uniform(-1.0, 1.0, (nz, ny, nx))
        f -= f.mean()
        fs.append(f)
        centres.append(centre)
        radii.append(rc)
    return {"dims": dims, "beta": betas, "f": fs, "dx": dx,
            "centres": np.array(centres), "radii": np.array(radii)}


def adjoint_case(n: int = 128, nrhs: int = 8, seed: int = 5):
    """Stellar beta, ``nrhs`` right-hand sides and targets on an n^3 box."""
    d = stellar(n, seed, nrhs=nrhs)
    return {"beta": d["beta"], "f": d["f_batch"], "phi_target": d["phi_target"],
            "dx": d["dx"]}


def config(i: int, scale: int = 1):
    """The five synthetic workloads; ``scale`` divides the linear size.

    1: manufactured 64^3; 2: stellar 256^3 (seed 2); 3: stellar 512^3 (seed 3);
    4: 64 uneven boxes (seed 4); 5: 128^3 with 8 right-hand sides (seed 5).
    """
    if i == 1:
        return manufactured(64 // scale)
    if i == 2:
        return stellar(256 // scale, 2)
    if i == 3:
        return stellar(512 // scale, 3)
    if i == 4:
        return batched(64, 4, sizes=tuple(s // scale for s in BATCH_SIZES),
                       dx=scale / 128.0)
    if i == 5:
        return adjoint_case(128 // scale, 8, 5)
    raise ValueError(f"no workload {i}")
