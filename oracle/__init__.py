"""Plain FP64 CPU oracle for the variable-coefficient Poisson solve.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The solver package never imports this
module, and this module imports nothing from the solver package.

The arithmetic lives in ``oracle.c`` (plain C loops, one definition per
function, each stated in that file's header); this wrapper only marshals
numpy arrays.  Arrays are float64 in C order: cells (nz, ny, nx), x faces
(nz, ny, nx+1), y faces (nz, ny+1, nx), z faces (nz+1, ny, nx).

Walls: every function that builds face coefficients takes ``bc``, a mask
with bit w set when wall w (x-, x+, y-, y+, z-, z+) is Neumann; 0 means every
wall Dirichlet.  ``bc_lift`` moves non-zero wall values to the right-hand side;
``wall_values`` gives the packed layout of those values.

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle.py`` (closed forms, invariants, dense direct solves and
finite differences); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I = ctypes.c_int
_F = ctypes.c_double

STATUS = {0: "ok", 1: "not_converged", 2: "nonfinite", 3: "bad_hierarchy"}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_num_threads.restype = _I
            L.oracle_set_threads.argtypes = [_I]
            L.oracle_face_beta.argtypes = [_I, _I, _I, _D, _D, _D, _D]
            L.oracle_face_beta_bc.argtypes = [_I, _I, _I, _D, _I, _D, _D, _D]
            L.oracle_bc_lift.argtypes = [_I, _I, _I, _F, _D, _I, _D, _D]
            L.oracle_coarsen_faces.argtypes = [_I, _I, _I, _D, _D, _D, _D, _D, _D]
            L.oracle_apply.argtypes = [_I, _I, _I, _F, _D, _D, _D, _D, _D]
            L.oracle_residual.argtypes = [_I, _I, _I, _F, _D, _D, _D, _D, _D, _D]
            L.oracle_rbgs_pass.argtypes = [_I, _I, _I, _F, _D, _D, _D, _D, _D, _I]
            L.oracle_restrict.argtypes = [_I, _I, _I, _D, _D]
            L.oracle_prolong_add.argtypes = [_I, _I, _I, _D, _D]
            L.oracle_norm2.argtypes = [ctypes.c_longlong, _D]
            L.oracle_norm2.restype = _F
            L.oracle_levels.argtypes = [_I, _I, _I, np.ctypeslib.ndpointer(dtype=np.int32)]
            L.oracle_levels.restype = _I
            L.oracle_solve.argtypes = [_I, _I, _I, _F, _D, _D, _D, _F, _I, _I, _I, _D,
                                       ctypes.POINTER(_I)]
            L.oracle_solve.restype = _I
            L.oracle_solve_bc.argtypes = [_I, _I, _I, _F, _D, _I, _D, _D, _F, _I, _I, _I, _D,
                                          ctypes.POINTER(_I)]
            L.oracle_solve_bc.restype = _I
            L.oracle_beta_grad_bc.argtypes = [_I, _I, _I, _F, _D, _I, _D, _D, _D]
            L.oracle_adjoint_bc.argtypes = [_I, _I, _I, _F, _D, _I, _D, _D, _D, _D, _F, _I,
                                            ctypes.POINTER(_I)]
            L.oracle_adjoint_bc.restype = _I
            L.oracle_beta_grad.argtypes = [_I, _I, _I, _F, _D, _D, _D, _D]
            L.oracle_adjoint.argtypes = [_I, _I, _I, _F, _D, _D, _D, _D, _D, _F, _I,
                                         ctypes.POINTER(_I)]
            L.oracle_adjoint.restype = _I
            DN = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
            L.oracle_divergence.argtypes = [_I, _I, _I, _F, _D, _D, _D, ctypes.c_void_p, _D]
            L.oracle_correct.argtypes = [_I, _I, _I, _F, _D, _D, DN, DN, DN]
            L.oracle_correct_bc.argtypes = [_I, _I, _I, _F, _D, _I, _D, DN, DN, DN]
            _M = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
            L.oracle_masked_face_beta.argtypes = [_I, _I, _I, _D, _M, _D, _D, _D]
            L.oracle_masked_solve.argtypes = [_I, _I, _I, _F, _D, _M, _D, _D, _F, _I,
                                              ctypes.POINTER(_I)]
            L.oracle_masked_solve.restype = _I
            L.oracle_face_beta_periodic.argtypes = [_I, _I, _I, _D, _I, _D, _D, _D]
            L.oracle_apply_periodic.argtypes = [_I, _I, _I, _F, _D, _D, _D, _I, _D, _D]
            L.oracle_periodic_solve.argtypes = [_I, _I, _I, _F, _D, _I, _D, _D, _F, _I,
                                                ctypes.POINTER(_I)]
            L.oracle_periodic_solve.restype = _I
            L.oracle_vcycle_apply.argtypes = [_I, _I, _I, _F, _D, _I, _I, _I, _D, _D]
            L.oracle_vcycle_apply.restype = _I
            L.oracle_pcg_solve.argtypes = [_I, _I, _I, _F, _D, _I, _D, _D, _F, _I, _I, _D,
                                           ctypes.POINTER(_I)]
            L.oracle_pcg_solve.restype = _I
            _lib = L
    return _lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(a):
    nz, ny, nx = a.shape
    return nx, ny, nz


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def face_beta(beta, bc=0):
    """Face coefficients (bx, by, bz) from cell beta: harmonic mean inside;
    2 beta on Dirichlet walls, 0 on the Neumann walls of the mask ``bc``."""
    beta = _c(beta)
    nx, ny, nz = _dims(beta)
    bx = np.empty((nz, ny, nx + 1))
    by = np.empty((nz, ny + 1, nx))
    bz = np.empty((nz + 1, ny, nx))
    lib().oracle_face_beta_bc(nx, ny, nz, beta, int(bc), bx, by, bz)
    return bx, by, bz


def wall_shapes(shape):
    """Shapes of the six packed wall arrays (x-, x+, y-, y+, z-, z+) of an
    (nz, ny, nx) box: x walls (nz, ny), y walls (nz, nx), z walls (ny, nx)."""
    nz, ny, nx = shape
    return [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]


def wall_values(walls):
    """Packs six wall arrays (x-, x+, y-, y+, z-, z+) into one flat array."""
    return np.concatenate([_c(w).ravel() for w in walls])


def bc_lift(beta, h, f, vals, bc=0):
    """f minus the lift of the packed wall values ``vals`` (Dirichlet: phi on
    the wall; Neumann: outward flux beta dphi/dn), for walls of mask ``bc``."""
    beta = _c(beta)
    f = _c(f).copy()
    vals = _c(vals).ravel()
    nx, ny, nz = _dims(beta)
    assert vals.size == 2 * (ny * nz + nz * nx + ny * nx)
    lib().oracle_bc_lift(nx, ny, nz, float(h), beta, int(bc), vals, f)
    return f


def coarsen_faces(bx, by, bz):
    """Coarse faces (mean of the 4 fine faces) of a fine level with even dimensions."""
    bx, by, bz = _c(bx), _c(by), _c(bz)
    nz, ny, nx = bx.shape[0], bx.shape[1], bx.shape[2] - 1
    cx, cy, cz = nx // 2, ny // 2, nz // 2
    cbx = np.empty((cz, cy, cx + 1))
    cby = np.empty((cz, cy + 1, cx))
    cbz = np.empty((cz + 1, cy, cx))
    lib().oracle_coarsen_faces(nx, ny, nz, bx, by, bz, cbx, cby, cbz)
    return cbx, cby, cbz


def apply(faces, h, phi):
    """A phi for faces (bx, by, bz) and spacing h."""
    bx, by, bz = (_c(a) for a in faces)
    phi = _c(phi)
    nx, ny, nz = _dims(phi)
    out = np.empty_like(phi)
    lib().oracle_apply(nx, ny, nz, float(h), bx, by, bz, phi, out)
    return out


def residual(faces, h, f, phi):
    bx, by, bz = (_c(a) for a in faces)
    f, phi = _c(f), _c(phi)
    nx, ny, nz = _dims(phi)
    r = np.empty_like(phi)
    lib().oracle_residual(nx, ny, nz, float(h), bx, by, bz, f, phi, r)
    return r


def rbgs_pass(faces, h, f, phi, color):
    """One red (0) or black (1) Gauss-Seidel pass; returns the updated copy."""
    bx, by, bz = (_c(a) for a in faces)
    f = _c(f)
    phi = _c(phi).copy()
    nx, ny, nz = _dims(phi)
    lib().oracle_rbgs_pass(nx, ny, nz, float(h), bx, by, bz, f, phi, int(color))
    return phi


def restrict(fine):
    fine = _c(fine)
    nx, ny, nz = _dims(fine)
    out = np.empty((nz // 2, ny // 2, nx // 2))
    lib().oracle_restrict(nx, ny, nz, fine, out)
    return out


def prolong_add(coarse, fine):
    """Returns fine + piecewise-constant prolongation of coarse."""
    coarse = _c(coarse)
    fine = _c(fine).copy()
    nx, ny, nz = _dims(fine)
    lib().oracle_prolong_add(nx, ny, nz, coarse, fine)
    return fine


def norm2(x) -> float:
    x = _c(x).ravel()
    return lib().oracle_norm2(x.size, x)


def levels(n):
    """Level dimensions [(nx, ny, nz), ...] of the multigrid hierarchy."""
    nx, ny, nz = n
    d = np.zeros(96, dtype=np.int32)
    k = lib().oracle_levels(int(nx), int(ny), int(nz), d)
    return [tuple(int(v) for v in d[3 * i:3 * i + 3]) for i in range(k)]


def solve(beta, f, h, tol=1e-13, max_cycles=200, phi0=None, nu1=2, nu2=2, bc=0):
    """Solve div(beta grad phi) = f with homogeneous walls of mask ``bc``;
    returns (phi, info dict).  With every wall Neumann (bc = 63) f loses its
    mean and phi has zero mean."""
    beta, f = _c(beta), _c(f)
    nx, ny, nz = _dims(f)
    phi = np.zeros_like(f) if phi0 is None else _c(phi0).copy()
    hist = np.zeros(max_cycles + 1)
    cyc = _I(0)
    s = lib().oracle_solve_bc(nx, ny, nz, float(h), beta, int(bc), f, phi, float(tol),
                              int(max_cycles), int(nu1), int(nu2), hist, ctypes.byref(cyc))
    return phi, {"status": STATUS[s], "cycles": cyc.value, "hist": hist[:cyc.value + 1].copy()}


def vcycle_apply(beta, h, r, nu=2, sym=True, bc=0):
    """z = V r: one V(nu, nu) cycle from a zero start on the right-hand side
    r; sym selects black-then-red post-smoothing (the symmetric cycle)."""
    beta, r = _c(beta), _c(r)
    nx, ny, nz = _dims(r)
    z = np.zeros_like(r)
    s = lib().oracle_vcycle_apply(nx, ny, nz, float(h), beta, int(bc), int(nu), int(bool(sym)),
                                  r, z)
    if s != 0:
        raise ValueError(f"oracle_vcycle_apply: status {STATUS[s]}")
    return z


def pcg_solve(beta, f, h, tol=1e-13, maxit=200, phi0=None, nu=2, bc=0):
    """Conjugate gradients on -A phi = -f preconditioned by -V (the
    symmetric V(nu, nu) cycle); returns (phi, info dict with status,
    iterations and the relative residual history)."""
    beta, f = _c(beta), _c(f)
    nx, ny, nz = _dims(f)
    phi = np.zeros_like(f) if phi0 is None else _c(phi0).copy()
    hist = np.zeros(maxit + 1)
    it = _I(0)
    s = lib().oracle_pcg_solve(nx, ny, nz, float(h), beta, int(bc), f, phi, float(tol),
                               int(maxit), int(nu), hist, ctypes.byref(it))
    return phi, {"status": STATUS[s], "cycles": it.value, "hist": hist[:it.value + 1].copy()}


def beta_grad(beta, h, phi, lam, bc=0):
    """dL/dbeta_cell from one (phi, lambda) pair."""
    beta, phi, lam = _c(beta), _c(phi), _c(lam)
    nx, ny, nz = _dims(beta)
    out = np.zeros_like(beta)
    lib().oracle_beta_grad_bc(nx, ny, nz, float(h), beta, int(bc), phi, lam, out)
    return out


def adjoint(beta, h, phi, g, tol=1e-13, max_cycles=200, bc=0):
    """Returns (lambda = dL/df, dL/dbeta_cell, info) for dL/dphi = g.

    ``phi`` and ``g`` may carry a leading right-hand-side dimension; the beta
    gradient is summed over it.
    """
    beta = _c(beta)
    phi, g = _c(phi), _c(g)
    single = phi.ndim == 3
    if single:
        phi, g = phi[None], g[None]
    nx, ny, nz = _dims(beta)
    lam = np.zeros_like(g)
    dbeta = np.zeros_like(beta)
    infos = []
    for b in range(phi.shape[0]):
        lb = np.zeros_like(beta)
        cyc = _I(0)
        s = lib().oracle_adjoint_bc(nx, ny, nz, float(h), beta, int(bc), _c(phi[b]), _c(g[b]),
                                    lb, dbeta, float(tol), int(max_cycles), ctypes.byref(cyc))
        lam[b] = lb
        infos.append({"status": STATUS[s], "cycles": cyc.value})
    return (lam[0] if single else lam), dbeta, infos


def divergence(u, v, w, h, S=None):
    """f = div(u, v, w) - S on the cells (face arrays in their natural layouts)."""
    u, v, w = _c(u), _c(v), _c(w)
    nz, ny, nx1 = u.shape
    nx = nx1 - 1
    f = np.empty((nz, ny, nx))
    Sp = None
    if S is not None:
        S = _c(S)
        Sp = S.ctypes.data_as(ctypes.c_void_p)
    lib().oracle_divergence(nx, ny, nz, float(h), u, v, w, Sp, f)
    return f


def correct(beta, h, phi, u, v, w, bc=0):
    """Returns the face velocities minus beta_face grad(phi) (copies)."""
    beta, phi = _c(beta), _c(phi)
    u, v, w = _c(u).copy(), _c(v).copy(), _c(w).copy()
    nx, ny, nz = _dims(beta)
    lib().oracle_correct_bc(nx, ny, nz, float(h), beta, int(bc), phi, u, v, w)
    return u, v, w


def dense_matrix(faces, h, shape):
    """A as a dense (N, N) matrix, column c = A e_c (small grids only)."""
    nz, ny, nx = shape
    n = nx * ny * nz
    A = np.empty((n, n))
    e = np.zeros(n)
    for c in range(n):
        e[:] = 0.0
        e[c] = 1.0
        A[:, c] = apply(faces, h, e.reshape(shape)).ravel()
    return A


def masked_face_beta(beta, mask):
    """Face coefficients of the domain mask != 0 inside beta's box: harmonic
    mean between domain cells, 2 beta on faces to the outside, 0 elsewhere."""
    beta = _c(beta)
    mask = np.ascontiguousarray(mask, dtype=np.int32)
    nx, ny, nz = _dims(beta)
    bx = np.empty((nz, ny, nx + 1))
    by = np.empty((nz, ny + 1, nx))
    bz = np.empty((nz + 1, ny, nx))
    lib().oracle_masked_face_beta(nx, ny, nz, beta, mask, bx, by, bz)
    return bx, by, bz


def masked_solve(beta, mask, f, h, tol=1e-13, maxit=100000):
    """Solve div(beta grad phi) = f on the domain mask != 0 (Dirichlet walls on
    its boundary) by conjugate gradients; phi = 0 outside.  Returns (phi, info)."""
    beta, f = _c(beta), _c(f)
    mask = np.ascontiguousarray(mask, dtype=np.int32)
    nx, ny, nz = _dims(beta)
    phi = np.zeros_like(f)
    it = _I(0)
    s = lib().oracle_masked_solve(nx, ny, nz, float(h), beta, mask, f, phi, float(tol),
                                  int(maxit), ctypes.byref(it))
    return phi, {"status": STATUS[s], "iterations": it.value}


def level_mask(los, ns, shape):
    """Mask over an (nz, ny, nx) bounding box of the union of boxes with lower
    corners los[b] = (i, j, k) and dims ns[b] = (nx, ny, nz)."""
    m = np.zeros(shape, dtype=np.int32)
    for (i, j, k), (a, b, c) in zip(los, ns):
        m[k:k + c, j:j + b, i:i + a] = 1
    return m


def face_beta_periodic(beta, bc):
    """Face coefficients with the wall mask bc, whose bits 6, 7, 8 make the x,
    y, z axis periodic (faces 0 and n: the face between cells n-1 and 0)."""
    beta = _c(beta)
    nx, ny, nz = _dims(beta)
    bx = np.empty((nz, ny, nx + 1))
    by = np.empty((nz, ny + 1, nx))
    bz = np.empty((nz + 1, ny, nx))
    lib().oracle_face_beta_periodic(nx, ny, nz, beta, int(bc), bx, by, bz)
    return bx, by, bz


def apply_periodic(faces, h, phi, bc):
    """A phi with periodic axes wrapped (faces from face_beta_periodic)."""
    bx, by, bz = (_c(a) for a in faces)
    phi = _c(phi)
    nx, ny, nz = _dims(phi)
    out = np.empty_like(phi)
    lib().oracle_apply_periodic(nx, ny, nz, float(h), bx, by, bz, int(bc), phi, out)
    return out


def periodic_solve(beta, f, h, bc, tol=1e-13, maxit=100000):
    """Solve div(beta grad phi) = f with the walls and periodic axes of bc by
    conjugate gradients (zero-mean solution when A is singular)."""
    beta, f = _c(beta), _c(f)
    nx, ny, nz = _dims(beta)
    phi = np.zeros_like(f)
    it = _I(0)
    s = lib().oracle_periodic_solve(nx, ny, nz, float(h), beta, int(bc), f, phi, float(tol),
                                    int(maxit), ctypes.byref(it))
    return phi, {"status": STATUS[s], "iterations": it.value}
