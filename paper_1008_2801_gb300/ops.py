"""Single-stage entry points (include/mg_ops.h) on torch tensors.

A level array of an (nz, ny, nx) box is a tensor of shape (nz + 2, ny + 1, P)
with P = round_up(nx + 1, 8): element (i, j, k) of the C layout sits at
[k + 1, j, i].  ``level()`` allocates one (zero-filled), ``put``/``get`` move
natural-layout data in and out.  Natural layouts: cells (nz, ny, nx), x faces
(nz, ny, nx + 1), y faces (nz, ny + 1, nx), z faces (nz + 1, ny, nx).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check

_PREC = {torch.float64: _lib.MG_OPS_F64, torch.float32: _lib.MG_OPS_F32}


def _n(shape):
    nz, ny, nx = shape
    return _lib.c_int3(nx, ny, nz)


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _s(t):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def layout(shape):
    P, Q, E = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    check(_lib.load().mg_layout(_n(shape), ctypes.byref(P), ctypes.byref(Q), ctypes.byref(E)),
          "mg_layout")
    return P.value, Q.value, E.value


def level(shape, dtype=torch.float64, device="cuda"):
    nz, ny, nx = shape
    P, Q, E = layout(shape)
    assert E == (nz + 2) * (ny + 1) * P
    return torch.zeros((nz + 2, ny + 1, P), dtype=dtype, device=device)


def _view(t, shape, kind):
    nz, ny, nx = shape
    if kind == "cell":
        return t[1:nz + 1, 0:ny, 0:nx]
    if kind == "x":
        return t[1:nz + 1, 0:ny, 0:nx + 1]
    if kind == "y":
        return t[1:nz + 1, 0:ny + 1, 0:nx]
    if kind == "z":
        return t[1:nz + 2, 0:ny, 0:nx]
    raise ValueError(kind)


def put(t, shape, data, kind="cell"):
    _view(t, shape, kind).copy_(torch.as_tensor(data, dtype=t.dtype, device=t.device))
    return t


def get(t, shape, kind="cell"):
    return _view(t, shape, kind).clone()


def face_weights(beta: torch.Tensor, h: float, bc: int = 0):
    shape = tuple(beta.shape)
    w = [level(shape, device=beta.device) for _ in range(3)]
    check(_lib.load().mg_op_face_weights(_n(shape), float(h), int(bc), _p(beta), *map(_p, w),
                                         _s(beta)), "mg_op_face_weights")
    return w


def coarsen_weights(w, shape):
    nz, ny, nx = shape
    c = (nz // 2, ny // 2, nx // 2)
    cw = [level(c, device=w[0].device) for _ in range(3)]
    check(_lib.load().mg_op_coarsen_weights(_n(shape), *map(_p, w), *map(_p, cw), _s(w[0])),
          "mg_op_coarsen_weights")
    return cw


def inv_diag(w, shape, with_diag=False):
    d = level(shape, device=w[0].device)
    D = level(shape, device=w[0].device) if with_diag else None
    check(_lib.load().mg_op_inv_diag(_n(shape), *map(_p, w), _p(d), _p(D), _s(d)),
          "mg_op_inv_diag")
    return (d, D) if with_diag else d


def round_f32(w, invD, shape):
    out = [level(shape, torch.float32, w[0].device) for _ in range(4)]
    check(_lib.load().mg_op_round_f32(_n(shape), *map(_p, w), _p(invD), *map(_p, out),
                                      _s(invD)), "mg_op_round_f32")
    return out[:3], out[3]


def rbgs_pass(w, invD, f, phi, shape, color):
    check(_lib.load().mg_op_rbgs_pass(_PREC[phi.dtype], _n(shape), *map(_p, w), _p(invD), _p(f),
                                      _p(phi), int(color), _s(phi)), "mg_op_rbgs_pass")
    return phi


def rbgs_sweep(w, f, phi_in, shape, phi_out=None, zc=0):
    """Fused red+black sweep, out of place (1/D from the weights)."""
    if phi_out is None:
        phi_out = torch.zeros_like(phi_in)
    check(_lib.load().mg_op_rbgs_sweep(_PREC[phi_in.dtype], _n(shape), *map(_p, w), _p(f),
                                       _p(phi_in), _p(phi_out), int(zc), _s(phi_in)),
          "mg_op_rbgs_sweep")
    return phi_out


def rbgs_sweep_tma(w, f, phi_in, shape, phi_out=None, zc=0):
    """FP32 fused sweep with TMA-staged tiles (bitwise equal to rbgs_sweep)."""
    if phi_out is None:
        phi_out = torch.zeros_like(phi_in)
    check(_lib.load().mg_op_rbgs_sweep_tma(_n(shape), *map(_p, w), _p(f), _p(phi_in),
                                           _p(phi_out), int(zc), _s(phi_in)),
          "mg_op_rbgs_sweep_tma")
    return phi_out


def rbgs_sweep_tma_prolong(w, f, phic, phi_in, shape, phi_out=None, zc=0):
    """The TMA sweep with the prolongation phi_in += phic(parent) fused
    (phi_in itself left unchanged)."""
    if phi_out is None:
        phi_out = torch.zeros_like(phi_in)
    check(_lib.load().mg_op_rbgs_sweep_tma_prolong(_n(shape), *map(_p, w), _p(f), _p(phic),
                                                   _p(phi_in), _p(phi_out), int(zc),
                                                   _s(phi_in)),
          "mg_op_rbgs_sweep_tma_prolong")
    return phi_out


def residual(w, f, phi, shape, D=None):
    r = torch.zeros_like(phi)
    check(_lib.load().mg_op_residual(_PREC[phi.dtype], _n(shape), *map(_p, w), _p(D), _p(f),
                                     _p(phi), _p(r), _s(phi)), "mg_op_residual")
    return r


def residual_restrict(w, f, phi, shape, D=None, red_only=False):
    nz, ny, nx = shape
    c = (nz // 2, ny // 2, nx // 2)
    fc = level(c, phi.dtype, phi.device)
    phic = level(c, phi.dtype, phi.device)
    phic.fill_(7.0)  # must come back zero inside the box
    L = _lib.load()
    fn = L.mg_op_residual_restrict_red if red_only else L.mg_op_residual_restrict
    check(fn(_PREC[phi.dtype], _n(shape), *map(_p, w), _p(D), _p(f), _p(phi), _p(fc), _p(phic),
             _s(phi)), "mg_op_residual_restrict")
    return fc, phic


def prolong_add(phic, phi, shape):
    check(_lib.load().mg_op_prolong_add(_PREC[phi.dtype], _n(shape), _p(phic), _p(phi), _s(phi)),
          "mg_op_prolong_add")
    return phi


def bottom_inverse(w, shape, singular=False):
    nz, ny, nx = shape
    n = nx * ny * nz
    work = torch.empty(n * n, dtype=torch.float64, device=w[0].device)
    ainv = torch.empty((n, n), dtype=torch.float64, device=w[0].device)
    check(_lib.load().mg_op_bottom_inverse(_n(shape), int(bool(singular)), *map(_p, w), _p(work),
                                           _p(ainv), _s(ainv)), "mg_op_bottom_inverse")
    return ainv


def bottom_solve(ainv, f, shape):
    phi = torch.zeros_like(f)
    check(_lib.load().mg_op_bottom_solve(_PREC[f.dtype], _n(shape), _p(ainv), _p(f), _p(phi),
                                         _s(f)), "mg_op_bottom_solve")
    return phi


def residual_norm(w, f, phi, shape, D=None):
    L = _lib.load()
    m = L.mg_op_norm_scratch(_n(shape))
    part = torch.empty(max(int(m), 1), dtype=torch.float64, device=phi.device)
    out = torch.zeros(1, dtype=torch.float64, device=phi.device)
    check(L.mg_op_residual_norm(_PREC[phi.dtype], _n(shape), *map(_p, w), _p(D), _p(f), _p(phi),
                                _p(part), _p(out), _s(phi)), "mg_op_residual_norm")
    return out


def refine(w, D, f, x, e32, c_e, c_r, shape):
    """x += c_e e in place, then e = 0; returns (x, r32 = (f - A x) / c_r, ||f - A x||)."""
    L = _lib.load()
    r32 = torch.zeros_like(e32)
    m = L.mg_op_norm_scratch(_n(shape))
    part = torch.empty(max(int(m), 1), dtype=torch.float64, device=x.device)
    out = torch.zeros(1, dtype=torch.float64, device=x.device)
    ce = torch.tensor([c_e], dtype=torch.float64, device=x.device)
    cr = torch.tensor([c_r], dtype=torch.float64, device=x.device)
    check(L.mg_op_refine(_n(shape), *map(_p, w), _p(D), _p(f), _p(x), _p(e32), _p(r32),
                         _p(ce), _p(cr), _p(part), _p(out), _s(x)), "mg_op_refine")
    return x, r32, out


def beta_grad(beta, phi, lam, h, dbeta=None, bc=0):
    if dbeta is None:
        dbeta = torch.zeros_like(beta)
    check(_lib.load().mg_op_beta_grad(_n(tuple(beta.shape)), float(h), int(bc), _p(beta),
                                      _p(phi), _p(lam), _p(dbeta), _s(beta)), "mg_op_beta_grad")
    return dbeta
