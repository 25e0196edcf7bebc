"""Python front end of the GB300 multigrid solver (torch tensors in, out).

Tensors are float64 with shape (nz, ny, nx) (x fastest), on the solver's CUDA
device or on the host (host tensors are copied in and out inside the call).
All arithmetic runs in libmgpu.so; this module only passes pointers and the
current CUDA stream.

The equation is the variable-coefficient Poisson equation of the paper's
Sec. 1, div(beta grad phi) = f.  Each wall is Dirichlet or Neumann, chosen by
``bc``: a mask with bit w set when wall w (x-, x+, y-, y+, z-, z+) is Neumann,
bits 6-8 for periodic x, y, z axes, or a string of six letters "D"/"N"/"P" in
that order (0 or "DDDDDD": phi = 0 on every wall; "PPDDDD": periodic in x).
Non-zero wall values enter through ``bc_lift``.
"""
from __future__ import annotations

import ctypes
import warnings

import torch

from . import _lib
from ._lib import MGError, check

PRECISIONS = {"fp64": _lib.MG_FP64, "mixed": _lib.MG_MIXED}
SMOOTHERS = {"auto": 0, "passes": 1, "fused": 2}


def _stream_of(t: torch.Tensor):
    if t.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(0)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _check_tensor(t, name, numel=None, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    if t.is_cuda and device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, solver on {device}")


def _torch_allocator(device):
    """dev_alloc / dev_free callbacks that take the context's device memory
    from PyTorch's caching allocator (they must outlive the context)."""
    index = torch.device(device).index

    def alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), index)
        except RuntimeError:          # out of memory: the library reports MG_ERR_OOM
            return None

    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return _lib.DEV_ALLOC(alloc), _lib.DEV_FREE(free)


def _opts(precision, nu1, nu2, max_cycles, use_graph, smoother, coarse_cells=0, inner_cycles=0,
          full_residual=False, tma=None, krylov=False, max_norm=False, hooks=None,
          wait_limit=0, persistent=False, sweep_zc=0, level_ctas=0, fp32_setup="coarse32"):
    o = _lib.mg_opts()
    _lib.load().mg_default_opts(ctypes.byref(o))
    o.precision = PRECISIONS[precision]
    o.nu1, o.nu2, o.max_cycles = nu1, nu2, max_cycles
    o.use_graph = 1 if use_graph else 0
    o.smoother = SMOOTHERS[smoother]
    o.coarse_cells = int(coarse_cells)
    o.inner_cycles = int(inner_cycles)
    o.full_residual = 1 if full_residual else 0
    o.tma = {None: 0, True: 1, False: -1}[tma]
    o.krylov = 1 if krylov else 0
    o.max_norm = 1 if max_norm else 0
    o.wait_limit = int(wait_limit)
    o.persistent = {False: 0, True: 2, "all": 2, "small": 1}.get(persistent, persistent)
    o.sweep_zc = int(sweep_zc)
    o.level_ctas = int(level_ctas)
    o.fp32_setup = {"coarse32": 0, "rounded": 1}[fp32_setup]
    if hooks is not None:
        o.dev_alloc, o.dev_free = hooks
    return o


def bc_mask(bc) -> int:
    """Wall mask from an int (0..511) or six letters for x-, x+, y-, y+, z-, z+:
    D (Dirichlet), N (Neumann) or P (periodic; both walls of the axis)."""
    if isinstance(bc, str):
        s = bc.upper()
        if len(s) != 6 or set(s) - {"D", "N", "P"}:
            raise ValueError("bc string needs six letters D, N or P (x-, x+, y-, y+, z-, z+)")
        m = 0
        for d in range(3):
            a, b = s[2 * d], s[2 * d + 1]
            if (a == "P") != (b == "P"):
                raise ValueError("a periodic axis has P on both walls")
            if a == "P":
                m |= 1 << (6 + d)
            else:
                m |= (a == "N") << (2 * d) | (b == "N") << (2 * d + 1)
        return m
    bc = int(bc)
    if not 0 <= bc <= 511:
        raise ValueError("bc mask must be in 0..511")
    for d in range(3):
        if (bc >> (6 + d)) & 1 and (bc >> (2 * d)) & 3:
            raise ValueError("a periodic axis cannot have a Neumann wall")
    return bc


def wall_shapes(shape):
    """Shapes of the six wall arrays (x-, x+, y-, y+, z-, z+) of an (nz, ny, nx)
    box, in the packed order ``bc_lift`` reads."""
    nz, ny, nx = shape
    return [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]


def _stats_dict(s: _lib.mg_stats):
    n = max(0, min(s.cycles + 1, _lib.MG_MAX_HIST))
    return {"status": _lib.STATUS_NAMES.get(s.status, str(s.status)), "cycles": s.cycles,
            "norm_f": s.norm_f, "rel_resid0": s.rel_resid0, "rel_resid": s.rel_resid,
            "hist": list(s.hist[:n]), "t_setup_ms": s.t_setup_ms, "t_solve_ms": s.t_solve_ms,
            "rel_resid_max": s.rel_resid_max}


_SOFT = (_lib.MG_OK, _lib.MG_ERR_NOT_CONVERGED)


def _profile_dict(p: _lib.mg_profile):
    out = {"kernels": p.kernels}
    for k, name in enumerate(_lib.PROF_NAMES):
        out[name] = {"ms": p.ms[k], "launches": p.launches[k], "cells": p.cells[k]}
    return out


class Solver:
    """Multigrid solver for one (nz, ny, nx) box with cubic cells of size dx.

    precision: "fp64" (everything FP64) or "mixed" (FP32 V-cycles inside an
    FP64 iterative-refinement loop; inner_cycles: FP32 V-cycles per
    refinement step, 0 (default) adaptive, up to 8, each box leaving them
    once its update is expected to meet tol, or 1..8 fixed).  bc: wall mask
    or D/N string (see the
    module docstring).  krylov: conjugate gradients preconditioned by one
    symmetric V-cycle per iteration instead of plain V-cycles, for
    high-contrast beta (with "mixed" the V-cycle runs in FP32, CG in FP64).
    allocator: "torch" takes the context's device memory from PyTorch's
    caching allocator instead of cudaMalloc.  tma: None (default) or True
    feeds the FP32 fused sweeps by the Tensor Memory Accelerator where a
    level fits, False forces plain loads (same result).  wait_limit: polls of a bounded
    device wait before it gives up (mg_opts.wait_limit; 0 default, -1 gives
    up at once).  persistent: one persistent launch per level and direction
    (mg_opts.persistent: True or "all" on every level smoothed with passes,
    "small" on those whose stages fit in one wave of resident CTAs); sweep_zc, level_ctas: tile depth of the fused FP32
    sweep and CTAs per SM of the persistent launches (0: the library's
    model; see mg_opts and ``autotune``).  fp32_setup ("mixed"): "coarse32"
    (default) rounds the finest level's FP64 weights to FP32 and sets the
    coarser levels up in FP32 only (averages of the finer FP32 weights);
    "rounded" sets every level up in FP64 and rounds it (mg_opts.fp32_setup).
    Not thread-safe.
    """

    def __init__(self, shape, dx, precision="fp64", nu1=2, nu2=2, max_cycles=100,
                 use_graph=True, smoother="auto", device=None, coarse_cells=0, inner_cycles=0,
                 full_residual=False, tma=None, bc=0, krylov=False, max_norm=False,
                 allocator=None, wait_limit=0, persistent=False, sweep_zc=0, level_ctas=0,
                 fp32_setup="coarse32"):
        L = _lib.load()
        self.shape = tuple(int(v) for v in shape)
        nz, ny, nx = self.shape
        self.dx = float(dx)
        self.precision = precision
        self.bc = bc_mask(bc)
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self._h = ctypes.c_void_p()
        self._hooks = _torch_allocator(self.device) if allocator == "torch" else None
        o = _opts(precision, nu1, nu2, max_cycles, use_graph, smoother, coarse_cells, inner_cycles,
                  full_residual, tma, krylov, max_norm, self._hooks, wait_limit, persistent,
                  sweep_zc, level_ctas, fp32_setup)
        with torch.cuda.device(self.device):
            check(L.mg_create(ctypes.byref(self._h), _lib.c_int3(nx, ny, nz), self.dx, self.bc,
                              ctypes.byref(o)), "mg_create")
        self._beta = None

    @property
    def numel(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def levels(self):
        n = ctypes.c_int()
        dims = (ctypes.c_int * 96)()
        check(_lib.load().mg_levels(self._h, ctypes.byref(n), dims), "mg_levels")
        return [(dims[3 * i + 2], dims[3 * i + 1], dims[3 * i]) for i in range(n.value)]

    def smoother_kind(self, level=0):
        """How level `level` is smoothed (mg_smoother_kind): "passes",
        "fused" (plain-load sweeps) or "fused_tma"."""
        k = ctypes.c_int()
        check(_lib.load().mg_smoother_kind(self._h, int(level), ctypes.byref(k)),
              "mg_smoother_kind")
        return ("passes", "fused", "fused_tma")[k.value]

    def set_beta(self, beta: torch.Tensor):
        _check_tensor(beta, "beta", self.numel, self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().mg_set_beta(self._h, _ptr(beta), _stream_of(beta)), "mg_set_beta")
        self._beta = beta

    def bc_lift(self, values, f: torch.Tensor, out: torch.Tensor | None = None):
        """f minus the lift of non-zero wall values (mg_bc_lift).  values: the
        six wall arrays (x-, x+, y-, y+, z-, z+; see ``wall_shapes``) or one
        packed float64 tensor; each is phi on a Dirichlet wall, the outward flux
        beta dphi/dn on a Neumann wall."""
        if not isinstance(values, torch.Tensor):
            values = torch.cat([torch.as_tensor(v, dtype=torch.float64).reshape(-1)
                                for v in values])
        nz, ny, nx = self.shape
        values = values.to(device=self.device, dtype=torch.float64).contiguous()
        _check_tensor(values, "values", 2 * (ny * nz + nz * nx + ny * nx), self.device)
        _check_tensor(f, "f", self.numel, self.device)
        if not f.is_cuda:
            raise ValueError("f must be on the solver's device")
        if out is None:
            out = torch.empty_like(f)
        _check_tensor(out, "out", self.numel, self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().mg_bc_lift(self._h, _ptr(values), _ptr(f), _ptr(out),
                                         _stream_of(f)), "mg_bc_lift")
        return out

    def solve(self, f: torch.Tensor, phi: torch.Tensor | None = None, tol: float = 1e-10,
              raise_on=("invalid_arg", "cuda", "oom", "nonfinite", "diverged", "timeout",
                        "unsupported"), bc_values=None, zero_guess: bool | None = None):
        """Solve A phi = f; returns (phi, stats).  phi (if given) is the initial
        guess and is overwritten; with zero_guess (the default when phi is not
        given) the iteration starts from 0 and phi is output only.  A leading
        batch dimension solves several right-hand sides with the same beta.
        bc_values (one box): non-zero wall values, lifted into f first (see
        ``bc_lift``)."""
        _check_tensor(f, "f", device=self.device)
        if bc_values is not None:
            if f.numel() != self.numel:
                raise ValueError("bc_values need a single right-hand side")
            f = self.bc_lift(bc_values, f.reshape(self.shape))
        if f.numel() % self.numel:
            raise ValueError("f must hold whole boxes")
        nrhs = f.numel() // self.numel
        if zero_guess is None:
            zero_guess = phi is None
        if phi is None:
            phi = torch.empty_like(f)
        _check_tensor(phi, "phi", f.numel(), self.device)
        st = (_lib.mg_stats * nrhs)()
        L = _lib.load()
        flags = _lib.MG_ZERO_GUESS if zero_guess else 0
        with torch.cuda.device(self.device):
            rc = L.mg_solve_ex(self._h, nrhs, _ptr(f), _ptr(phi), float(tol), flags, st,
                               _stream_of(f))
        stats = [_stats_dict(s) for s in st]
        if _lib.STATUS_NAMES.get(rc) in raise_on:
            raise MGError(rc, "mg_solve")
        return phi, (stats[0] if nrhs == 1 else stats)

    def adjoint(self, phi: torch.Tensor, g: torch.Tensor, tol: float = 1e-10,
                dbeta: torch.Tensor | None = None, stats: bool = False):
        """Returns (dL/df = lambda, dL/dbeta) for dL/dphi = g (see mg_adjoint),
        and the adjoint solve's stats (a list for several right-hand sides)
        as a third item when ``stats`` is set."""
        _check_tensor(phi, "phi", device=self.device)
        _check_tensor(g, "g", phi.numel(), self.device)
        nrhs = phi.numel() // self.numel
        lam = torch.empty_like(g)
        if dbeta is None:
            dbeta = torch.zeros(self.shape, dtype=torch.float64, device=phi.device)
        _check_tensor(dbeta, "dbeta", self.numel, self.device)
        st = (_lib.mg_stats * nrhs)()
        with torch.cuda.device(self.device):
            rc = _lib.load().mg_adjoint(self._h, nrhs, _ptr(phi), _ptr(g), _ptr(lam),
                                        _ptr(dbeta), float(tol), st, _stream_of(phi))
        if rc not in _SOFT:
            raise MGError(rc, "mg_adjoint")
        if stats:
            sd = [_stats_dict(s) for s in st]
            return lam, dbeta, (sd[0] if nrhs == 1 else sd)
        return lam, dbeta

    # ---- projection steps around the solve (the velocity constraint)

    def _vel_check(self, u, v, w):
        nz, ny, nx = self.shape
        for t, nm, shp in ((u, "u", (nz, ny, nx + 1)), (v, "v", (nz, ny + 1, nx)),
                           (w, "w", (nz + 1, ny, nx))):
            _check_tensor(t, nm, shp[0] * shp[1] * shp[2], self.device)
            if not t.is_cuda:
                raise ValueError(f"{nm} must be on the solver's device")

    def project_rhs(self, u, v, w, S=None):
        """f = div(u, v, w) - S (face velocities in natural layouts)."""
        self._vel_check(u, v, w)
        f = torch.empty(self.shape, dtype=torch.float64, device=u.device)
        if S is not None:
            _check_tensor(S, "S", self.numel, self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().mg_project_rhs(self._h, _ptr(u), _ptr(v), _ptr(w),
                                             _ptr(S) if S is not None else None, _ptr(f),
                                             _stream_of(u)), "mg_project_rhs")
        return f

    def project_correct(self, phi, u, v, w):
        """u, v, w -= beta_face grad(phi), in place."""
        self._vel_check(u, v, w)
        _check_tensor(phi, "phi", self.numel, self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().mg_project_correct(self._h, _ptr(phi), _ptr(u), _ptr(v), _ptr(w),
                                                 _stream_of(u)), "mg_project_correct")
        return u, v, w

    def project(self, u, v, w, S=None, tol=1e-10):
        """Make div(u, v, w) = S: form f, solve div(beta grad phi) = f, correct
        the face velocities in place.  Returns (phi, stats)."""
        f = self.project_rhs(u, v, w, S)
        phi, st = self.solve(f, tol=tol)
        self.project_correct(phi, u, v, w)
        return phi, st

    def profile(self, on: bool = True):
        """Record per-stage device times (CUDA events inside the V-cycle graph)."""
        check(_lib.load().mg_profile_enable(self._h, 1 if on else 0), "mg_profile_enable")

    def read_profile(self, reset: bool = False):
        p = _lib.mg_profile()
        check(_lib.load().mg_profile_read(self._h, ctypes.byref(p), 1 if reset else 0),
              "mg_profile_read")
        return _profile_dict(p)

    def close(self):
        if self._h:
            _lib.load().mg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Independent boxes of uneven size solved together (one launch per stage
    over the tiles of every active box).  shapes: list of (nz, ny, nx); arrays
    are packed back to back in box order (see ``pack``/``unpack``).
    persistent: each level smoothed with passes runs as one persistent
    launch per direction over all boxes (mg_opts.persistent; True/"all" or
    "small", as for ``Solver``); fp32_setup as for ``Solver``."""

    def __init__(self, shapes, dx, precision="fp64", nu1=2, nu2=2, max_cycles=100,
                 use_graph=True, smoother="auto", device=None, coarse_cells=0, inner_cycles=0,
                 full_residual=False, tma=None, bc=0, krylov=False, max_norm=False,
                 allocator=None, wait_limit=0, persistent=False, sweep_zc=0, level_ctas=0,
                 fp32_setup="coarse32"):
        L = _lib.load()
        self.bc = bc_mask(bc)
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        nb = len(self.shapes)
        dxs = [float(dx)] * nb if isinstance(dx, (int, float)) else [float(v) for v in dx]
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        n = (ctypes.c_int * (3 * nb))(*[v for s in self.shapes for v in (s[2], s[1], s[0])])
        d = (ctypes.c_double * nb)(*dxs)
        self._h = ctypes.c_void_p()
        self._hooks = _torch_allocator(self.device) if allocator == "torch" else None
        o = _opts(precision, nu1, nu2, max_cycles, use_graph, smoother, coarse_cells, inner_cycles,
                  full_residual, tma, krylov, max_norm, self._hooks, wait_limit, persistent,
                  sweep_zc, level_ctas, fp32_setup)
        with torch.cuda.device(self.device):
            check(L.mg_batch_create(ctypes.byref(self._h), nb, n, d, self.bc, ctypes.byref(o)),
                  "mg_batch_create")
        self.sizes = [s[0] * s[1] * s[2] for s in self.shapes]
        self.total = sum(self.sizes)

    def pack(self, arrays):
        return torch.cat([a.reshape(-1) for a in arrays])

    def unpack(self, packed):
        out, o = [], 0
        for s, k in zip(self.shapes, self.sizes):
            out.append(packed[o:o + k].view(s))
            o += k
        return out

    def set_beta(self, beta_packed: torch.Tensor):
        _check_tensor(beta_packed, "beta", self.total, self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().mg_batch_set_beta(self._h, _ptr(beta_packed),
                                                _stream_of(beta_packed)), "mg_batch_set_beta")
        self._beta = beta_packed

    def solve(self, f_packed, phi_packed=None, tol=1e-10, zero_guess=None):
        """Returns (phi_packed, per-box stats); zero_guess as in Solver.solve."""
        _check_tensor(f_packed, "f", self.total, self.device)
        if zero_guess is None:
            zero_guess = phi_packed is None
        if phi_packed is None:
            phi_packed = torch.empty_like(f_packed)
        _check_tensor(phi_packed, "phi", self.total, self.device)
        st = (_lib.mg_stats * len(self.shapes))()
        flags = _lib.MG_ZERO_GUESS if zero_guess else 0
        with torch.cuda.device(self.device):
            rc = _lib.load().mg_solve_batched_ex(self._h, _ptr(f_packed), _ptr(phi_packed),
                                                 float(tol), flags, st, _stream_of(f_packed))
        if rc not in _SOFT:
            raise MGError(rc, "mg_solve_batched")
        return phi_packed, [_stats_dict(s) for s in st]

    def profile(self, on: bool = True):
        check(_lib.load().mg_batch_profile_enable(self._h, 1 if on else 0),
              "mg_batch_profile_enable")

    def read_profile(self, reset: bool = False):
        p = _lib.mg_profile()
        check(_lib.load().mg_batch_profile_read(self._h, ctypes.byref(p), 1 if reset else 0),
              "mg_batch_profile_read")
        return _profile_dict(p)

    def close(self):
        if self._h:
            _lib.load().mg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def level_intersections(los, ns, brute=False):
    """Ghost-exchange records of boxes with lower corners los[b] = (i, j, k)
    and dims ns[b] = (nx, ny, nz) (host only, no device work): a list of
    dicts dst, src, d (patch origin in dst), s (in src), e (extents)."""
    L = _lib.load()
    nb = len(los)
    lo = (ctypes.c_int * (3 * nb))(*[int(v) for c in los for v in c])
    n = (ctypes.c_int * (3 * nb))(*[int(v) for c in ns for v in c])
    cnt = ctypes.c_int()
    check(L.mg_level_intersections(nb, lo, n, 1 if brute else 0, ctypes.byref(cnt), None, 0),
          "mg_level_intersections")
    buf = (ctypes.c_int * (11 * max(cnt.value, 1)))()
    check(L.mg_level_intersections(nb, lo, n, 1 if brute else 0, ctypes.byref(cnt), buf,
                                   cnt.value), "mg_level_intersections")
    out = []
    for q in range(cnt.value):
        v = buf[11 * q:11 * q + 11]
        out.append({"dst": v[0], "src": v[1], "d": tuple(v[2:5]), "s": tuple(v[5:8]),
                    "e": tuple(v[8:11])})
    return out


class LevelSolver:
    """The boxes of one level solved as one domain (mg_level): box b covers
    cells los[b] .. los[b] + shape - 1 of a common index space, los[b] given
    as (i, j, k) (x first) and shapes[b] as (nz, ny, nx) like every array
    here.  Arrays are packed back to back in box order (see ``pack`` /
    ``unpack``).  Interfaces between boxes are interior faces; the union's
    boundary has Dirichlet walls (phi = 0)."""

    def __init__(self, los, shapes, dx, precision="fp64", nu1=2, nu2=2, max_cycles=100,
                 use_graph=True, device=None, inner_cycles=0, persistent=False, wait_limit=0):
        L = _lib.load()
        self.los = [tuple(int(v) for v in c) for c in los]
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        nb = len(self.shapes)
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        lo = (ctypes.c_int * (3 * nb))(*[v for c in self.los for v in c])
        n = (ctypes.c_int * (3 * nb))(*[v for s in self.shapes for v in (s[2], s[1], s[0])])
        self._h = ctypes.c_void_p()
        o = _opts(precision, nu1, nu2, max_cycles, use_graph, "passes", 0, inner_cycles,
                  wait_limit=wait_limit, persistent=persistent)
        with torch.cuda.device(self.device):
            check(L.mg_level_create(ctypes.byref(self._h), nb, lo, n, float(dx), 0,
                                    ctypes.byref(o)), "mg_level_create")
        self.sizes = [s[0] * s[1] * s[2] for s in self.shapes]
        self.total = sum(self.sizes)

    def pack(self, arrays):
        return torch.cat([torch.as_tensor(a).reshape(-1) for a in arrays])

    def unpack(self, packed):
        out, o = [], 0
        for s, k in zip(self.shapes, self.sizes):
            out.append(packed[o:o + k].view(s))
            o += k
        return out

    def levels(self):
        n = ctypes.c_int()
        check(_lib.load().mg_level_levels(self._h, ctypes.byref(n)), "mg_level_levels")
        return n.value

    def set_beta(self, beta_packed: torch.Tensor):
        _check_tensor(beta_packed, "beta", self.total, self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().mg_level_set_beta(self._h, _ptr(beta_packed),
                                                _stream_of(beta_packed)), "mg_level_set_beta")

    def solve(self, f_packed, phi_packed=None, tol=1e-10, zero_guess=None):
        """Returns (phi_packed, stats) with the union's residual history;
        zero_guess as in Solver.solve."""
        _check_tensor(f_packed, "f", self.total, self.device)
        if zero_guess is None:
            zero_guess = phi_packed is None
        if phi_packed is None:
            phi_packed = torch.empty_like(f_packed)
        _check_tensor(phi_packed, "phi", self.total, self.device)
        st = (_lib.mg_stats * len(self.shapes))()
        flags = _lib.MG_ZERO_GUESS if zero_guess else 0
        with torch.cuda.device(self.device):
            rc = _lib.load().mg_level_solve_ex(self._h, _ptr(f_packed), _ptr(phi_packed),
                                               float(tol), flags, st, _stream_of(f_packed))
        if rc not in _SOFT:
            raise MGError(rc, "mg_level_solve")
        return phi_packed, _stats_dict(st[0])

    def profile(self, on: bool = True):
        check(_lib.load().mg_level_profile_enable(self._h, 1 if on else 0),
              "mg_level_profile_enable")

    def read_profile(self, reset: bool = False):
        p = _lib.mg_profile()
        check(_lib.load().mg_level_profile_read(self._h, ctypes.byref(p), 1 if reset else 0),
              "mg_level_profile_read")
        return _profile_dict(p)

    def close(self):
        if self._h:
            _lib.load().mg_level_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MGSolve(torch.autograd.Function):
    """phi = A(beta)^{-1} f as a differentiable op.

    Forward: set beta, solve (f may carry a leading right-hand-side dim).
    Backward: the adjoint solve A lambda = dL/dphi gives dL/df = lambda and
    the face products give dL/dbeta (summed over right-hand sides).


    A solve or adjoint solve that stops short of tol (cycle cap or stalled
    residual) raises MGError when ``strict`` is set on the solver
    (``solver.strict = True``); otherwise it emits a RuntimeWarning naming the
    residual reached, so that a gradient is never returned silently from an
    unconverged solve.  Hard failures (non-finite values, divergence, CUDA
    errors) always raise.
    """

    @staticmethod
    def forward(ctx, f, beta, solver: Solver, tol: float = 1e-10):
        solver.set_beta(beta)
        phi, st = solver.solve(f.contiguous(), tol=tol)
        _unconverged(solver, "forward solve", st)
        ctx.solver, ctx.tol = solver, tol
        ctx.save_for_backward(phi, beta)
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        phi, beta = ctx.saved_tensors
        solver = ctx.solver
        if solver._beta is not beta:
            solver.set_beta(beta)
        lam, dbeta, st = solver.adjoint(phi, grad_phi.contiguous(), tol=ctx.tol, stats=True)
        _unconverged(solver, "adjoint solve", st)
        return lam, dbeta, None, None


def _unconverged(solver, what, stats):
    """Warn (or raise, with solver.strict) if any right-hand side of a solve
    did not reach its tolerance."""
    stats = stats if isinstance(stats, list) else [stats]
    bad = [s for s in stats if s["status"] != "ok"]
    if not bad:
        return
    worst = max(s["rel_resid"] for s in bad)
    msg = (f"MGSolve {what}: {len(bad)} of {len(stats)} right-hand sides stopped at "
           f"status {bad[0]['status']} (relative residual {worst:.3e})")
    if getattr(solver, "strict", False):
        raise MGError(_lib.MG_ERR_NOT_CONVERGED, msg)
    warnings.warn(msg, RuntimeWarning, stacklevel=3)


_cache: dict = {}


def solve(f: torch.Tensor, beta: torch.Tensor, dx: float, tol: float = 1e-10,
          precision: str = "fp64", bc=0):
    """Functional form: phi with div(beta grad phi) = f (differentiable in f
    and beta).  Solvers are cached per (shape, dx, precision, walls, device)."""
    shape = tuple(beta.shape)
    key = (shape, float(dx), precision, bc_mask(bc), f.device)
    s = _cache.get(key)
    if s is None:
        s = _cache[key] = Solver(shape, dx, precision=precision, device=f.device, bc=bc)
    return MGSolve.apply(f, beta, s, tol)


def slab_plan(shape, nslab):
    """Host only: (z0, gather_level) of an (nz, ny, nx) box split into nslab
    slabs (mg_slab_plan): slab r holds planes z0[r] .. z0[r+1]-1; levels below
    gather_level are smoothed slab by slab."""
    nz, ny, nx = (int(v) for v in shape)
    z0 = (ctypes.c_int * (nslab + 1))()
    g = ctypes.c_int()
    check(_lib.load().mg_slab_plan(_lib.c_int3(nx, ny, nz), int(nslab), z0, ctypes.byref(g)),
          "mg_slab_plan")
    return list(z0), g.value


def slab_halo(shape, nslab, level):
    """Host only: the halo copies of one slab level (mg_slab_halo), as dicts
    src, src_k, dst, dst_k (local plane indices; -1 and the slab's thickness
    are its guard planes)."""
    nz, ny, nx = (int(v) for v in shape)
    L = _lib.load()
    n = ctypes.c_int()
    check(L.mg_slab_halo(_lib.c_int3(nx, ny, nz), int(nslab), int(level), ctypes.byref(n),
                         None, 0), "mg_slab_halo")
    buf = (ctypes.c_int * (4 * max(n.value, 1)))()
    check(L.mg_slab_halo(_lib.c_int3(nx, ny, nz), int(nslab), int(level), ctypes.byref(n), buf,
                         n.value), "mg_slab_halo")
    return [{"src": buf[4 * i], "src_k": buf[4 * i + 1], "dst": buf[4 * i + 2],
             "dst_k": buf[4 * i + 3]} for i in range(n.value)]


class SlabSolver:
    """One (nz, ny, nx) box split in z into ``nslab`` equal slabs, slab r on
    CUDA device ``devices[r]`` (mg_slab_*): the levels down to the gather
    level are smoothed slab by slab with halo exchanges of one plane, the
    rest of the V-cycle runs on ``devices[0]``.  FP64 V-cycles.  Arrays are
    full-box tensors; each slab's part is a view when the tensor already sits
    on that slab's device, else a copy."""

    def __init__(self, shape, dx, nslab, devices=None, nu1=2, nu2=2, max_cycles=100):
        L = _lib.load()
        self.shape = tuple(int(v) for v in shape)
        nz, ny, nx = self.shape
        self.nslab = int(nslab)
        if devices is None:
            devices = [torch.cuda.current_device()] * self.nslab
        self.devices = [torch.device("cuda", torch.device("cuda", d).index
                                     if isinstance(d, int) else torch.device(d).index)
                        for d in devices]
        if len(self.devices) != self.nslab:
            raise ValueError("one device per slab")
        self.z0, self.gather = slab_plan(self.shape, self.nslab)
        o = _opts("fp64", nu1, nu2, max_cycles, False, "passes")
        devs = (ctypes.c_int * self.nslab)(*[d.index for d in self.devices])
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.devices[0]):
            check(L.mg_slab_create(ctypes.byref(self._h), _lib.c_int3(nx, ny, nz), float(dx),
                                   self.nslab, devs, ctypes.byref(o)), "mg_slab_create")

    def _parts(self, t, name):
        _check_tensor(t, name, self.shape[0] * self.shape[1] * self.shape[2])
        t = t.reshape(self.shape)
        out = []
        for r, d in enumerate(self.devices):
            part = t[self.z0[r]:self.z0[r + 1]]
            out.append(part if part.device == d else part.to(d).contiguous())
        return out

    def _ptrs(self, parts):
        return (ctypes.c_void_p * self.nslab)(*[p.data_ptr() for p in parts])

    def _sync(self):
        for d in set(self.devices):
            torch.cuda.synchronize(d)

    def set_beta(self, beta: torch.Tensor):
        parts = self._parts(beta, "beta")
        self._sync()
        check(_lib.load().mg_slab_set_beta(self._h, self._ptrs(parts)), "mg_slab_set_beta")

    def solve(self, f: torch.Tensor, phi: torch.Tensor | None = None, tol: float = 1e-10,
              zero_guess: bool | None = None):
        """Returns (phi, stats); phi is a full-box tensor on devices[0]."""
        if zero_guess is None:
            zero_guess = phi is None
        if phi is None:
            phi = torch.zeros(self.shape, dtype=torch.float64, device=self.devices[0])
        fp = self._parts(f, "f")
        pp = self._parts(phi, "phi")
        self._sync()
        st = _lib.mg_stats()
        flags = _lib.MG_ZERO_GUESS if zero_guess else 0
        rc = _lib.load().mg_slab_solve(self._h, self._ptrs(fp), self._ptrs(pp), float(tol), flags,
                                       ctypes.byref(st))
        if rc not in _SOFT:
            raise MGError(rc, "mg_slab_solve")
        out = phi.reshape(self.shape)
        for r, p in enumerate(pp):
            dst = out[self.z0[r]:self.z0[r + 1]]
            if p.data_ptr() != dst.data_ptr():
                dst.copy_(p)
        return out, _stats_dict(st)

    def close(self):
        if self._h:
            _lib.load().mg_slab_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
