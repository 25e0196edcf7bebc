"""Measured choice of solver options and tile shapes per GPU, box shape(s)
and precision.

The library picks its launch shapes from models (the fused sweep's z-chunk
fills whole waves of resident CTAs; small levels go to the one-CTA coarse
kernel; a persistent launch takes as many CTAs as can be resident).  What a
model cannot know well is where the cross-overs sit on a given GPU for a
given shape.  ``tune`` searches in two stages on a synthetic stellar-profile
problem of the requested shape(s):

1. options: fused sweeps or single-colour passes, how many cells the one-CTA
   coarse kernel takes, (mixed precision) FP32 V-cycles per FP64 refinement
   step, and per-stage launches or one persistent launch per level and
   direction;
2. tile shapes for the best options: the fused FP32 sweep's tile depth
   (planes of z per CTA, ``sweep_zc``; its tile is 64 x 8 cells in x, y) and
   the persistent launches' CTAs per SM (``level_ctas``).

It keeps the fastest and caches it in a JSON file keyed by GPU name, shape
and precision (``MG_TUNE_CACHE`` or ``~/.cache/mgpu_tune.json``), with the
time of the library's defaults beside it.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

_lock = threading.Lock()

SMOOTHERS = ("auto", "passes", "fused")
COARSE = (0, 512, 2048, 8192)
INNER = (0, 2, 4)   # 0: adaptive (the default)
PERSISTENT = (False, "small", "all")
SWEEP_ZC = (0, 8, 16, 32, 64)      # 0: the library's wave model
LEVEL_CTAS = (0, 1, 2)             # 0: every resident CTA
DEFAULTS = {"smoother": "auto", "coarse_cells": 0, "inner_cycles": 0, "persistent": False,
            "sweep_zc": 0, "level_ctas": 0}


def cache_path() -> str:
    return os.environ.get("MG_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mgpu_tune.json"))


def key(gpu: str, shapes, precision: str) -> str:
    shp = ";".join("x".join(str(int(v)) for v in s) for s in shapes)
    return f"{gpu}|{precision}|{shp}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(gpu: str, shapes, precision: str):
    with _lock:
        return _load(cache_path()).get(key(gpu, shapes, precision))


def record(gpu: str, shapes, precision: str, opts: dict, ms: float, default_ms=None):
    with _lock:
        path = cache_path()
        data = _load(path)
        data[key(gpu, shapes, precision)] = {"opts": opts, "ms": ms, "default_ms": default_ms}
        _store(path, data)


def candidates(precision: str):
    """Stage 1: option sets (tile shapes at the library's models).  FP64
    levels always smooth with passes, so FP64 tries no smoother choice."""
    inner = INNER if precision == "mixed" else (0,)
    smoothers = SMOOTHERS if precision == "mixed" else ("auto",)
    for sm, cc, it, pe in itertools.product(smoothers, COARSE, inner, PERSISTENT):
        yield dict(DEFAULTS, smoother=sm, coarse_cells=cc, inner_cycles=it, persistent=pe)


def tile_candidates(opts: dict, precision: str):
    """Stage 2: tile shapes for one option set: the fused sweep's tile depth
    where FP32 levels may fuse, the persistent launches' CTAs per SM where
    they are on."""
    zcs = SWEEP_ZC if precision == "mixed" and opts["smoother"] != "passes" else (0,)
    lcs = LEVEL_CTAS if opts["persistent"] else (0,)
    for zc, lc in itertools.product(zcs, lcs):
        yield dict(opts, sweep_zc=zc, level_ctas=lc)


def tune(shapes, dx: float, precision: str = "fp64", device=None, trials: int = 2,
         tol: float = 1e-10, force: bool = False, report: bool = False):
    """Best options and tile shapes for solving boxes of these (nz, ny, nx)
    shapes; cached.  With ``report`` returns (opts, ms, default_ms)."""
    import numpy as np
    import torch

    from . import inputs
    from .solver import BatchSolver, Solver

    shapes = [tuple(int(v) for v in s) for s in shapes]
    dev = torch.device(device) if device is not None else torch.device("cuda", 0)
    gpu = torch.cuda.get_device_name(dev)
    if not force:
        hit = lookup(gpu, shapes, precision)
        if hit and set(hit["opts"]) == set(DEFAULTS):
            return (hit["opts"], hit["ms"], hit.get("default_ms")) if report else hit["opts"]
    betas, fs = [], []
    for i, (nz, ny, nx) in enumerate(shapes):
        d = inputs.stellar((nx, ny, nz), 1000 + i, dx=dx)
        betas.append(d["beta"].ravel())
        fs.append(d["f"].ravel())
    beta = torch.from_numpy(np.concatenate(betas)).to(dev)
    f = torch.from_numpy(np.concatenate(fs)).to(dev)

    def time_of(opts):
        if len(shapes) == 1:
            s = Solver(shapes[0], dx, precision=precision, device=dev, **opts)
            b, ff = beta.view(shapes[0]), f.view(shapes[0])
        else:
            s = BatchSolver(shapes, dx, precision=precision, device=dev, **opts)
            b, ff = beta, f
        try:
            s.set_beta(b)
            s.solve(ff, tol=tol)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for _ in range(trials):
                s.set_beta(b)
                s.solve(ff, tol=tol)
            ev1.record()
            torch.cuda.synchronize(dev)
            return ev0.elapsed_time(ev1) / trials
        finally:
            s.close()

    default_ms = time_of(dict(DEFAULTS))
    best, best_ms = dict(DEFAULTS), default_ms
    for opts in candidates(precision):
        if opts == DEFAULTS:
            continue
        ms = time_of(opts)
        if ms < best_ms:
            best, best_ms = opts, ms
    for opts in tile_candidates(best, precision):
        if opts == best:
            continue
        ms = time_of(opts)
        if ms < best_ms:
            best, best_ms = opts, ms
    record(gpu, shapes, precision, best, best_ms, default_ms)
    return (best, best_ms, default_ms) if report else best
