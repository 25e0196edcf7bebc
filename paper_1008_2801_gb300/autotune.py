"""Measured choice of solver options per GPU, box shape(s) and precision.

The library picks its launch shapes from a model (the fused sweep's z-chunk
fills whole waves of resident CTAs; small levels go to the one-CTA coarse
kernel).  What a model cannot know well is where the cross-overs sit on a
given GPU for a given shape: fused sweeps or single-colour passes, how many
cells the one-CTA coarse kernel should take, and (mixed precision) how many
FP32 V-cycles to run per FP64 refinement step.  ``tune`` times candidate
option sets on a synthetic stellar-profile problem of the requested shape and
keeps the fastest; results are cached in a JSON file keyed by GPU name, shape
and precision (``MG_TUNE_CACHE`` or ``~/.cache/mgpu_tune.json``).
"""
from __future__ import annotations

import itertools
import json
import os
import threading

_lock = threading.Lock()

SMOOTHERS = ("auto", "passes", "fused")
COARSE = (0, 512, 2048, 8192)
INNER = (1, 2, 3)


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


def record(gpu: str, shapes, precision: str, opts: dict, ms: float):
    with _lock:
        path = cache_path()
        data = _load(path)
        data[key(gpu, shapes, precision)] = {"opts": opts, "ms": ms}
        _store(path, data)


def candidates(precision: str):
    inner = INNER if precision == "mixed" else (0,)
    for sm, cc, it in itertools.product(SMOOTHERS, COARSE, inner):
        yield {"smoother": sm, "coarse_cells": cc, "inner_cycles": it}


def tune(shapes, dx: float, precision: str = "fp64", device=None, trials: int = 2,
         tol: float = 1e-10, force: bool = False):
    """Best options for solving boxes of these (nz, ny, nx) shapes; cached."""
    import numpy as np
    import torch

    from . import inputs
    from .solver import BatchSolver, Solver

    shapes = [tuple(int(v) for v in s) for s in shapes]
    dev = torch.device(device) if device is not None else torch.device("cuda", 0)
    gpu = torch.cuda.get_device_name(dev)
    if not force:
        hit = lookup(gpu, shapes, precision)
        if hit:
            return hit["opts"]
    betas, fs = [], []
    for i, (nz, ny, nx) in enumerate(shapes):
        d = inputs.stellar((nx, ny, nz), 1000 + i, dx=dx)
        betas.append(d["beta"].ravel())
        fs.append(d["f"].ravel())
    beta = torch.from_numpy(np.concatenate(betas)).to(dev)
    f = torch.from_numpy(np.concatenate(fs)).to(dev)
    best, best_ms = None, float("inf")
    for opts in candidates(precision):
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
            ms = ev0.elapsed_time(ev1) / trials
        finally:
            s.close()
        if ms < best_ms:
            best, best_ms = opts, ms
    record(gpu, shapes, precision, best, best_ms)
    return best
