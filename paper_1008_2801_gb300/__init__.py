"""GB300-native geometric multigrid for the cell-centred variable-coefficient
Poisson equation div(beta grad phi) = f (the linear solve of each MAESTRO
time step, paper Sec. 1), with hand-written sm_103a CUDA kernels behind a C
ABI (include/mg.h, include/mg_ops.h).

Importing the package loads nothing; the CUDA library is loaded (and built
from source if needed) on first use, and a missing or unbuildable library is
an error, never a fallback.
"""
from __future__ import annotations

__all__ = ["Solver", "BatchSolver", "LevelSolver", "SlabSolver", "MGSolve", "solve", "bc_mask",
           "wall_shapes", "level_intersections", "slab_plan", "slab_halo", "MGError", "build",
           "inputs", "ops"]


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def __getattr__(name):
    if name in ("Solver", "BatchSolver", "LevelSolver", "SlabSolver", "MGSolve", "solve",
                "bc_mask", "wall_shapes", "level_intersections", "slab_plan", "slab_halo"):
        from . import solver
        return getattr(solver, name)
    if name == "MGError":
        from ._lib import MGError
        return MGError
    if name in ("inputs", "ops"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
