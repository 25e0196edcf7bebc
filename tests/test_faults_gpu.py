"""Failure paths on the GPU, made without faulting it (GPU).

- A bounded device wait that runs out: the TMA sweep's tile-copy waits are
  given no polls at all (mg_opts.wait_limit = -1), so every wait gives up
  at once; each CTA still drains the copies it issued before it exits.  The
  solve must return MG_ERR_TIMEOUT, and the device and the library must
  stay usable afterwards.
- An allocator that fails on the host (mg_opts.dev_alloc returning NULL at
  its first, second or third call) -> MG_ERR_OOM, with every block that
  was handed out given back.
- An autograd solve that stops short of its tolerance warns (or raises with
  ``strict``) instead of returning a gradient silently.
"""
import ctypes
import warnings

import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import MGError, MGSolve, Solver, _lib, inputs

pytestmark = pytest.mark.gpu


def _dev(a, dev):
    return torch.from_numpy(np.array(a, order="C", copy=True)).to(dev)


def test_tma_wait_that_runs_out_returns_timeout(cuda_device):
    # nx = 128 and ny = 16 hold a whole TMA copy box (72 x 12)
    d = inputs.stellar((128, 16, 32), 3)
    beta, f = _dev(d["beta"], cuda_device), _dev(d["f"], cuda_device)
    with Solver(f.shape, d["dx"], precision="mixed", smoother="fused", tma=True,
                wait_limit=-1, max_cycles=3, device=cuda_device) as s:
        s.set_beta(beta)
        for _ in range(2):   # the error word is cleared after each report
            with pytest.raises(MGError) as ei:
                s.solve(f, tol=1e-10)
            assert ei.value.name == "timeout"
            assert "gave up" in _lib.last_error() or "status 7" in _lib.last_error()
    torch.cuda.synchronize(cuda_device)   # the context is intact
    # the same problem with the default bound solves, bitwise as the plain sweep
    out = {}
    for tma in (True, False):
        with Solver(f.shape, d["dx"], precision="mixed", smoother="fused", tma=tma,
                    device=cuda_device) as s:
            s.set_beta(beta)
            phi, st = s.solve(f, tol=1e-10)
            assert st["status"] == "ok"
            out[tma] = phi
    assert torch.equal(out[True], out[False])
    ref, _ = O.solve(d["beta"], d["f"], d["dx"], tol=1e-13)
    phi = out[True].cpu().numpy()
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)


def test_wait_limit_is_validated(cuda_device):
    with pytest.raises(MGError) as ei:
        Solver((8, 8, 8), 0.125, wait_limit=-2, device=cuda_device)
    assert ei.value.name == "invalid_arg"


class _FailingAllocator:
    """dev_alloc / dev_free hooks backed by PyTorch's caching allocator that
    return NULL at the fail_at-th request."""

    def __init__(self, device, fail_at):
        self.index = torch.device(device).index
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()
        self.alloc = _lib.DEV_ALLOC(self._alloc)
        self.free = _lib.DEV_FREE(self._free)

    def _alloc(self, nbytes, user):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), self.index)
        self.live.add(p)
        return p

    def _free(self, ptr, user):
        self.live.discard(ptr)
        torch.cuda.caching_allocator_delete(ptr)


@pytest.mark.parametrize("fail_at", [1, 2, 3])
def test_failing_allocator_returns_oom(cuda_device, fail_at):
    L = _lib.load()
    hook = _FailingAllocator(cuda_device, fail_at)
    o = _lib.mg_opts()
    L.mg_default_opts(ctypes.byref(o))
    o.dev_alloc, o.dev_free = hook.alloc, hook.free
    h = ctypes.c_void_p()
    with torch.cuda.device(cuda_device):
        rc = L.mg_create(ctypes.byref(h), _lib.c_int3(48, 40, 32), 1 / 48, 0, ctypes.byref(o))
    if hook.calls < fail_at:
        # the context needed fewer blocks than fail_at: it must be whole
        assert rc == _lib.MG_OK
        L.mg_destroy(h)
    else:
        assert rc == _lib.MG_ERR_OOM, _lib.last_error()
        assert not h.value
    assert not hook.live   # every block handed out was given back
    # the device is usable after the failure
    with Solver((8, 8, 8), 0.125, device=cuda_device) as s:
        s.set_beta(torch.ones((8, 8, 8), dtype=torch.float64, device=cuda_device))
        _, st = s.solve(torch.ones((8, 8, 8), dtype=torch.float64, device=cuda_device))
        assert st["status"] == "ok"


def test_autograd_warns_on_an_unconverged_solve(cuda_device):
    d = inputs.stellar(16, 4)
    beta = _dev(d["beta"], cuda_device).requires_grad_(True)
    f = _dev(d["f"], cuda_device).requires_grad_(True)
    s = Solver((16, 16, 16), d["dx"], max_cycles=1, device=cuda_device)
    with pytest.warns(RuntimeWarning, match="not_converged"):
        phi = MGSolve.apply(f, beta, s, 1e-12)
    with pytest.warns(RuntimeWarning, match="adjoint solve"):
        (0.5 * (phi ** 2).sum()).backward()
    s.strict = True
    with pytest.raises(MGError):
        MGSolve.apply(f, beta, s, 1e-12)
    # a converged solve is silent
    s2 = Solver((16, 16, 16), d["dx"], device=cuda_device)
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        phi = MGSolve.apply(f, beta, s2, 1e-10)
        (0.5 * (phi ** 2).sum()).backward()
    s.close()
    s2.close()
