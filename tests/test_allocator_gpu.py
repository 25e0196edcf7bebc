"""Caller-provided device memory (mg_opts.dev_alloc / dev_free): a context
whose arena, descriptors and staging buffers come from PyTorch's caching
allocator solves bit for bit like one on cudaMalloc, and its memory goes back
to that allocator at destroy."""
import numpy as np
import pytest
import torch

from paper_1008_2801_gb300 import BatchSolver, Solver, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_torch_allocator_solves_identically(cuda_device, precision):
    d = inputs.stellar((48, 32, 40), 80)
    shape = d["f"].shape
    beta, f = torch.from_numpy(d["beta"]), torch.from_numpy(d["f"])
    out = []
    for allocator in (None, "torch"):
        torch.cuda.synchronize(cuda_device)
        before = torch.cuda.memory_allocated(cuda_device)
        s = Solver(shape, d["dx"], precision=precision, device=cuda_device, allocator=allocator)
        held = torch.cuda.memory_allocated(cuda_device) - before
        s.set_beta(beta.to(cuda_device))
        phi_d, st = s.solve(f.to(cuda_device))
        phi_h, _ = s.solve(f.clone())                 # host buffers: staging through the hook
        assert st["status"] == "ok" and torch.equal(phi_h, phi_d.cpu())
        out.append((phi_d.cpu(), held))
        s.close()
        torch.cuda.synchronize(cuda_device)
        if allocator == "torch":
            assert held > 8 * np.prod(shape)          # the arena came from torch
            assert torch.cuda.memory_allocated(cuda_device) == before
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == 0


def test_torch_allocator_batched(cuda_device):
    shapes = [(16, 16, 24), (32, 16, 16)]
    cases = [inputs.stellar(sh[::-1], 81 + i) for i, sh in enumerate(shapes)]
    res = []
    for allocator in (None, "torch"):
        with BatchSolver(shapes, 1.0 / 32, device=cuda_device, allocator=allocator) as b:
            b.set_beta(b.pack([torch.from_numpy(c["beta"]) for c in cases]).to(cuda_device))
            phi, st = b.solve(b.pack([torch.from_numpy(c["f"]) for c in cases]).to(cuda_device))
            res.append(phi.cpu())
    assert torch.equal(res[0], res[1])
