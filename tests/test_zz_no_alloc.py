"""The allocation-free residual norm (mg_op_residual_norm_noalloc) against
the existing one (mg_op_residual_norm), called through the C ABI (GPU).

It serves callers that may not allocate device memory (their memory belongs
to a pool allocator of their own, or their loop cannot take cudaMalloc's
implicit synchronisation): its partial sums live in a static device array
instead of caller scratch.  Two calls in a row must both match, since every
call reuses that array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1008_2801_gb300 import _lib, inputs
from paper_1008_2801_gb300 import ops as K

pytestmark = pytest.mark.gpu


def _noalloc(prec, shape, w, D, f, phi):
    L = _lib.load()
    fn = L.mg_op_residual_norm_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, _lib.c_int3] + [ctypes.c_void_p] * 8
    out = torch.full((1,), -1.0, dtype=torch.float64, device=phi.device)
    nz, ny, nx = shape
    p = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)  # noqa: E731
    rc = fn(prec, _lib.c_int3(nx, ny, nz), p(w[0]), p(w[1]), p(w[2]), p(D), p(f), p(phi), p(out),
            ctypes.c_void_p(torch.cuda.current_stream(phi.device).cuda_stream))
    assert rc == 0, _lib.last_error()
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_norm_matches_existing_entry_point(cuda_device, dtype):
    prec = _lib.MG_OPS_F64 if dtype == torch.float64 else _lib.MG_OPS_F32
    tol = 1e-13 if dtype == torch.float64 else 1e-5
    for shape, seed in (((70, 20, 130), 1), ((33, 17, 64), 2)):
        nz, ny, nx = shape
        d = inputs.stellar((nx, ny, nz), seed)
        beta = torch.from_numpy(d["beta"]).to(cuda_device)
        w = K.face_weights(beta, d["dx"])
        invD, D = K.inv_diag(w, shape, with_diag=True)
        if dtype == torch.float32:
            w, _ = K.round_f32(w, invD, shape)
            D = None
        f = K.put(K.level(shape, dtype, cuda_device), shape, torch.from_numpy(d["f"]))
        phi = K.put(K.level(shape, dtype, cuda_device), shape,
                    torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, shape)))
        want = K.residual_norm(w, f, phi, shape, D).item()
        for _ in range(2):   # two calls in a row share the static scratch
            got = _noalloc(prec, shape, w, D, f, phi)
            assert abs(got - want) <= tol * want, (shape, got, want)


def test_noalloc_norm_allocates_nothing(cuda_device):
    # after one warm-up call (which looks up the array's device address),
    # further calls change neither PyTorch's allocator state nor the
    # device's free memory
    shape = (40, 24, 96)
    d = inputs.stellar(shape[::-1], 5)
    beta = torch.from_numpy(d["beta"]).to(cuda_device)
    w = K.face_weights(beta, d["dx"])
    invD, D = K.inv_diag(w, shape, with_diag=True)
    f = K.put(K.level(shape, torch.float64, cuda_device), shape, torch.from_numpy(d["f"]))
    phi = K.level(shape, torch.float64, cuda_device)
    first = _noalloc(_lib.MG_OPS_F64, shape, w, D, f, phi)
    torch.cuda.synchronize()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _noalloc(_lib.MG_OPS_F64, shape, w, D, f, phi) == first
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_norm_rejects_sizes_beyond_its_scratch(cuda_device):
    L = _lib.load()
    fn = L.mg_op_residual_norm_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, _lib.c_int3] + [ctypes.c_void_p] * 8
    # one box just past the limit: 512 x 512 x 1040 cells is 16 * 64 * 65 =
    # 66560 column tiles.  Its arrays are real, full-size FP32 level arrays
    # (1.1 GB each), so that were the size check ever to come after the
    # launch, the call would return a wrong status instead of reading
    # outside its buffers
    shape = (1040, 512, 512)
    arrs = [K.level(shape, torch.float32, cuda_device) for _ in range(5)]
    out = torch.full((1,), -1.0, dtype=torch.float64, device=cuda_device)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = fn(_lib.MG_OPS_F32, _lib.c_int3(512, 512, 1040), p(arrs[0]), p(arrs[1]), p(arrs[2]),
            None, p(arrs[3]), p(arrs[4]), p(out),
            ctypes.c_void_p(torch.cuda.current_stream(cuda_device).cuda_stream))
    torch.cuda.synchronize()
    assert rc == _lib.MG_ERR_INVALID_ARG
    assert "static scratch" in _lib.last_error()
    assert out.item() == -1.0   # nothing ran
    del arrs
    torch.cuda.empty_cache()
