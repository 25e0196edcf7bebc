"""Per-stage parity of the CUDA kernels with the CPU oracle (GPU).

Every stage is called through the C ABI (include/mg_ops.h) on the same
seeded inputs the oracle gets, and compared element by element.

Tolerances, from the arithmetic: each output is a sum of at most 8 products
(plus one multiply by the reciprocal of the diagonal, stored or computed), so its rounding error is below
about 10 u * (sum of |terms|), u = 2^-53 in FP64 and 2^-24 in FP32.  The
tests allow 1e-13 (FP64) and 1e-5 (FP32) times that term scale, i.e. 100x
headroom; the FP32 kernels are compared with the FP64 oracle.

Shapes span several tiles with ragged tails: tiles are 32 x 8 cells (64 x 8
for the fused sweep, which also cuts z into chunks of 32 planes).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import inputs
from paper_1008_2801_gb300 import ops as K

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (3, 2, 5), (5, 7, 9), (20, 17, 33), (70, 20, 130)]
EVEN = [(2, 2, 2), (4, 6, 8), (18, 10, 34), (66, 20, 130)]


def _case(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    r = np.random.default_rng(seed + 100)
    phi = r.uniform(-1, 1, shape)
    return d["beta"], d["f"], phi, d["dx"]


def _t(a, dev, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


def _level(shape, data, dev, dtype=torch.float64, kind="cell"):
    return K.put(K.level(shape, dtype, dev), shape, _t(data, dev, dtype), kind)


def _weights(beta, h, shape, dev, dtype=torch.float64):
    w = K.face_weights(_t(beta, dev), h)
    if dtype == torch.float32:
        invD = K.inv_diag(w, shape)
        w32, inv32 = K.round_f32(w, invD, shape)
        return w32, inv32
    return w, K.inv_diag(w, shape)


def _tol(dtype):
    return 1e-13 if dtype == torch.float64 else 1e-5


@pytest.mark.parametrize("shape", SHAPES)
def test_face_weights_and_inverse_diagonal(cuda_device, shape):
    beta, _, _, h = _case(shape, 1)
    w = K.face_weights(_t(beta, cuda_device), h)
    faces = O.face_beta(beta)
    for wt, fo, kind in zip(w, faces, "xyz"):
        got = K.get(wt, shape, kind).cpu().numpy()
        want = fo / h ** 2
        assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-15
    invD = K.get(K.inv_diag(w, shape), shape).cpu().numpy()
    bx, by, bz = faces
    D = (bx[:, :, :-1] + bx[:, :, 1:] + by[:, :-1, :] + by[:, 1:, :] + bz[:-1] + bz[1:]) / h ** 2
    assert np.max(np.abs(invD * D - 1.0)) <= 1e-14


def test_inverse_diagonal_over_the_fp64_range(cuda_device):
    # 1/D without an FP64 division (FP32 seed, one cubic Newton step): within
    # one ulp of the correctly rounded reciprocal, and equal to it but for
    # rare near-midpoint cases, for D log-uniform over 1e-300..1e300; values
    # whose FP32 reciprocal is not normal and finite take the division
    m = 4096
    shape = (1, m, 1)           # nx = nz = 1: each cell owns its two x faces
    rng = np.random.default_rng(7)
    d = 10.0 ** rng.uniform(-300, 300, m)
    d[:10] = [1e-45, 1.2e-38, 2.0 ** -126, 3.4e38, 3.5e38, 2.0 ** 127, 1.0, 3.0, 1e-300, 1e300]
    wx = np.zeros((1, m, 2))
    wx[0, :, 0] = d              # D = d + 0 + 0 + 0 + 0 + 0 exactly
    w = (_level(shape, wx, cuda_device, kind="x"),
         _level(shape, np.zeros((1, m + 1, 1)), cuda_device, kind="y"),
         _level(shape, np.zeros((2, m, 1)), cuda_device, kind="z"))
    got = K.get(K.inv_diag(w, shape), shape).cpu().numpy().ravel()
    want = 1.0 / d
    assert np.all(np.abs(got - want) <= np.spacing(want))
    assert np.mean(got == want) >= 0.99
    exact = [0, 2, 3, 4, 5, 6, 8, 9]     # the division fallback and powers of two
    np.testing.assert_array_equal(got[exact], want[exact])


def _rounding_cases(m, rng):
    """Doubles that exercise float rounding: random magnitudes 1e-50..1e50
    (FP32 subnormals, zeros and overflow among them), exact midpoints between
    neighbouring floats and the doubles just either side of them, the ends
    of FP32's normal range, and signed zeros."""
    v = np.sign(rng.uniform(-1, 1, m)) * 10.0 ** rng.uniform(-50, 50, m)
    f = (rng.uniform(1, 2, m) * 2.0 ** rng.integers(-120, 120, m)).astype(np.float32)
    f = f.astype(np.float64)
    half = np.spacing(f.astype(np.float32)).astype(np.float64) / 2
    k = m // 8
    v[:k] = f[:k] + half[:k]                                   # ties: to the even neighbour
    v[k:2 * k] = np.nextafter(f[k:2 * k] + half[k:2 * k], 0)   # just below a midpoint
    v[2 * k:3 * k] = np.nextafter(f[2 * k:3 * k] + half[2 * k:3 * k], np.inf)  # just above
    v[3 * k:4 * k] *= -1
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    v[4 * k:4 * k + 12] = [fmax, fmax + 2.0 ** 103, np.nextafter(fmax + 2.0 ** 103, 0),
                           fmax + 2.0 ** 104, tiny, np.nextafter(tiny, 0),
                           tiny * (1 - 2.0 ** -25), -tiny, 0.0, -0.0, 1.0, -3.0]
    return v


def test_fp32_rounding_is_round_to_nearest_even(cuda_device):
    # the FP32 copies of the weights and of 1/D (mg_op_round_f32) are the
    # IEEE round-to-nearest-even images of the FP64 values, bit for bit
    # (numpy's float64 -> float32 conversion is that rounding)
    m = 4096
    shape = (1, m, 1)
    rng = np.random.default_rng(21)
    vals = {"x": _rounding_cases(2 * m, rng).reshape(1, m, 2),
            "y": _rounding_cases(m + 1, rng).reshape(1, m + 1, 1),
            "z": _rounding_cases(2 * m, rng).reshape(2, m, 1),
            "cell": _rounding_cases(m, rng).reshape(1, m, 1)}
    w = [_level(shape, vals[k], cuda_device, kind=k) for k in "xyz"]
    invD = _level(shape, vals["cell"], cuda_device)
    w32, inv32 = K.round_f32(w, invD, shape)
    with np.errstate(over="ignore"):
        for t, k in zip(list(w32) + [inv32], "xyz" + "c"):
            kind = "cell" if k == "c" else k
            got = K.get(t, shape, kind).cpu().numpy()
            want = vals[kind].astype(np.float32)
            np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))


def test_refinement_update_widens_exactly(cuda_device):
    # x += 1 * e from x = 0 (mg_op_refine): every FP32 correction, zeros,
    # subnormals and the ends of the range included, lands in x unchanged
    m = 4096
    shape = (1, m, 1)
    rng = np.random.default_rng(22)
    e = (np.sign(rng.uniform(-1, 1, m)) * 10.0 ** rng.uniform(-45, 38, m)).astype(np.float32)
    fi = np.finfo(np.float32)
    e[:8] = [0.0, -0.0, fi.tiny, fi.tiny / 8, -fi.tiny / 3, fi.max, -fi.max, 1.0]
    dims = {"x": (1, m, 2), "y": (1, m + 1, 1), "z": (2, m, 1), "cell": (1, m, 1)}
    zero = lambda kind: _level(shape, np.zeros(dims[kind]), cuda_device, kind=kind)
    w = [zero(k) for k in "xyz"]
    x = _level(shape, np.zeros((1, m, 1)), cuda_device)
    et = _level(shape, e.reshape(1, m, 1), cuda_device, torch.float32)
    xo, _, _ = K.refine(w, zero("cell"), zero("cell"), x, et, 1.0, 1.0, shape)
    got = K.get(xo, shape).cpu().numpy().ravel()
    np.testing.assert_array_equal(got, e.astype(np.float64))


@pytest.mark.parametrize("shape", EVEN)
def test_coarsened_weights(cuda_device, shape):
    beta, _, _, h = _case(shape, 2)
    w = K.face_weights(_t(beta, cuda_device), h)
    cw = K.coarsen_weights(w, shape)
    c = tuple(s // 2 for s in shape)
    for wt, fo, kind in zip(cw, O.coarsen_faces(*O.face_beta(beta)), "xyz"):
        got = K.get(wt, c, kind).cpu().numpy()
        want = fo / (2 * h) ** 2
        assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-14


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", SHAPES)
def test_single_colour_passes(cuda_device, shape, dtype):
    beta, f, phi, h = _case(shape, 3)
    w, invD = _weights(beta, h, shape, cuda_device, dtype)
    ft = _level(shape, f, cuda_device, dtype)
    pt = _level(shape, phi, cuda_device, dtype)
    faces = O.face_beta(beta)
    ref = phi
    for color in (0, 1):
        K.rbgs_pass(w, invD, ft, pt, shape, color)
        ref = O.rbgs_pass(faces, h, f, ref, color)
        got = K.get(pt, shape).cpu().double().numpy()
        scale = np.max(np.abs(ref)) + np.max(np.abs(f)) * h * h / np.min(faces[0])
        assert np.max(np.abs(got - ref)) <= _tol(dtype) * scale, color
    # the guard cells around the box stay zero
    full = pt.cpu()
    assert not full[0].any() and not full[-1].any()
    assert not full[:, shape[1]].any() and not full[:, :, shape[2]:].any()


@pytest.mark.parametrize("zc", [0, 1, 3, 8])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", SHAPES)
def test_fused_sweep_equals_red_then_black(cuda_device, shape, dtype, zc):
    beta, f, phi, h = _case(shape, 4)
    w, invD = _weights(beta, h, shape, cuda_device, dtype)
    ft = _level(shape, f, cuda_device, dtype)
    pin = _level(shape, phi, cuda_device, dtype)
    before = pin.clone()
    out = K.rbgs_sweep(w, ft, pin, shape, zc=zc)
    assert torch.equal(pin, before)  # out of place
    faces = O.face_beta(beta)
    ref = O.rbgs_pass(faces, h, f, O.rbgs_pass(faces, h, f, phi, 0), 1)
    got = K.get(out, shape).cpu().double().numpy()
    scale = np.max(np.abs(ref)) + np.max(np.abs(f)) * h * h / np.min(faces[0])
    assert np.max(np.abs(got - ref)) <= _tol(dtype) * scale
    # and equals the two single-colour passes on the GPU
    p2 = _level(shape, phi, cuda_device, dtype)
    K.rbgs_pass(w, invD, ft, p2, shape, 0)
    K.rbgs_pass(w, invD, ft, p2, shape, 1)
    assert torch.allclose(K.get(out, shape), K.get(p2, shape), rtol=0,
                          atol=_tol(dtype) * scale)
    full = out.cpu()
    assert not full[0].any() and not full[-1].any() and not full[:, :, shape[2]:].any()


@pytest.mark.parametrize("zc", [0, 1, 3, 8])
@pytest.mark.parametrize("shape", [(12, 11, 64), (70, 20, 130), (33, 40, 136)])
def test_tma_sweep_is_bitwise_the_plain_sweep(cuda_device, shape, zc):
    # same arithmetic in the same order; only the operand staging differs
    beta, f, phi, h = _case(shape, 14)
    w, _ = _weights(beta, h, shape, cuda_device, torch.float32)
    ft = _level(shape, f, cuda_device, torch.float32)
    pin = _level(shape, phi, cuda_device, torch.float32)
    before = pin.clone()
    a = K.rbgs_sweep(w, ft, pin, shape, zc=zc)
    b = K.rbgs_sweep_tma(w, ft, pin, shape, zc=zc)
    assert torch.equal(pin, before)
    assert torch.equal(a, b)
    full = b.cpu()
    assert not full[0].any() and not full[-1].any() and not full[:, :, shape[2]:].any()


@pytest.mark.parametrize("zc", [0, 3, 8])
@pytest.mark.parametrize("shape", [(12, 12, 64), (70, 20, 130), (34, 40, 136)])
def test_tma_sweep_with_prolongation_is_prolongation_then_sweep(cuda_device, shape, zc):
    # the fused form adds each red update's neighbours' parent corrections to
    # their staged values: bitwise the prolongation kernel followed by the
    # sweep, and phi_in itself stays unprolonged
    beta, f, phi, h = _case(shape, 15)
    w, _ = _weights(beta, h, shape, cuda_device, torch.float32)
    ft = _level(shape, f, cuda_device, torch.float32)
    pin = _level(shape, phi, cuda_device, torch.float32)
    c = tuple(s // 2 for s in shape)
    e = np.random.default_rng(16).uniform(-1, 1, c).astype(np.float32)
    pc = _level(c, e, cuda_device, torch.float32)
    before = pin.clone()
    fused = K.rbgs_sweep_tma_prolong(w, ft, pc, pin, shape, zc=zc)
    assert torch.equal(pin, before)
    prolonged = K.prolong_add(pc, pin.clone(), shape)
    want = K.rbgs_sweep(w, ft, prolonged, shape, zc=zc)
    assert torch.equal(fused, want)
    # against the oracle: a red-black sweep of the prolonged iterate
    faces = O.face_beta(beta)
    up = phi.astype(np.float64) + np.repeat(np.repeat(np.repeat(e, 2, 0), 2, 1), 2, 2)
    ref = O.rbgs_pass(faces, h, f, O.rbgs_pass(faces, h, f, up, 0), 1)
    got = K.get(fused, shape).cpu().double().numpy()
    scale = np.max(np.abs(ref)) + np.max(np.abs(f)) * h * h / np.min(faces[0])
    assert np.max(np.abs(got - ref)) <= _tol(torch.float32) * scale


@pytest.mark.parametrize("stored_diag", [False, True])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", SHAPES)
def test_residual_and_norm(cuda_device, shape, dtype, stored_diag):
    if stored_diag and dtype == torch.float32:
        pytest.skip("the stored diagonal is an FP64-level array")
    beta, f, phi, h = _case(shape, 5)
    w, _ = _weights(beta, h, shape, cuda_device, dtype)
    D = K.inv_diag(w, shape, with_diag=True)[1] if stored_diag else None
    ft = _level(shape, f, cuda_device, dtype)
    pt = _level(shape, phi, cuda_device, dtype)
    faces = O.face_beta(beta)
    ref = O.residual(faces, h, f, phi)
    got = K.get(K.residual(w, ft, pt, shape, D), shape).cpu().double().numpy()
    scale = np.max(np.abs(f)) + 2 * 6 * np.max(faces[0]) / h ** 2 * np.max(np.abs(phi))
    assert np.max(np.abs(got - ref)) <= _tol(dtype) * scale
    nrm = K.residual_norm(w, ft, pt, shape, D).item()
    want = O.norm2(ref)
    assert abs(nrm - want) <= _tol(dtype) * scale * np.sqrt(ref.size)


@pytest.mark.parametrize("stored_diag", [False, True])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", EVEN)
def test_residual_restrict_and_prolong(cuda_device, shape, dtype, stored_diag):
    if stored_diag and dtype == torch.float32:
        pytest.skip("the stored diagonal is an FP64-level array")
    beta, f, phi, h = _case(shape, 6)
    w, _ = _weights(beta, h, shape, cuda_device, dtype)
    D = K.inv_diag(w, shape, with_diag=True)[1] if stored_diag else None
    ft = _level(shape, f, cuda_device, dtype)
    pt = _level(shape, phi, cuda_device, dtype)
    faces = O.face_beta(beta)
    c = tuple(s // 2 for s in shape)
    fc, phic = K.residual_restrict(w, ft, pt, shape, D)
    ref = O.restrict(O.residual(faces, h, f, phi))
    got = K.get(fc, c).cpu().double().numpy()
    scale = np.max(np.abs(f)) + 2 * 6 * np.max(faces[0]) / h ** 2 * np.max(np.abs(phi))
    assert np.max(np.abs(got - ref)) <= _tol(dtype) * scale
    assert not K.get(phic, c).any()
    # prolongation: phi += coarse value of the parent
    e = np.random.default_rng(7).uniform(-1, 1, c)
    et = _level(c, e, cuda_device, dtype)
    K.prolong_add(et, pt, shape)
    want = O.prolong_add(e, phi)
    got = K.get(pt, shape).cpu().double().numpy()
    assert np.max(np.abs(got - want)) <= _tol(dtype) * 2


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", EVEN)
def test_red_children_restriction_after_a_sweep(cuda_device, shape, dtype):
    # right after a red then black pass the black residuals vanish (to
    # rounding), so restricting the red children alone equals the oracle's
    # residual + restriction of the same state
    beta, f, phi, h = _case(shape, 13)
    faces = O.face_beta(beta)
    phi = O.rbgs_pass(faces, h, f, O.rbgs_pass(faces, h, f, phi, 0), 1)
    w, _ = _weights(beta, h, shape, cuda_device, dtype)
    D = K.inv_diag(w, shape, with_diag=True)[1] if dtype == torch.float64 else None
    fc, phic = K.residual_restrict(w, _level(shape, f, cuda_device, dtype),
                                   _level(shape, phi, cuda_device, dtype), shape, D, red_only=True)
    c = tuple(s // 2 for s in shape)
    ref = O.restrict(O.residual(faces, h, f, phi))
    scale = np.max(np.abs(f)) + 2 * 6 * np.max(faces[0]) / h ** 2 * np.max(np.abs(phi))
    assert np.max(np.abs(K.get(fc, c).cpu().double().numpy() - ref)) <= _tol(dtype) * scale
    assert not K.get(phic, c).any()


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 2, 2), (3, 8, 8), (7, 3, 5), (4, 16, 16)])
def test_coarsest_level_inverse_and_solve(cuda_device, shape):
    beta, f, _, h = _case(shape, 8)
    w = K.face_weights(_t(beta, cuda_device), h)
    ainv = K.bottom_inverse(w, shape)
    A = O.dense_matrix(O.face_beta(beta), h, shape)
    got = ainv.cpu().numpy()
    want = np.linalg.inv(A)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    for dtype in (torch.float64, torch.float32):
        ft = _level(shape, f, cuda_device, dtype)
        phi = K.bottom_solve(ainv.to(dtype), ft, shape)
        x = np.linalg.solve(A, f.ravel()).reshape(shape)
        g = K.get(phi, shape).cpu().double().numpy()
        assert np.max(np.abs(g - x)) <= (1e-12 if dtype == torch.float64 else 1e-5) * \
            np.max(np.abs(x))


@pytest.mark.parametrize("shape", [(5, 7, 9), (20, 17, 33), (70, 20, 130)])
def test_refinement_step(cuda_device, shape):
    # x += c_e e in FP64; r = f - A x in FP64; r32 = float(r) * float(1/c_r)
    # (two FP32 roundings plus the product: <= 3 ulp = 2^-22 relative);
    # ||r|| from the FP32 squares to FP32 accuracy.
    beta, f, x, h = _case(shape, 9)
    w = K.face_weights(_t(beta, cuda_device), h)
    _, D = K.inv_diag(w, shape, with_diag=True)
    e = np.random.default_rng(10).uniform(-1, 1, shape).astype(np.float32)
    c_e, c_r = 0.37, 2.5
    xt = _level(shape, x, cuda_device)
    et = _level(shape, e, cuda_device, torch.float32)
    xo, r32, nrm = K.refine(w, D, _level(shape, f, cuda_device), xt, et, c_e, c_r, shape)
    assert not et.any()          # the correction is used up: the next cycles start from 0
    faces = O.face_beta(beta)
    want_x = x + c_e * e.astype(np.float64)
    r = O.residual(faces, h, f, want_x)
    gx = K.get(xo, shape).cpu().numpy()
    assert np.max(np.abs(gx - want_x)) <= 1e-15 * np.max(np.abs(want_x))
    scale = np.max(np.abs(f)) + 12 * np.max(faces[0]) / h ** 2 * np.max(np.abs(want_x))
    gr = K.get(r32, shape).cpu().double().numpy()
    assert np.max(np.abs(gr - r / c_r)) <= 1e-13 * scale / c_r + 2.0 ** -22 * np.max(np.abs(r / c_r))
    assert abs(nrm.item() - O.norm2(r)) <= 1e-6 * O.norm2(r)


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 7, 9), (20, 17, 33)])
def test_beta_gradient_assembly(cuda_device, shape):
    beta, _, phi, h = _case(shape, 11)
    lam = np.random.default_rng(12).uniform(-1, 1, shape)
    got = K.beta_grad(_t(beta, cuda_device), _t(phi, cuda_device), _t(lam, cuda_device), h)
    want = O.beta_grad(beta, h, phi, lam)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got.cpu().numpy() - want)) <= 1e-13 * scale
