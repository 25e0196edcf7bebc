"""Coupled levels on the GPU (mg_level) against the oracle's masked-domain
solve: the boxes of one level (paper Sec. 2: the disjoint grids of a
MultiFAB level) solved as one domain.  Parity bar as for single boxes:
relative L2 difference <= 1e-9 from the oracle at a 1e-13 relative residual,
and the oracle's own residual of the GPU solution <= 1.01 x the tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_2801_gb300 import LevelSolver, MGError, Solver, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _domain(shape, seed):
    nz, ny, nx = shape
    d = inputs.stellar((nx, ny, nz), seed)
    return d["beta"], d["f"], d["dx"]


def _level_solve(los, ns, beta, f, h, dev, precision="fp64", **kw):
    """Solve the level made of boxes (lo (i, j, k), n (nx, ny, nz)) cut out of
    bounding-box arrays; returns the solution on the bounding box (0 outside)
    and the stats."""
    shapes = [(c, b, a) for (a, b, c) in ns]
    sl = [(slice(k, k + c), slice(j, j + b), slice(i, i + a))
          for (i, j, k), (a, b, c) in zip(los, ns)]
    with LevelSolver(los, shapes, h, precision=precision, device=dev, **kw) as lv:
        lv.set_beta(_t(np.concatenate([beta[s].ravel() for s in sl]), dev))
        phi, st = lv.solve(_t(np.concatenate([f[s].ravel() for s in sl]), dev), tol=TOL)
        parts = lv.unpack(phi.cpu())
        nlev = lv.levels()
    out = np.zeros(beta.shape)
    for s, p in zip(sl, parts):
        out[s] = p.numpy()
    return out, st, nlev


def _check(los, ns, beta, f, h, dev, precision="fp64"):
    mask = O.level_mask(los, ns, beta.shape)
    f = f * mask
    phi, st, nlev = _level_solve(los, ns, beta, f, h, dev, precision)
    assert st["status"] == "ok", st
    ref, info = O.masked_solve(beta, mask, f, h, tol=1e-13)
    assert info["status"] == "ok"
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)
    r = O.residual(O.masked_face_beta(beta, mask), h, f, phi) * mask
    assert O.norm2(r) <= TOL * 1.01 * O.norm2(f)
    assert np.all(phi[mask == 0] == 0.0)
    return st, nlev


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rectangle_tiled_by_boxes_is_the_single_box_solve(cuda_device, precision):
    beta, f, h = _domain((32, 32, 32), 1)
    los = [(i, j, k) for k in (0, 16) for j in (0, 16) for i in (0, 16)]
    ns = [(16, 16, 16)] * 8
    st, nlev = _check(los, ns, beta, f, h, cuda_device, precision)
    assert nlev == 5                      # 16 -> 8 -> 4 -> 2 -> 1: an 8-cell union bottom
    with Solver(beta.shape, h, precision=precision, device=cuda_device) as s:
        s.set_beta(_t(beta, cuda_device))
        one, _ = s.solve(_t(f, cuda_device), tol=TOL)
    phi, _, _ = _level_solve(los, ns, beta, f, h, cuda_device, precision)
    assert np.linalg.norm(phi - one.cpu().numpy()) <= 1e-9 * np.linalg.norm(phi)


def test_mixed_level_leaves_inner_cycles_as_one_domain(cuda_device):
    # the boxes of a level share ghost cells: the adaptive inner cycles end
    # for all of them at once, on the domain's inner residual, so the level
    # takes the refinement steps of the single box it tiles
    beta, f, h = _domain((96, 96, 96), 4)
    los = [(i, j, k) for k in (0, 32, 64) for j in (0, 32, 64) for i in (0, 32, 64)]
    ns = [(32, 32, 32)] * 27
    st, _ = _check(los, ns, beta, f, h, cuda_device, "mixed")
    with Solver(beta.shape, h, precision="mixed", device=cuda_device) as s:
        s.set_beta(_t(beta, cuda_device))
        _, st1 = s.solve(_t(f, cuda_device), tol=TOL)
    assert st["cycles"] <= st1["cycles"] + 1, (st["hist"], st1["hist"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_l_shaped_level(cuda_device, precision):
    beta, f, h = _domain((8, 32, 32), 2)
    los = [(0, 0, 0), (16, 0, 0), (0, 16, 0)]
    ns = [(16, 16, 8)] * 3
    _check(los, ns, beta, f, h, cuda_device, precision)


def _aligned_tiling(rng, shape, unit, depth):
    """Random k-d splits of the box on a grid of `unit` cells."""
    out = []

    def rec(lo, hi, d):
        sizes = [hi[i] - lo[i] for i in range(3)]
        if d == 0 or max(sizes) <= unit:
            out.append((tuple(lo), tuple(sizes)))
            return
        ax = int(np.argmax(np.array(sizes) * rng.uniform(0.5, 1.0, 3)))
        if sizes[ax] <= unit:
            out.append((tuple(lo), tuple(sizes)))
            return
        cut = lo[ax] + unit * int(rng.integers(1, sizes[ax] // unit))
        a_hi, b_lo = list(hi), list(lo)
        a_hi[ax] = cut
        b_lo[ax] = cut
        rec(lo, a_hi, d - 1)
        rec(b_lo, hi, d - 1)

    nz, ny, nx = shape
    rec([0, 0, 0], [nx, ny, nz], depth)
    return out


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_random_aligned_tilings_with_holes(cuda_device, seed):
    rng = np.random.default_rng(seed)
    shape = (24, 32, 40)
    boxes = _aligned_tiling(rng, shape, 8, 5)
    keep = [b for b in boxes if rng.uniform() > 0.15] or boxes
    los = [b[0] for b in keep]
    ns = [b[1] for b in keep]
    beta, f, h = _domain(shape, 10 + seed)
    _check(los, ns, beta, f, h, cuda_device)


def test_boxes_with_a_gap_solve_independently(cuda_device):
    beta, f, h = _domain((16, 16, 40), 6)
    los, ns = [(0, 0, 0), (24, 0, 0)], [(16, 16, 16), (16, 16, 16)]
    phi, st, _ = _level_solve(los, ns, beta, f, h, cuda_device)
    assert st["status"] == "ok"
    for (i, j, k), (a, b, c) in zip(los, ns):
        sl = (slice(k, k + c), slice(j, j + b), slice(i, i + a))
        ref, _ = O.solve(beta[sl], f[sl], h, tol=1e-13)
        assert np.linalg.norm(phi[sl] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_device_loop_matches_host_loop(cuda_device):
    beta, f, h = _domain((16, 32, 32), 7)
    los = [(0, 0, 0), (16, 0, 0), (0, 16, 0), (16, 16, 0)]
    ns = [(16, 16, 16)] * 4
    sl = [(slice(k, k + c), slice(j, j + b), slice(i, i + a))
          for (i, j, k), (a, b, c) in zip(los, ns)]
    res = []
    for use_graph in (True, False):
        with LevelSolver(los, [(16, 16, 16)] * 4, h, device=cuda_device,
                         use_graph=use_graph) as lv:
            lv.set_beta(_t(np.concatenate([beta[s].ravel() for s in sl]), cuda_device))
            phi, st = lv.solve(_t(np.concatenate([f[s].ravel() for s in sl]), cuda_device))
            res.append((phi.cpu(), st["cycles"], st["hist"]))
    assert torch.equal(res[0][0], res[1][0]) and res[0][1:] == res[1][1:]


def test_invalid_levels_are_rejected(cuda_device):
    with pytest.raises(MGError) as e:
        LevelSolver([(0, 0, 0), (8, 0, 0)], [(16, 16, 16)] * 2, 0.1, device=cuda_device)
    assert e.value.name == "invalid_arg"            # overlapping boxes
    with pytest.raises(MGError) as e:
        # 33 cells on each axis cannot be halved: a 35937-cell coarsest union
        LevelSolver([(0, 0, 0)], [(33, 33, 33)], 0.1, device=cuda_device)
    assert e.value.name == "unsupported"
