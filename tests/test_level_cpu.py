"""Host logic of a coupled level (no GPU): the ghost-exchange records that the
hash-binned intersection search produces (paper Sec. 2: boxes binned by the
region of their lowest corner, search of the own and neighbouring regions)
equal an independent all-pairs search written here, on random tilings with
holes; overlapping boxes are rejected; every interior face of the union is
seen from both sides and no boundary face is."""
import itertools

import numpy as np
import pytest

from paper_1008_2801_gb300 import MGError, level_intersections


def brute(los, ns):
    recs = set()
    for b, (lo, n) in enumerate(zip(los, ns)):
        for f in range(6):
            d = f // 2
            slo = list(lo)
            shi = [lo[i] + n[i] for i in range(3)]
            if f & 1:
                slo[d], shi[d] = shi[d], shi[d] + 1
            else:
                slo[d], shi[d] = slo[d] - 1, slo[d]
            for c, (lo2, n2) in enumerate(zip(los, ns)):
                if c == b:
                    continue
                ilo = [max(slo[i], lo2[i]) for i in range(3)]
                ihi = [min(shi[i], lo2[i] + n2[i]) for i in range(3)]
                if all(ilo[i] < ihi[i] for i in range(3)):
                    recs.add((b, c, tuple(ilo[i] - lo[i] for i in range(3)),
                              tuple(ilo[i] - lo2[i] for i in range(3)),
                              tuple(ihi[i] - ilo[i] for i in range(3))))
    return recs


def as_set(recs):
    return {(r["dst"], r["src"], r["d"], r["s"], r["e"]) for r in recs}


def kd_tiling(rng, lo, hi, depth, out):
    """Random axis-aligned splits of [lo, hi) into boxes."""
    sizes = [hi[i] - lo[i] for i in range(3)]
    if depth == 0 or max(sizes) < 4:
        out.append((tuple(lo), tuple(sizes)))
        return
    d = int(np.argmax(np.array(sizes) * rng.uniform(0.5, 1.0, 3)))
    cut = int(rng.integers(lo[d] + 1, hi[d]))
    a_hi = list(hi)
    a_hi[d] = cut
    b_lo = list(lo)
    b_lo[d] = cut
    kd_tiling(rng, lo, a_hi, depth - 1, out)
    kd_tiling(rng, b_lo, hi, depth - 1, out)


@pytest.mark.parametrize("seed", range(6))
def test_hash_binned_records_equal_all_pairs(seed):
    rng = np.random.default_rng(seed)
    boxes = []
    kd_tiling(rng, [-7, 3, 0], [25, 30, 21], 6, boxes)
    keep = [b for b in boxes if rng.uniform() > 0.2]          # holes in the union
    los = [b[0] for b in keep]
    ns = [b[1] for b in keep]
    want = brute(los, ns)
    got = as_set(level_intersections(los, ns))
    assert got == want
    assert as_set(level_intersections(los, ns, brute=True)) == want
    assert len(level_intersections(los, ns)) == len(want)   # no duplicates


def test_every_interior_face_is_exchanged_from_both_sides():
    rng = np.random.default_rng(42)
    boxes = []
    kd_tiling(rng, [0, 0, 0], [16, 12, 10], 5, boxes)
    los = [b[0] for b in boxes]
    ns = [b[1] for b in boxes]
    owner = -np.ones((10, 12, 16), dtype=int)
    for b, ((i, j, k), (a, bb, c)) in enumerate(zip(los, ns)):
        owner[k:k + c, j:j + bb, i:i + a] = b
    assert (owner >= 0).all()          # the tiling covers the rectangle
    inter = 0
    for ax in range(3):
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[2 - ax] = slice(0, -1)
        sl1[2 - ax] = slice(1, None)
        inter += int((owner[tuple(sl0)] != owner[tuple(sl1)]).sum())
    cells = sum(np.prod(r["e"]) for r in level_intersections(los, ns))
    assert cells == 2 * inter          # each interface face: one guard cell per side


def test_overlapping_boxes_are_rejected():
    with pytest.raises(MGError):
        level_intersections([(0, 0, 0), (3, 0, 0)], [(4, 4, 4), (4, 4, 4)])
    # touching is fine, and boxes only touching along an edge exchange nothing
    assert level_intersections([(0, 0, 0), (4, 4, 0)], [(4, 4, 4), (4, 4, 4)]) == []


def test_many_boxes_in_a_line_find_only_their_neighbours():
    los = [(8 * i, 0, 0) for i in range(200)]
    ns = [(8, 4, 4)] * 200
    recs = level_intersections(los, ns)
    assert len(recs) == 2 * 199
    assert all(abs(r["dst"] - r["src"]) == 1 for r in recs)
