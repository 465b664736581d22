"""Regridding (Sec. 5.4, RDM-2/3), host only: the oracle's Berger-Rigoutsos clustering against
hand-derived cases and the properties that define it, and the library's amr_regrid box lists
bit-identical to the oracle's on structured and random tag sets in 2-D and 3-D, with
refinement ratios 2 and 4; every result passes both hierarchy validators."""
import os

import numpy as np
import pytest

from oracle import regrid as orr
from oracle.hierarchy import OK, validate


@pytest.fixture(scope="module")
def amr():
    from paper_2506_02663_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    from paper_2506_02663_gb300 import amr as m
    return m


def _rect(lo, hi):
    g = np.meshgrid(*[np.arange(a, b + 1) for a, b in zip(lo, hi)], indexing="ij")
    return np.stack([x.ravel() for x in g], axis=1)


def test_cluster_hand_cases():
    # one rectangle: its bounding box
    assert orr.cluster(_rect((3, 5), (9, 8)), (0, 0), (31, 31), 1.0, 2) == [((3, 5), (9, 8))]
    # two rectangles with a gap: cut at the hole
    t = np.concatenate([_rect((0, 0), (3, 3)), _rect((8, 0), (11, 3))])
    assert orr.cluster(t, (0, 0), (31, 31), 1.0, 2) == [((0, 0), (3, 3)), ((8, 0), (11, 3))]
    # an L: no hole; the signatures' second differences change sign at x = 4 and y = 4 with
    # equal jumps (8), equal distance to the middle and equal lengths: the lower dimension
    t = np.concatenate([_rect((0, 0), (7, 3)), _rect((0, 4), (3, 7))])
    assert orr.cluster(t, (0, 0), (31, 31), 1.0, 2) == [((0, 0), (3, 7)), ((4, 0), (7, 3))]
    # a single tagged cell widened to the minimum width, upwards first, then downwards
    assert orr.cluster(np.array([[5, 31]]), (0, 0), (31, 31), 0.5, 3) == [((5, 29), (7, 31))]
    # low efficiency accepts the bounding box of scattered tags
    t = np.array([[0, 0], [9, 9]])
    assert orr.cluster(t, (0, 0), (31, 31), 0.01, 2) == [((0, 0), (9, 9))]


def _properties(tags, boxes, eff, w):
    covered = np.zeros(len(tags), int)
    for lo, hi in boxes:
        n = [b - a + 1 for a, b in zip(lo, hi)]
        assert min(n) >= w
        inside = np.all((tags >= lo) & (tags <= hi), axis=1)
        covered += inside
        # accepted by efficiency, or no cut allowed (every dimension shorter than 2 w, and no
        # hole or inflection cut either, which needs a dimension of at least 2 w as well)
        assert inside.sum() >= eff * np.prod(n) or max(n) < 2 * w
    assert np.all(covered == 1)  # every tag in exactly one box
    for i in range(len(boxes)):
        for j in range(i + 1, len(boxes)):
            (a0, a1), (b0, b1) = boxes[i], boxes[j]
            assert any(a1[d] < b0[d] or b1[d] < a0[d] for d in range(len(a0)))  # disjoint


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("dim", [2, 3])
def test_cluster_properties_on_random_blobs(seed, dim):
    rng = np.random.default_rng(seed)
    n = 40 if dim == 2 else 16
    c = rng.integers(0, n, size=(3, dim))
    g = np.stack(np.meshgrid(*[np.arange(n)] * dim, indexing="ij"), axis=-1).reshape(-1, dim)
    d2 = np.min([np.sum((g - ci) ** 2, axis=1) for ci in c], axis=0)
    tags = g[d2 <= rng.integers(4, 30)]
    for eff, w in ((0.7, 2), (0.9, 3), (1.0, 2)):
        boxes = orr.cluster(tags, (0,) * dim, (n - 1,) * dim, eff, w)
        _properties(tags, boxes, eff, w)


def _vortex_tags(dim, n, level, rng, thresh):
    """Cells of level `level` whose distance to a few random centres is below a radius: the
    stand-in for |curl u| >= eps around vortex cores."""
    nd = n * 2 ** level
    g = np.stack(np.meshgrid(*[np.arange(nd)] * dim, indexing="ij"), axis=-1).reshape(-1, dim)
    x = (g + 0.5) / nd
    c = rng.random((3, dim)) * 0.6 + 0.2
    d = np.min([np.sqrt(np.sum((x - ci) ** 2, axis=1)) for ci in c], axis=0)
    return g[d < thresh]


CASES = [
    (2, (32, 32), 2, 2, (0.75, 2)),
    (2, (32, 32), 3, 2, (0.7, 2)),
    (2, (24, 40), 3, 2, (0.8, 3)),
    (3, (16, 16, 16), 2, 2, (0.7, 2)),
    (3, (16, 16, 16), 3, 2, (0.75, 2)),
    (2, (16, 16), 3, 4, (0.7, 1)),
]


@pytest.mark.parametrize("dim,n0,nlevels,ratio,par", CASES)
@pytest.mark.parametrize("seed", range(3))
def test_library_regrid_matches_oracle(amr, dim, n0, nlevels, ratio, par, seed):
    rng = np.random.default_rng(100 + seed)
    eff, w = par
    tags = []
    for l in range(nlevels - 1):
        nd = [v * ratio ** l for v in n0]
        g = np.stack(np.meshgrid(*[np.arange(v) for v in nd], indexing="ij"), axis=-1).reshape(-1, dim)
        x = (g + 0.5) / np.asarray(nd)
        c = rng.random((2, dim)) * 0.5 + 0.25
        d = np.min([np.sqrt(np.sum((x - ci) ** 2, axis=1)) for ci in c], axis=0)
        tags.append(g[d < 0.12 / (l + 1)])
    ref = orr.regrid(dim, n0, nlevels, tags, eff, w, ratio)
    got = amr.regrid(dim, n0, nlevels, tags, eff, w, ratio)
    assert got == ref
    code, msg = validate(dim, ratio, tuple(n0), ref, [0] * (2 * dim))
    assert code == OK, msg
    if ratio == 2:
        amr.Hierarchy(dim, n0, ref)  # the library's own checks (nesting margin, sizes)
    # every tag of level l lies in the new level l + 1 (coarsened)
    for l in range(1, len(ref)):
        lo = np.array([b[0] for b in ref[l]]) // ratio
        hi = np.array([b[1] for b in ref[l]]) // ratio
        t = tags[l - 1]
        inside = np.zeros(len(t), bool)
        for a, b in zip(lo, hi):
            inside |= np.all((t >= a) & (t <= b), axis=1)
        assert inside.all()


def test_regrid_edge_cases(amr):
    # no tags: level 0 only
    assert amr.regrid(2, (16, 16), 3, [np.zeros((0, 2)), np.zeros((0, 2))], 0.7, 2) == [[((0, 0), (15, 15))]]
    assert orr.regrid(2, (16, 16), 3, [np.zeros((0, 2)), np.zeros((0, 2))], 0.7, 2) == [[((0, 0), (15, 15))]]
    # the whole domain tagged: one box over the refined domain
    t = _rect((0, 0), (15, 15))
    assert amr.regrid(2, (16, 16), 2, [t], 1.0, 2) == [[((0, 0), (15, 15))], [((0, 0), (31, 31))]]
    # tags only on level 1 of three: level 1 is made from the grown coarsened level 2
    t1 = _rect((12, 12), (15, 15))
    got = amr.regrid(2, (16, 16), 3, [np.zeros((0, 2)), t1], 0.7, 2)
    assert got == orr.regrid(2, (16, 16), 3, [np.zeros((0, 2)), t1], 0.7, 2)
    assert len(got) == 3
    # argument errors
    with pytest.raises(amr.AmrError):
        amr.regrid(2, (16, 16), 2, [np.array([[16, 0]])], 0.7, 2)  # outside the level
    with pytest.raises(amr.AmrError):
        amr.regrid(2, (16, 16), 2, [t], 0.7, 1)  # refined boxes would have fewer than 4 cells
    with pytest.raises(amr.AmrError):
        amr.regrid(2, (16, 16), 2, [t], 0.0, 2)
