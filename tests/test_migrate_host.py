"""Data migration after regridding (Sec. 5.4, last paragraph), host side (no GPU): the oracle's
migration pinned (identity on an unchanged hierarchy, exact on quartic cell averages), and the
library's migration plan checked against it cell by cell -- which cells are copied, which
interpolated, each window's first coarse cell, and every element offset the device kernels
use (inside the fields, at the right cells)."""
import os

import numpy as np
import pytest

from oracle import regrid as orr
from oracle.cfi import window_start
from oracle.hierarchy import Hierarchy as OH


@pytest.fixture(scope="module")
def amr():
    from paper_2506_02663_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    from paper_2506_02663_gb300 import amr as m
    return m


PAIRS = {
    # 2-D: the fine box moves and grows; a new second box
    "move2d": (2, (32, 32), [[((0, 0), (31, 31))], [((16, 16), (39, 39))]],
               [[((0, 0), (31, 31))], [((20, 12), (47, 39)), ((8, 44), (19, 55))]]),
    # 2-D three levels, the finest level appears; an old level disappears at the top
    "three2d": (2, (24, 24), [[((0, 0), (23, 23))], [((12, 12), (35, 35))]],
                [[((0, 0), (23, 23))], [((8, 8), (39, 39))], [((24, 24), (55, 55))]]),
    "drop2d": (2, (24, 24), [[((0, 0), (23, 23))], [((8, 8), (39, 39))], [((24, 24), (55, 55))]],
               [[((0, 0), (23, 23))], [((12, 12), (35, 35))]]),
    # a box on the physical boundary (windows slid inward)
    "edge2d": (2, (16, 16), [[((0, 0), (15, 15))], [((8, 8), (23, 23))]],
               [[((0, 0), (15, 15))], [((0, 0), (15, 31))]]),
    "move3d": (3, (12, 12, 12), [[((0, 0, 0), (11, 11, 11))], [((4, 4, 4), (15, 15, 15))]],
               [[((0, 0, 0), (11, 11, 11))], [((8, 6, 4), (19, 17, 15))]]),
    # new level 1 of two boxes sharing a face, new level 2 across it: windows over two patches
    "split2d": (2, (24, 24), [[((0, 0), (23, 23))], [((12, 12), (35, 35))]],
                [[((0, 0), (23, 23))], [((8, 8), (23, 39)), ((24, 8), (39, 39))], [((36, 28), (59, 51))]]),
    "split3d": (3, (12, 12, 12), [[((0, 0, 0), (11, 11, 11))], [((4, 4, 4), (15, 15, 15))]],
                [[((0, 0, 0), (11, 11, 11))], [((4, 4, 4), (11, 19, 19)), ((12, 4, 4), (19, 19, 19))],
                 [((18, 14, 14), (29, 25, 25))]]),
}


def _quartic_field(H):
    """Exact cell averages of p(x) = prod_d (x_d^4 - x_d^2 + x_d) + sum_d x_d^3 on every
    covered cell of every level (NaN elsewhere)."""
    from oracle import composite as cp
    F = cp.new_field(H, (), np.nan)
    for l, lev in enumerate(H.levels):
        h = lev.h
        cells = np.argwhere(lev.covered)
        g = cells + np.asarray(lev.origin)

        def avg(P, a):
            return (P(a + h) - P(a)) / h
        prod = np.ones(len(g))
        tot = np.zeros(len(g))
        for d in range(H.D):
            a = g[:, d] * h
            prod *= avg(lambda t: t ** 5 / 5 - t ** 3 / 3 + t ** 2 / 2, a)
            tot += avg(lambda t: t ** 4 / 4, a)
        F[l][tuple(cells.T)] = prod + tot
    return F


@pytest.mark.parametrize("name", list(PAIRS))
def test_oracle_migration_exact_on_quartics_and_identity(name):
    dim, n0, bo, bn = PAIRS[name]
    hi = tuple(n0[d] / n0[0] for d in range(dim))
    Ho, Hn = OH(dim, n0, bo, bc=[0] * (2 * dim), hi=hi), OH(dim, n0, bn, bc=[0] * (2 * dim), hi=hi)
    Fo, Fn_exact = _quartic_field(Ho), _quartic_field(Hn)
    Fn = orr.migrate(Ho, Fo, Hn)
    for l, lev in enumerate(Hn.levels):
        assert np.max(np.abs(Fn[l][lev.covered] - Fn_exact[l][lev.covered])) <= 1e-12
    # unchanged hierarchy: the migration copies every covered cell
    rng = np.random.default_rng(1)
    Fr = [np.where(lev.covered, rng.standard_normal(lev.shape), np.nan) for lev in Ho.levels]
    Fs = orr.migrate(Ho, Fr, Ho)
    for l, lev in enumerate(Ho.levels):
        assert np.array_equal(Fs[l][lev.covered], Fr[l][lev.covered])


def _offset(gh, l, g):
    """Element offset of global cell g of level l in gh's composite layout, and its patch."""
    for i, p in enumerate(gh.patches):
        if p["level"] != l:
            continue
        if all(p["lo"][e] <= g[e] <= p["hi"][e] for e in range(gh.dim)):
            a = [g[e] - p["lo"][e] + 2 for e in range(gh.dim)]
            return p["offset"] + a[0] + a[1] * p["sy"] + (a[2] * p["sz"] if gh.dim == 3 else 0), p
    return None, None


@pytest.mark.parametrize("name", list(PAIRS))
def test_migration_plan_matches_oracle(amr, name):
    dim, n0, bo, bn = PAIRS[name]
    Ho = OH(dim, n0, bo, bc=[0] * (2 * dim))
    Hn = OH(dim, n0, bn, bc=[0] * (2 * dim))
    go, gn = amr.Hierarchy(dim, n0, bo), amr.Hierarchy(dim, n0, bn)
    for l, lev in enumerate(Hn.levels):
        plan = amr.migrate_plan(go, gn, l)
        cells = np.argwhere(lev.covered)
        g = cells + np.asarray(lev.origin)
        in_old = np.zeros(len(g), bool)
        if l < len(Ho.levels):
            old = Ho.levels[l]
            a = g - np.asarray(old.origin)
            ok = np.all((a >= 0) & (a < np.asarray(old.shape)), axis=1)
            in_old[ok] = old.covered[tuple(a[ok].T)]
        # copied cells: the blocks tile exactly the new cells inside old boxes
        count = {}
        for b in plan["blocks"]:
            npch, opch, lo, hi_ = b[0], b[1], b[2:2 + dim], b[2 + dim:]
            nbox, obox = bn[l][npch], bo[l][opch]
            assert all(max(nbox[0][e], obox[0][e]) == lo[e] and min(nbox[1][e], obox[1][e]) == hi_[e]
                       for e in range(dim))
            for c in np.ndindex(*[hi_[e] - lo[e] + 1 for e in range(dim)]):
                key = tuple(int(lo[e] + c[e]) for e in range(dim))
                count[key] = count.get(key, 0) + 1
        want_copy = {tuple(int(v) for v in x) for x in g[in_old]}
        assert set(count) == want_copy and all(v == 1 for v in count.values())
        # interpolated cells: the others, with the oracle's windows and valid offsets
        got = {tuple(int(v) for v in c) for c in plan["cells"]}
        assert got == {tuple(int(v) for v in x) for x in g[~in_old]}
        assert len(got) == len(plan["cells"])
        crs = Hn.levels[l - 1] if l > 0 else None
        W = 5
        nside = 0
        for i, c in enumerate(plan["cells"]):
            start = [window_start(int(c[e]) // 2, crs.ndom[e]) for e in range(dim)]
            assert list(plan["starts"][i]) == start
            off, _ = _offset(gn, l, c)
            assert plan["dst"][i] == off and 0 <= off < gn.nelems
            # window cells with x fastest (ndindex varies its last index fastest)
            win = [tuple(start[e] + o[dim - 1 - e] for e in range(dim)) for o in np.ndindex(*([W] * dim))]
            offs = [_offset(gn, l - 1, w)[0] for w in win]
            assert all(o is not None and 0 <= o < gn.nelems for o in offs)
            src = plan["src"][i]
            if src >= 0:
                first, p = _offset(gn, l - 1, start)
                assert src == first
                assert all(p["lo"][e] <= start[e] and start[e] + W - 1 <= p["hi"][e] for e in range(dim))
            else:
                k = -1 - src
                assert list(plan["side"][k * W ** dim:(k + 1) * W ** dim]) == offs
                nside += 1
        if name.startswith("split") and l == 2:
            assert nside > 0  # the side tables were exercised


@pytest.mark.parametrize("name", list(PAIRS))
def test_migration_plan_executed_on_host_reproduces_oracle(amr, name):
    """The plan run on the host the way the device kernels read it (block copies between the
    two packed fields; AMRCFI values at dst from the window at src, or through the side table,
    in the packed new field) gives the oracle's migrated field."""
    from oracle import solve as so
    from oracle.cfi import weights_1d
    from _gpu_helpers import from_packed, to_packed
    dim, n0, bo, bn = PAIRS[name]
    Ho, Hn = OH(dim, n0, bo, bc=[0] * (2 * dim)), OH(dim, n0, bn, bc=[0] * (2 * dim))
    go, gn = amr.Hierarchy(dim, n0, bo), amr.Hierarchy(dim, n0, bn)
    U = so.Unknowns(Ho)
    Fo = U.scatter(np.random.default_rng(5).standard_normal(U.n), fill_invalid=True)
    po = to_packed(go, Ho, Fo, fill=np.nan)
    pn = np.full(gn.nelems, np.nan)
    W = 5
    for l in range(len(Hn.levels)):
        plan = amr.migrate_plan(go, gn, l)
        for b in plan["blocks"]:
            lo, hi_ = b[2:2 + dim], b[2 + dim:]
            for c in np.ndindex(*[hi_[e] - lo[e] + 1 for e in range(dim)]):
                g = tuple(int(lo[e] + c[e]) for e in range(dim))
                pn[_offset(gn, l, g)[0]] = po[_offset(go, l, g)[0]]
        for i, c in enumerate(plan["cells"]):
            start = plan["starts"][i]
            par = [int(c[e]) // 2 for e in range(dim)]
            w = [np.array([float(v) for v in weights_1d(par[e] - int(start[e]), int(c[e]) - 2 * par[e], 2)])
                 for e in range(dim)]
            src = plan["src"][i]
            if src >= 0:
                _, p = _offset(gn, l - 1, tuple(int(v) for v in start))
                offs = [src + o[dim - 1] + o[dim - 2] * p["sy"] + (o[0] * p["sz"] if dim == 3 else 0)
                        for o in np.ndindex(*([W] * dim))]
            else:
                k = -1 - src
                offs = list(plan["side"][k * W ** dim:(k + 1) * W ** dim])
            acc = 0.0
            for q, o in enumerate(np.ndindex(*([W] * dim))):
                wt = np.prod([w[e][o[dim - 1 - e]] for e in range(dim)])
                acc += wt * pn[offs[q]]
            pn[plan["dst"][i]] = acc
    got = from_packed(gn, Hn, pn)
    ref = orr.migrate(Ho, Fo, Hn)
    for l, lev in enumerate(Hn.levels):
        assert np.max(np.abs(got[l][lev.covered] - ref[l][lev.covered])) <= 1e-13, (name, l)
