"""Regridding (Sec. 5.4, RDM-2 and RDM-3) -- new level boxes from tagged cells (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper delegates the clustering to Berger & Rigoutsos and fixes the order of the levels:
the finest new level from the tags of the level below it (RDM-2); then, level by level
downwards, the tags of level l united with the boxes of the new level l+2 coarsened twice and
grown, clustered into the new level l+1 (RDM-3).  Readings (the paper states neither):
* growth: ceil(3 / r) cells of level l, clipped to the domain (the paper's one cell at r = 4);
  it gives every new level the three-cell margin that the AMRCFI windows need around the
  next finer level (R7);
* clustering of the tags T of a region (the recursion partitions the level's domain into
  disjoint regions at least w cells wide): the bounding box of T widened inside the region
  to w cells (first upwards, then downwards); accepted when |T| >= efficiency |box|;
  otherwise cut along one dimension, both parts at least w wide, at (a) a hole (a cut next
  to an empty slice of the signature), the one closest to the middle of its dimension, else
  (b) an inflection point (the second differences of the signature on the two sides of the
  cut have strictly opposite signs), the one with the largest jump between them, else
  (c) the middle of the longest dimension that can be cut; ties: closest to the middle, then
  the longer dimension, then the lower dimension, then the lower position; lower region
  first; a box that cannot be cut is accepted.
"""
import math

import numpy as np

NEST_MARGIN = 3
MIN_BOX = 4


def _signatures(tags, lo, n):
    """Tags per slice along every dimension (Berger-Rigoutsos signatures)."""
    return [np.bincount(tags[:, d] - lo[d], minlength=n[d]).astype(np.int64) for d in range(len(n))]


def _cut_order(c, n, d):
    """Tie-break key of a cut at offset c in a dimension of n cells: distance to the middle,
    longer dimension, lower dimension, lower position."""
    return (abs(2 * c - n), -n, d, c)


def choose_cut(tags, lo, n, w):
    """(d, c) of the Berger-Rigoutsos cut of the box [lo, lo + n) holding ``tags``, or None."""
    D = len(n)
    sig = _signatures(tags, lo, n)
    holes = []
    for d in range(D):
        for c in range(w, n[d] - w + 1):
            if sig[d][c - 1] == 0 or sig[d][c] == 0:
                holes.append((_cut_order(c, n[d], d), d, c))
    if holes:
        _, d, c = min(holes)
        return d, c
    infl = []
    for d in range(D):
        lap = sig[d][:-2] - 2 * sig[d][1:-1] + sig[d][2:]  # lap[i] is at slice i + 1
        for c in range(max(w, 2), min(n[d] - w, n[d] - 2) + 1):
            a, b = lap[c - 2], lap[c - 1]  # at slices c - 1 and c
            if a * b < 0:
                infl.append(((-abs(int(b) - int(a)),) + _cut_order(c, n[d], d), d, c))
    if infl:
        _, d, c = min(infl)
        return d, c
    cand = [((-n[d], d), d, n[d] // 2) for d in range(D) if n[d] >= 2 * w]
    if cand:
        _, d, c = min(cand)
        return d, c
    return None


def cluster(tags, region_lo, region_hi, efficiency, w):
    """Berger-Rigoutsos clustering of the tagged cells (an (m, D) integer array) of the region
    [region_lo, region_hi]: a list of disjoint boxes (lo, hi) covering every tag."""
    tags = np.asarray(tags, dtype=np.int64)
    if len(tags) == 0:
        return []
    D = tags.shape[1]
    lo = list(tags.min(axis=0))
    hi = list(tags.max(axis=0))
    for d in range(D):
        need = w - (hi[d] - lo[d] + 1)
        if need > 0:
            up = min(need, region_hi[d] - hi[d])
            hi[d] += up
            lo[d] -= need - up
    n = [hi[d] - lo[d] + 1 for d in range(D)]
    if len(tags) >= efficiency * float(np.prod(n)):
        return [(tuple(int(v) for v in lo), tuple(int(v) for v in hi))]
    cut = choose_cut(tags, lo, n, w)
    if cut is None:
        return [(tuple(int(v) for v in lo), tuple(int(v) for v in hi))]
    d, c = cut
    split = lo[d] + c
    lo_hi = list(hi)
    lo_hi[d] = split - 1
    hi_lo = list(lo)
    hi_lo[d] = split
    below = tags[:, d] < split
    return (cluster(tags[below], lo, lo_hi, efficiency, w) +
            cluster(tags[~below], hi_lo, hi, efficiency, w))


def regrid(dim, n0, nlevels, tags, efficiency, min_width, ratio=2):
    """RDM-2 and RDM-3: the boxes of the new hierarchy per level (level 0: the domain), from
    ``tags[l]`` (cells of level l, l = 0 .. nlevels - 2).  Levels end at the first empty one."""
    r = ratio
    grow = math.ceil(NEST_MARGIN / r)
    new = [None] * nlevels
    for l in range(nlevels - 2, -1, -1):
        nd = [n0[d] * r ** l for d in range(dim)]
        cells = [np.asarray(tags[l], dtype=np.int64).reshape(-1, dim)]
        if l + 2 < nlevels and new[l + 2]:
            for blo, bhi in new[l + 2]:
                lo = [max(blo[d] // (r * r) - grow, 0) for d in range(dim)]
                hi = [min(bhi[d] // (r * r) + grow, nd[d] - 1) for d in range(dim)]
                grid = np.meshgrid(*[np.arange(lo[d], hi[d] + 1) for d in range(dim)], indexing="ij")
                cells.append(np.stack([g.ravel() for g in grid], axis=1))
        allc = np.unique(np.concatenate(cells, axis=0), axis=0) if sum(len(c) for c in cells) else np.zeros((0, dim))
        boxes = cluster(allc, [0] * dim, [v - 1 for v in nd], efficiency, min_width)
        new[l + 1] = [(tuple(v * r for v in lo), tuple((v + 1) * r - 1 for v in hi)) for lo, hi in boxes]
    out = [[((0,) * dim, tuple(v - 1 for v in n0))]]
    for l in range(1, nlevels):
        if not new[l]:
            break
        out.append(new[l])
    return out


def migrate(H_old, F_old, H_new):
    """Data migration (the paragraph after RDM-4): the new composite field (level arrays of
    H_new).  Levels in order; a cell of a new box inside a box of the old same level takes the
    old value; any other cell the AMRCFI value (Sec. 5.2) from the new level below, which is
    complete by then (reading: the interpolation source is the old data as carried onto the
    new coarser level).  Cells outside the new boxes stay NaN."""
    from . import composite as cp
    from .cfi import cfi_values
    F_new = cp.new_field(H_new, (), np.nan)
    for l, lev in enumerate(H_new.levels):
        cells = np.argwhere(lev.covered)
        g = cells + np.asarray(lev.origin)
        in_old = np.zeros(len(g), bool)
        if l < len(H_old.levels):
            old = H_old.levels[l]
            a = g - np.asarray(old.origin)
            ok = np.all((a >= 0) & (a < np.asarray(old.shape)), axis=1)
            in_old[ok] = old.covered[tuple(a[ok].T)]
            F_new[l][tuple(cells[in_old].T)] = F_old[l][tuple(a[in_old].T)]
        rest = ~in_old
        if rest.any():
            crs = H_new.levels[l - 1]
            vals, _ = cfi_values(F_new[l - 1], crs.origin, crs.ndom, g[rest], H_new.ratio, H_new.D)
            F_new[l][tuple(cells[rest].T)] = vals
    return F_new
