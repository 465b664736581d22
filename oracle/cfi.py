"""Conservative fifth-order coarse-fine interpolation (AMRCFI), Sec. 5.2 (oracle).

The paper states what AMRCFI is -- a predetermined matrix applied to coarse cell averages,
depending only on r and the relative position of the fine cell, exactly conservative
(Eq. AMR_avergingDownToCrse holds) and fifth-order accurate -- but cites its formulas
instead of printing them.  The oracle therefore takes this reading:

* the reconstruction is the tensor product of one-dimensional reconstructions;
* in each dimension it is the polynomial of degree 4 whose averages over 5 consecutive
  coarse cells equal the given coarse averages (exact for degree <= 4, hence fifth order);
* the 5 cells are centred on the parent coarse cell {-2..2}; where that would leave the
  physical domain the window slides inward ({-1..3}, {0..4}, or mirrored);
* the fine value is the average of that polynomial over the fine sub-cell.

Because the windows and sub-cell weights are the same for every fine sub-cell of a parent,
the fine averages of the r^D children of a coarse cell average back to the coarse value
exactly (conservation).  The weights are derived here from that definition in exact
rational arithmetic; nothing is tabulated by hand.
"""
from fractions import Fraction as Fr
from functools import lru_cache

import numpy as np

WIDTH = 5  # cells per 1-D window (degree-4 polynomial)


def _solve_rational(M, b):
    """Gauss-Jordan elimination over the rationals: solve M x = b (M square)."""
    n = len(M)
    A = [list(M[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        p = next(i for i in range(c, n) if A[i][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [v / piv for v in A[c]]
        for i in range(n):
            if i != c and A[i][c] != 0:
                f = A[i][c]
                A[i] = [vi - f * vc for vi, vc in zip(A[i], A[c])]
    return [A[i][n] for i in range(n)]


@lru_cache(maxsize=None)
def weights_1d(pos, sub, r):
    """Weights w[0..4] (Fractions) such that the average over fine sub-cell ``sub``
    (0..r-1, low to high) of coarse cell ``pos`` (0..4 within the window) of the quartic
    matching the window's 5 coarse averages is sum_a w[a] * coarse[a].

    Coarse cell a of the window spans [a, a+1] in coarse-cell units.
    """
    # moments: M[a][m] = int_a^{a+1} x^m dx ; the quartic p(x) = sum_m c_m x^m satisfies
    # M c = Phi.  The fine average is v . c with v[m] = r * int_{pos+sub/r}^{pos+(sub+1)/r} x^m.
    def integ(lo, hi, m):
        return (hi ** (m + 1) - lo ** (m + 1)) / (m + 1)

    M = [[integ(Fr(a), Fr(a + 1), m) for m in range(WIDTH)] for a in range(WIDTH)]
    lo = Fr(pos) + Fr(sub, r)
    hi = Fr(pos) + Fr(sub + 1, r)
    v = [r * integ(lo, hi, m) for m in range(WIDTH)]
    # w = v^T M^{-1}  <=>  M^T w = v
    MT = [[M[a][m] for a in range(WIDTH)] for m in range(WIDTH)]
    return tuple(_solve_rational(MT, v))


def window_start(parent, ncoarse):
    """First coarse cell of the 5-cell window for a parent coarse cell (one dimension):
    centred, slid inward at the physical boundary."""
    return int(min(max(parent - 2, 0), ncoarse - WIDTH))


def cfi_values(coarse, coarse_origin, ncoarse, fine_cells, r, D):
    """AMRCFI fine cell averages at the given fine global cells.

    coarse        coarse level array (values needed on every window cell)
    coarse_origin global index of coarse[0,...]
    ncoarse       domain cells per dimension at the coarse level
    fine_cells    int array (n, D) of fine global indices
    Returns (values (n,) or (n, batch), stencil info dict for index-map parity).
    """
    fine_cells = np.asarray(fine_cells, dtype=np.int64)
    n = fine_cells.shape[0]
    parent = np.floor_divide(fine_cells, r)
    sub = fine_cells - r * parent
    start = np.empty_like(parent)
    for d in range(D):
        start[:, d] = [window_start(p, ncoarse[d]) for p in parent[:, d]]
    pos = parent - start
    batch = coarse.shape[D:]
    vals = np.zeros((n,) + batch)
    # weights per dimension: W[d][i, a]
    W = []
    for d in range(D):
        W.append(np.array([[float(w) for w in weights_1d(int(pos[i, d]), int(sub[i, d]), r)]
                           for i in range(n)]).reshape(n, WIDTH))
    for offs in np.ndindex(*([WIDTH] * D)):
        w = np.ones(n)
        idx = []
        for d in range(D):
            w = w * W[d][:, offs[d]]
            idx.append(start[:, d] + offs[d] - coarse_origin[d])
        for d in range(D):
            if np.any(idx[d] < 0) or np.any(idx[d] >= coarse.shape[d]):
                raise ValueError("AMRCFI window leaves the coarse level array")
        cv = coarse[tuple(idx)]
        if not np.all(np.isfinite(cv)):
            raise ValueError("AMRCFI window reads an undefined coarse cell")
        vals = vals + (w.reshape((n,) + (1,) * len(batch)) * cv)
    info = {"start": start, "pos": pos, "sub": sub}
    return vals, info
