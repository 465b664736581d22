"""Geometric multigrid of Sec. 6.5 (oracle; test infrastructure).

The paper fixes: restriction by "injection", prolongation by linear interpolation, weighted
Jacobi with omega = 2/3, 4 pre- and 4 post-smoothing sweeps (Fig. mg_convergenceRate), and
the max-norm residual stopping test.  Readings taken where it is silent:

* cell-centred data have no coincident points, so "injection" is the r^D volume average
  (the same map as Eq. AMR_avergingDownToCrse);
* linear interpolation is cell-centred tensor-product linear interpolation (weights 3/4, 1/4
  per dimension); coarse ghosts outside the domain are filled by the homogeneous physical
  formulas first;
* the Jacobi diagonal is the true diagonal of the assembled level operator (including the
  ghost-cell coefficients of Eqs. velBCHomoDiri5th / Neumann5); here it is read off the
  operator by probing, by definition;
* coarse multigrid operators are re-discretisations (same formulas, h doubled, same
  boundary types, homogeneous data);
* the bottom solver is a dense direct solve on the coarsest grid (at most 1024 cells); for
  the pure-Neumann operator it is bordered with the mean constraint;
* AMR levels: a composite V-cycle in correction form visits the finest AMR level first,
  smoothing each level with zero coarse-fine ghosts, passes to the next coarser level the
  average of its residual on the invalid region and the composite residual on the valid
  region, runs a single-level V-cycle on all of level 0, then interpolates corrections back
  up and post-smooths.
"""
import numpy as np

from . import composite as cp
from . import stencil as st
from .hierarchy import Hierarchy, mg_grids

NU1 = 4
NU2 = 4
OMEGA = 2.0 / 3.0


def level_apply(H, l, X, alpha, beta, cf="zero", coarse=None):
    """alpha*X + beta*L X on the covered cells of level l with homogeneous physical ghosts
    and CF ghosts either zero or AMRCFI from the coarse level array ``coarse``."""
    lev = H.levels[l]
    P = X.copy()
    if l > 0:
        if cf == "zero":
            P[lev.cf_ghost] = 0.0
        else:
            F = [None] * (l + 1)
            F[l - 1], F[l] = coarse, P
            cp.fill_cf_ghosts(H, F, l)
    st.fill_physical_ghosts(P, lev.origin, lev.ndom, lev.covered, H.D, lev.h, H.bc, None)
    Y = st.helmholtz(P, H.D, lev.h, alpha, beta)
    Y[~lev.covered] = np.nan
    return Y


def jacobi_diagonal(H, l, alpha, beta, period=8):
    """Diagonal of the level-l operator (zero CF ghosts, homogeneous physical ghosts), read
    off by probing with indicator vectors of cells congruent modulo ``period`` (couplings of
    the level operator span at most 3 cells)."""
    lev = H.levels[l]
    diag = np.full(lev.shape, np.nan)
    gidx = np.indices(lev.shape)
    for d in range(H.D):
        gidx[d] += lev.origin[d]
    keys = np.zeros(lev.shape, np.int64)
    for d in range(H.D):
        keys = keys * period + np.mod(gidx[d], period)
    for key in np.unique(keys[lev.covered]):
        m = (keys == key) & lev.covered
        X = np.where(lev.covered, 0.0, np.nan)
        X[m] = 1.0
        Y = level_apply(H, l, X, alpha, beta)
        diag[m] = Y[m]
    return diag


def jacobi(H, l, X, B, diag, alpha, beta, omega=OMEGA):
    """One weighted Jacobi sweep X + omega * (B - A X) / diag on the covered cells."""
    R = B - level_apply(H, l, X, alpha, beta)
    out = X.copy()
    m = H.levels[l].covered
    out[m] = X[m] + omega * R[m] / diag[m]
    return out


def restrict_children(Hf, lf, Xf, Hc, lc, Xc, region_boxes):
    """Volume average of the r^D children (the reading of "injection"), written into the
    coarse cells of ``region_boxes`` (fine-level boxes)."""
    r, D = Hf.ratio, Hf.D
    fine, crs = Hf.levels[lf], Hc.levels[lc]
    for lo, hi in region_boxes:
        block = Xf[fine.box_slice(lo, hi)]
        acc = 0.0
        for offs in np.ndindex(*([r] * D)):
            acc = acc + block[tuple(slice(offs[d], None, r) for d in range(D))]
        Xc[crs.box_slice(tuple(v // r for v in lo), tuple(v // r for v in hi))] = acc / r ** D


def prolong_add(Hc, lc, Xc, Hf, lf, Xf):
    """Xf += cell-centred tensor linear interpolation of Xc on every covered fine cell.
    Xc must carry homogeneous physical ghosts (corners included) where the stencil leaves
    the domain."""
    r, D = Hf.ratio, Hf.D
    assert r == 2
    crs, fine = Hc.levels[lc], Hf.levels[lf]
    cells = np.argwhere(fine.covered)
    g = cells + np.asarray(fine.origin)
    parent = np.floor_divide(g, 2)
    q = g - 2 * parent
    sgn = np.where(q == 0, -1, 1)
    acc = 0.0
    for corner in np.ndindex(*([2] * D)):
        w = np.ones(len(cells))
        idx = []
        for d in range(D):
            w = w * (0.75 if corner[d] == 0 else 0.25)
            idx.append(parent[:, d] + corner[d] * sgn[:, d] - crs.origin[d])
        acc = acc + w * Xc[tuple(idx)]
    Xf[tuple(cells.T)] = Xf[tuple(cells.T)] + acc


class LevelZeroMG:
    """Single-level V-cycle on the whole level-0 grid (re-discretised coarse grids)."""

    def __init__(self, H, alpha, beta, nu1=NU1, nu2=NU2, omega=OMEGA):
        self.alpha, self.beta = alpha, beta
        self.nu1, self.nu2, self.omega = nu1, nu2, omega
        self.grids = []
        for n in mg_grids(H.n0):
            box = [((0,) * H.D, tuple(v - 1 for v in n))]
            self.grids.append(Hierarchy(H.D, n, [box], H.bc, ratio=2, lo=H.lo, hi=H.hi, mg_grid=True))
        self.diag = [jacobi_diagonal(g, 0, alpha, beta) for g in self.grids]
        g = self.grids[-1]
        lev = g.levels[0]
        n = int(np.prod(g.n0))
        cells = np.argwhere(lev.covered)
        A = np.zeros((n, n))
        for j, c in enumerate(cells):
            X = np.where(lev.covered, 0.0, np.nan)
            X[tuple(c)] = 1.0
            A[:, j] = level_apply(g, 0, X, alpha, beta)[tuple(cells.T)]
        self.neumann = alpha == 0.0 and all(b == 1 for b in H.bc)
        if self.neumann:
            A = np.block([[A, np.ones((n, 1))], [np.ones((1, n)), np.zeros((1, 1))]])
        self.bottom = A
        self.bottom_cells = cells

    def bottom_solve(self, b):
        lev = self.grids[-1].levels[0]
        rhs = b[tuple(self.bottom_cells.T)]
        if self.neumann:
            rhs = np.concatenate([rhs, [0.0]])
        x = np.linalg.solve(self.bottom, rhs)
        X = np.where(lev.covered, 0.0, np.nan)
        X[tuple(self.bottom_cells.T)] = x[:len(self.bottom_cells)]
        return X

    def vcycle(self, B, m=0):
        g = self.grids[m]
        if m == len(self.grids) - 1:
            return self.bottom_solve(B)
        lev = g.levels[0]
        X = np.where(lev.covered, 0.0, np.nan)
        for _ in range(self.nu1):
            X = jacobi(g, 0, X, B, self.diag[m], self.alpha, self.beta, self.omega)
        R = B - level_apply(g, 0, X, self.alpha, self.beta)
        gc = self.grids[m + 1]
        Bc = np.where(gc.levels[0].covered, 0.0, np.nan)
        restrict_children(g, 0, R, gc, 0, Bc, g.levels[0].boxes)
        Xc = self.vcycle(Bc, m + 1)
        st.fill_physical_ghosts(Xc, gc.levels[0].origin, gc.levels[0].ndom, gc.levels[0].covered,
                                g.D, gc.levels[0].h, g.bc, None, corners=True)
        prolong_add(gc, 0, Xc, g, 0, X)
        for _ in range(self.nu2):
            X = jacobi(g, 0, X, B, self.diag[m], self.alpha, self.beta, self.omega)
        return X


class CompositeMG:
    """Composite V-cycle over an AMR hierarchy (see module docstring)."""

    def __init__(self, H, alpha, beta, nu1=NU1, nu2=NU2, omega=OMEGA):
        self.H, self.alpha, self.beta = H, alpha, beta
        self.nu1, self.nu2, self.omega = nu1, nu2, omega
        self.mg0 = LevelZeroMG(H, alpha, beta, nu1, nu2, omega)
        self.diag = [None] + [jacobi_diagonal(H, l, alpha, beta) for l in range(1, H.lmax + 1)]

    def _smooth(self, l, X, B, n):
        for _ in range(n):
            X = jacobi(self.H, l, X, B, self.diag[l], self.alpha, self.beta, self.omega)
        return X

    def vcycle(self, phi, f, bc_data=None):
        """One V-cycle; returns the updated composite field (valid cells meaningful)."""
        H, a, b = self.H, self.alpha, self.beta
        L = H.lmax
        phi = [p.copy() for p in phi]
        e = [None] * (L + 1)
        R = [None] * (L + 1)
        R[L] = cp.residual(H, phi, f, a, b, bc_data)[L]
        for l in range(L, 0, -1):
            lev = H.levels[l]
            zero = np.where(lev.covered, 0.0, np.nan)
            e[l] = self._smooth(l, zero, R[l], self.nu1)
            rt = R[l] - level_apply(H, l, e[l], a, b)
            phi[l] = phi[l] + e[l]
            crs = H.levels[l - 1]
            Rc = cp.residual(H, phi, f, a, b, bc_data)[l - 1]
            Rc[crs.invalid] = np.nan
            restrict_children(H, l, rt, H, l - 1, Rc, lev.boxes)
            R[l - 1] = Rc
        e[0] = self.mg0.vcycle(R[0])
        phi[0] = phi[0] + e[0]
        for l in range(1, L + 1):
            lev, crs = H.levels[l], H.levels[l - 1]
            ec = e[l - 1].copy()
            st.fill_physical_ghosts(ec, crs.origin, crs.ndom, crs.covered, H.D, crs.h, H.bc, None,
                                    corners=True)
            dz = np.where(lev.covered, 0.0, np.nan)
            prolong_add(H, l - 1, ec, H, l, dz)
            e[l] = e[l] + dz
            phi[l] = phi[l] + dz
            R[l] = R[l] - level_apply(H, l, e[l], a, b, cf="field", coarse=e[l - 1])
            zero = np.where(lev.covered, 0.0, np.nan)
            dpost = self._smooth(l, zero, R[l], self.nu2)
            e[l] = e[l] + dpost
            phi[l] = phi[l] + dpost
        return phi


def max_norm_valid(H, F):
    """max over valid cells of all levels (Sec. 7, p = infinity)."""
    return max(float(np.max(np.abs(F[l][lev.valid]))) for l, lev in enumerate(H.levels))


def solve(H, f, alpha, beta, bc_data=None, rtol=1e-10, max_cycles=50):
    """V-cycles until ||f - A phi||_inf <= rtol * ||f||_inf over the valid cells.
    Returns (phi, residual history)."""
    mg = CompositeMG(H, alpha, beta)
    phi = cp.new_field(H)
    fn = max_norm_valid(H, f)
    hist = []
    for _ in range(max_cycles + 1):
        res = cp.residual(H, phi, f, alpha, beta, bc_data)
        hist.append(max_norm_valid(H, res))
        if hist[-1] <= rtol * fn:
            break
        phi = mg.vcycle(phi, f, bc_data)
    return phi, hist
