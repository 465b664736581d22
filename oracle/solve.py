"""Composite linear systems: unknowns, sparse assembly, direct solves, solvability,
mean-zero and transposes (oracle; test infrastructure).

The multigrid solver only reaches the exact solution of the composite system faster, so
the oracle's answer is that exact solution, phi* = A^{-1} f, computed by a sparse direct
solve (a library primitive used as one step).  The system is defined as follows:

* unknowns: the valid cells of every level (Eq. validRegion); invalid cells are not
  unknowns, their values are the average of their children (Eq. AMR_avergingDownToCrse);
* equations: one per valid cell, the composite operator of COH-1..4 (``composite.apply``);
* pure Neumann PPE (alpha = 0, all faces Neumann): the right-hand side is first made
  compatible by the uniform correction of Sec. 6.4 (Eq. correctingFaceAvg applied to the
  RHS, as the paragraph after it states for the PPE), and the solution is the one with
  zero h^D-weighted mean over the valid cells (bordered system).

The assembled matrix is obtained by probing the linear map ``composite.apply`` with
coloured indicator vectors; ``A @ x == apply(x)`` is checked in the tests.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import composite as cp

PROBE_PERIOD = 40  # colour period; couplings span fewer than PROBE_PERIOD/2 cells


class Unknowns:
    """Valid cells numbered level by level, box by box, x fastest inside a box."""

    def __init__(self, H):
        self.H = H
        self.index = []
        self.level_of = []
        self.cells = []  # per level (n_l, D) global cell indices in unknown order
        n = 0
        for l, lev in enumerate(H.levels):
            idx = np.full(lev.shape, -1, np.int64)
            cells_l = []
            for lo, hi in lev.boxes:
                s = lev.box_slice(lo, hi)
                sub = lev.valid[s]
                # x-fastest order == Fortran order over (x, y, z) axes
                loc = np.argwhere(sub.transpose())[:, ::-1]  # C-order over (z,y,x) -> (x,y,z)
                g = loc + np.asarray(lo)
                cells_l.append(g)
                a = g - np.asarray(lev.origin)
                idx[tuple(a.T)] = np.arange(n, n + len(g))
                n += len(g)
            self.index.append(idx)
            self.cells.append(np.concatenate(cells_l) if cells_l else np.zeros((0, H.D), int))
            self.level_of.append(l)
        self.n = n
        self.offsets = np.cumsum([0] + [len(c) for c in self.cells])

    def scatter(self, x, fill_invalid=True):
        """Vector (n,) or (n, B) -> composite field (invalid cells averaged down)."""
        x = np.asarray(x, dtype=np.float64)
        batch = x.shape[1:]
        F = cp.new_field(self.H, batch, 0.0)
        for l, lev in enumerate(self.H.levels):
            m = self.index[l] >= 0
            F[l][m] = x[self.index[l][m]]
        if fill_invalid:
            cp.average_down_all(self.H, F)
        return F

    def gather(self, F):
        """Composite field -> vector over the valid cells."""
        batch = F[0].shape[self.H.D:]
        x = np.zeros((self.n,) + batch)
        for l in range(len(self.H.levels)):
            m = self.index[l] >= 0
            x[self.index[l][m]] = F[l][m]
        return x

    def weights(self):
        """h^D of every unknown (the composite L_p norms of Sec. 7 use these)."""
        w = np.zeros(self.n)
        for l, lev in enumerate(self.H.levels):
            w[self.offsets[l]:self.offsets[l + 1]] = lev.h ** self.H.D
        return w


def assemble(H, op, period=PROBE_PERIOD, chunk=256):
    """Sparse matrix of the linear map ``op`` (composite field -> composite field) over the
    valid cells.  Unknowns of one level whose global indices agree modulo ``period`` share
    a probe; each nonzero of a probe's response is attributed to the unique unknown of that
    colour within period/2 cells of the row (in the probed level's index space)."""
    U = Unknowns(H)
    r = H.ratio
    rows_all, cols_all, vals_all = [], [], []
    row_level = np.concatenate([np.full(len(U.cells[l]), l) for l in range(len(H.levels))])
    row_cells = np.concatenate(U.cells)
    for lp, lev in enumerate(H.levels):
        cells = U.cells[lp]
        if len(cells) == 0:
            continue
        ids = np.arange(U.offsets[lp], U.offsets[lp + 1])
        col_of = {tuple(c): j for c, j in zip(cells, ids)}
        color = np.mod(cells, period)
        keys = np.ravel_multi_index(tuple(color.T), (period,) * H.D)
        uniq = np.unique(keys)
        # row positions expressed in level-lp index space
        pos = np.empty_like(row_cells, dtype=np.float64)
        for l in range(len(H.levels)):
            m = row_level == l
            f = float(r) ** (lp - l)
            pos[m] = (row_cells[m] + 0.5) * f - 0.5
        for c0 in range(0, len(uniq), chunk):
            cols = uniq[c0:c0 + chunk]
            X = np.zeros((U.n, len(cols)))
            for b, key in enumerate(cols):
                X[ids[keys == key], b] = 1.0
            Y = U.gather(op(U.scatter(X)))
            for b, key in enumerate(cols):
                nz = np.nonzero(Y[:, b])[0]
                if len(nz) == 0:
                    continue
                cc = np.array(np.unravel_index(key, (period,) * H.D)).reshape(1, -1)
                p = pos[nz]
                # the unique g == cc (mod period) nearest to p
                g = cc + np.round((p - cc) / period).astype(np.int64) * period
                ok = []
                for i, gi in zip(nz, g):
                    j = col_of.get(tuple(gi))
                    if j is None:
                        raise RuntimeError("probe response outside any coupled unknown")
                    ok.append(j)
                rows_all.append(nz)
                cols_all.append(np.asarray(ok))
                vals_all.append(Y[nz, b])
    A = sp.csr_matrix((np.concatenate(vals_all), (np.concatenate(rows_all), np.concatenate(cols_all))),
                      shape=(U.n, U.n))
    return A, U


def helmholtz_matrix(H, alpha, beta):
    """Assembled composite alpha*I + beta*L^comp with homogeneous physical data."""
    return assemble(H, lambda F: cp.apply(H, F, alpha, beta, None))


def affine_part(H, alpha, beta, bc_data, U):
    """A^comp applied to the zero field with the given boundary data (the affine part)."""
    return U.gather(cp.apply(H, cp.new_field(H), alpha, beta, bc_data))


def is_pure_neumann(H, alpha):
    return alpha == 0.0 and all(b == 1 for b in H.bc)


def fsum_weighted(values, weights):
    """Exactly rounded sum of values*weights (Python's math.fsum, Shewchuk's algorithm);
    the products are rounded once each."""
    return math.fsum(float(v) * float(w) for v, w in zip(np.ravel(values), np.ravel(weights)))


def boundary_flux_sum(H, bc_data):
    """sum over physical faces of valid boundary cells of h^(D-1) * (Neumann datum)."""
    if bc_data is None:
        return 0.0
    terms = []
    D = H.D
    for l, lev in enumerate(H.levels):
        if bc_data[l] is None:
            continue
        for d in range(D):
            for side in (0, 1):
                f = 2 * d + side
                g = bc_data[l].get(f)
                if g is None:
                    continue
                gi = 0 if side == 0 else lev.ndom[d] - 1
                a = gi - lev.origin[d]
                if a < 0 or a >= lev.shape[d]:
                    continue
                idx = [slice(None)] * D
                idx[d] = a
                vmask = lev.valid[tuple(idx)]
                # transverse global indices of the window
                tdims = [e for e in range(D) if e != d]
                sub = np.argwhere(vmask)
                for t in sub:
                    gt = tuple(int(t[k] + lev.origin[e]) for k, e in enumerate(tdims))
                    terms.append(float(np.asarray(g)[gt]) * lev.h ** (D - 1))
    return math.fsum(terms)


def solvability_fix(H, f, beta=1.0, bc_data=None):
    """Sec. 6.4 (Eq. correctingFaceAvg, applied to the PPE right-hand side): subtract from
    f on every valid cell the constant m with
        m * sum_valid h^D = sum_valid h^D f - beta * sum_boundary h^(D-1) g.
    Returns (corrected field, m).  One component: the composite domain is connected."""
    U = Unknowns(H)
    x = U.gather(f)
    w = U.weights()
    vol = math.fsum(w)
    m = (fsum_weighted(x, w) - beta * boundary_flux_sum(H, bc_data)) / vol
    out = [a.copy() for a in f]
    for l, lev in enumerate(H.levels):
        out[l][lev.valid] = out[l][lev.valid] - m
    return out, m


def mean_zero(H, phi):
    """Subtract the h^D-weighted mean over the valid cells; invalid cells follow by
    average-down."""
    U = Unknowns(H)
    x = U.gather(phi)
    w = U.weights()
    mean = fsum_weighted(x, w) / math.fsum(w)
    return U.scatter(x - mean), mean


def solve_direct(H, f, alpha, beta, bc_data=None, A=None, U=None):
    """phi* = A^{-1}(f - affine part) over the valid cells; pure Neumann: bordered with the
    h^D-weighted mean constraint (f must already be compatible)."""
    if A is None:
        A, U = helmholtz_matrix(H, alpha, beta)
    rhs = U.gather(f) - (affine_part(H, alpha, beta, bc_data, U) if bc_data is not None else 0.0)
    if is_pure_neumann(H, alpha):
        w = U.weights()
        ones = np.ones((U.n, 1))
        Ab = sp.bmat([[A, sp.csr_matrix(ones)], [sp.csr_matrix(w.reshape(1, -1)), None]], format="csc")
        x = spla.spsolve(Ab, np.concatenate([rhs, [0.0]]))[:-1]
    else:
        x = spla.spsolve(A.tocsc(), rhs)
    return U.scatter(x), A, U


def solve_transpose_direct(H, g, alpha, beta, A=None, U=None):
    """lambda = A^{-T} g over the valid cells (homogeneous data): the adjoint solve."""
    if A is None:
        A, U = helmholtz_matrix(H, alpha, beta)
    x = spla.spsolve(A.T.tocsc(), U.gather(g))
    return U.scatter(x, fill_invalid=False), A, U


def project(Hn, W, bc_w=None):
    """Composite projection u = P^comp w = w - G^comp (L^comp)^{-1} D^comp w, Eq. (comp_ProjOp).

    Hn    hierarchy whose boundary types are Neumann (the PPE of the projection)
    W     list of D composite fields (velocity components)
    bc_w  None (homogeneous) or per component a list over levels of Dirichlet face data of w
    D^comp uses Dirichlet ghosts for w (COH-1..4 with refluxing); the right-hand side is made
    compatible (Sec. 6.4); phi is the mean-zero solution; G^comp uses homogeneous Neumann
    ghosts and COH-4 on G phi, and no average-down is applied to u afterwards (Lemma
    compositeProjection).  Returns (u components, phi)."""
    D = Hn.D
    dirichlet = [0] * (2 * D)
    psi = cp.divergence(Hn, W, bc_data=bc_w, bc_types=dirichlet)
    psi, _ = solvability_fix(Hn, psi)
    phi, _, _ = solve_direct(Hn, psi, 0.0, 1.0)
    phi, _ = mean_zero(Hn, phi)
    G = cp.gradient(Hn, phi)
    U = []
    for d in range(D):
        U.append([W[d][l] - G[d][l] for l in range(len(Hn.levels))])
    return U, phi
