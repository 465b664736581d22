"""Transposes of the composite maps G^comp, D^comp, the pure-Neumann solve and the
composite projection (oracle; test infrastructure: only tests, the smoke check and the
benchmark's CPU baseline use this package).

The adjoint of a linear map is its matrix transpose.  Every map here is assembled as a
sparse matrix over the unknowns (the valid cells, ``solve.Unknowns``) by probing the
forward oracle function (``solve.assemble``), and the transpose is that matrix's
transpose; nothing is transposed by hand except the closed form of E^T below.

Composite fields carry values on invalid cells that are averages of their children
(Eq. AMR_avergingDownToCrse; COH-4 for the outputs of G^comp and D^comp).  With E the map
from unknowns to such a field, a weight y on the cells of a composite field is pulled back
to the unknowns by E^T: a valid cell c of level m receives its own weight plus, for every
coarser level l < m, the weight of its ancestor there times r^{-D (m - l)} (each average
spreads its weight uniformly over the r^D children, recursively).

Transposes of maps whose output is a composite field (G^comp, D^comp, the solves) apply
E^T to their input first; their output is a composite field with values on the valid cells
and 0 on the invalid cells (the adjoint of reading only the valid cells).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import composite as cp
from .solve import Unknowns, assemble, helmholtz_matrix


def average_down_transpose(H, Y):
    """E^T Y as a vector over the unknowns (closed form stated in the module docstring)."""
    U = Unknowns(H)
    r, D = H.ratio, H.D
    x = U.gather(Y).astype(np.float64)
    for m in range(1, len(H.levels)):
        cells = U.cells[m]
        if len(cells) == 0:
            continue
        rows = np.arange(U.offsets[m], U.offsets[m + 1])
        for l in range(m):
            lev = H.levels[l]
            anc = cells // (r ** (m - l))
            a = anc - np.asarray(lev.origin)
            x[rows] += Y[l][tuple(a.T)] * float(r) ** (-D * (m - l))
    return x


def gradient_matrices(H, bc_types=None):
    """[G_d]: component d of G^comp (COH-1, 2, 4) as a matrix over the unknowns."""
    return [assemble(H, lambda F, d=d: cp.gradient(H, F, bc_types=bc_types)[d])[0] for d in range(H.D)]


def divergence_matrices(H, bc_types=None):
    """[D_d]: the contribution of velocity component d to D^comp (COH-1..4, refluxing of the
    face values of Eq. cell2face) as a matrix over the unknowns; D^comp w = sum_d D_d w_d."""
    def op(F, d):
        comps = [F if e == d else [np.zeros_like(a) for a in F] for e in range(H.D)]
        return cp.divergence(H, comps, bc_types=bc_types)
    return [assemble(H, lambda F, d=d: op(F, d))[0] for d in range(H.D)]


def gradient_transpose(H, Y, bc_types=None, G=None):
    """(G^comp)^T applied to the D composite fields Y (weights on invalid cells included)."""
    U = Unknowns(H)
    G = gradient_matrices(H, bc_types) if G is None else G
    x = sum(G[d].T @ average_down_transpose(H, Y[d]) for d in range(H.D))
    return U.scatter(x, fill_invalid=False)


def divergence_transpose(H, y, bc_types=None, Dm=None):
    """(D^comp)^T y: one composite field per velocity component."""
    U = Unknowns(H)
    Dm = divergence_matrices(H, bc_types) if Dm is None else Dm
    ey = average_down_transpose(H, y)
    return [U.scatter(Dm[d].T @ ey, fill_invalid=False) for d in range(H.D)]


def neumann_bordered(A, U):
    """The bordered matrix of the pure-Neumann solve: [[A, 1], [w^T, 0]], w = h^D."""
    w = U.weights()
    ones = np.ones((U.n, 1))
    return sp.bmat([[A, sp.csr_matrix(ones)], [sp.csr_matrix(w.reshape(1, -1)), None]], format="csc")


def neumann_solve_transpose(H, G, A=None, U=None):
    """Adjoint of the pure-Neumann solve map f -> phi (Sec. 6.4 solvability correction of f,
    bordered solve, h^D-weighted mean zero of phi).

    With w = h^D over the unknowns and F = I - 1 w^T / (w^T 1), the forward map is
    M = B F, B the unknown block of the bordered inverse; B 1 = 0 and w^T (B y) = 0 make
    M = B = F B.  Hence M^T = B^T: lambda solves [[A^T, w], [1^T, 0]] [lambda; mu] = [g; 0]
    with g = E^T G, i.e. A^T lambda = g - w (1^T g)/(1^T w) and 1^T lambda = 0."""
    if A is None:
        A, U = helmholtz_matrix(H, 0.0, 1.0)
    g = average_down_transpose(H, G)
    x = spla.spsolve(neumann_bordered(A, U).T.tocsc(), np.concatenate([g, [0.0]]))[:-1]
    return U.scatter(x, fill_invalid=False), A, U


def project_transpose(Hn, V, vel_bc_types=None, mats=None):
    """Adjoint of the composite projection u = w - G^comp phi, phi = M D^comp w (Eq.
    comp_ProjOp as ``composite.project`` computes it), as a map on the covered cells of all
    levels of every component: on invalid cells u_d reads w_d directly (no average-down of u,
    Lemma compositeProjection), on valid cells through the chain.  Therefore
        (P^T v)_e = v_e - R^T D_e^T M^T sum_d G_d^T E^T v_d,
    R^T writing the unknowns into the valid cells (0 on invalid cells).
    ``mats``: optional (G, Dm, A, U) from a previous call on the same hierarchy."""
    D = Hn.D
    dirichlet = [0] * (2 * D) if vel_bc_types is None else vel_bc_types
    if mats is None:
        A, U = helmholtz_matrix(Hn, 0.0, 1.0)
        mats = (gradient_matrices(Hn), divergence_matrices(Hn, dirichlet), A, U)
    G, Dm, A, U = mats
    s = sum(G[d].T @ average_down_transpose(Hn, V[d]) for d in range(D))
    lam = spla.spsolve(neumann_bordered(A, U).T.tocsc(), np.concatenate([s, [0.0]]))[:-1]
    out = []
    for e in range(D):
        t = U.scatter(Dm[e].T @ lam, fill_invalid=False)
        out.append([V[e][l] - t[l] for l in range(len(Hn.levels))])
    return out, mats
