"""Single-level fourth-order finite-volume formulas of Sec. 3 (oracle; test infrastructure).

Every coefficient below is the paper's, written as an exact rational:

* Eq. (cell2face): face average and face-averaged normal derivative from cell averages.
* Eq. (discreteOps): the discrete gradient G, divergence D and Laplacian L.
* Eq. (velBCHomoDiri5th): two ghost layers for a Dirichlet face average.
* Eq. (Neumann5): two ghost layers for a Neumann face average (outward normal derivative).

A *level array* ``P`` has one axis per dimension (axis d = paper dimension d, x = 0),
optionally followed by one batch axis.  Its element ``P[a]`` is the cell with global
index ``origin + a``.  The "core" of an array is everything but its outermost two layers
(the two ghost layers of the wrapping paragraph after Eq. (appProj)).
"""
from fractions import Fraction as Fr

import numpy as np

NG = 2  # ghost layers (Sec. 3, wrapping paragraph)

# Eq. (cell2face), face i+1/2 along e^d, keyed by cell offset from i
FACE_VALUE = {-1: Fr(-1, 12), 0: Fr(7, 12), 1: Fr(7, 12), 2: Fr(-1, 12)}
FACE_DERIV = {-1: Fr(1, 12), 0: Fr(-15, 12), 1: Fr(15, 12), 2: Fr(-1, 12)}  # x 1/h

# Eq. (discreteOps a,b): gradient / divergence stencil along e^d (x 1/h)
GRAD = {-2: Fr(1, 12), -1: Fr(-8, 12), 1: Fr(8, 12), 2: Fr(-1, 12)}
# Eq. (discreteOps c): Laplacian stencil along e^d (x 1/h^2)
LAPL = {-2: Fr(-1, 12), -1: Fr(16, 12), 0: Fr(-30, 12), 1: Fr(16, 12), 2: Fr(-1, 12)}

# Eq. (velBCHomoDiri5th).  Interior cells are numbered m = 0..3 inward from the boundary
# face (m = 0 is the cell that owns the face).  ghost = sum_m c[m] phi_m + b * <phi>_face
DIRICHLET = {
    1: ([Fr(-77, 12), Fr(43, 12), Fr(-17, 12), Fr(3, 12)], Fr(5)),
    2: ([Fr(-505, 12), Fr(335, 12), Fr(-145, 12), Fr(27, 12)], Fr(75, 3)),
}
# Eq. (Neumann5).  ghost = sum_m c[m] phi_m + b * h * <d phi / d n>_face  (n outward)
NEUMANN = {
    1: ([Fr(5, 10), Fr(9, 10), Fr(-5, 10), Fr(1, 10)], Fr(6, 5)),
    2: ([Fr(-75, 10), Fr(145, 10), Fr(-75, 10), Fr(15, 10)], Fr(6)),
}

BC_DIRICHLET = 0
BC_NEUMANN = 1


def _core(P, D, shift=None):
    """View of the core of ``P`` shifted by ``shift = (d, k)`` cells along axis d."""
    idx = []
    for a in range(D):
        k = shift[1] if (shift is not None and shift[0] == a) else 0
        idx.append(slice(NG + k, P.shape[a] - NG + k))
    return P[tuple(idx)]


def _embed(core, like, D):
    """Place a core-shaped result into a NaN array shaped like ``like``."""
    out = np.full(like.shape, np.nan)
    out[tuple(slice(NG, like.shape[a] - NG) for a in range(D))] = core
    return out


def laplacian(P, D, h):
    """Eq. (discreteOps c) on every core cell of ``P`` (ghosts must be filled)."""
    acc = np.zeros(_core(P, D).shape)
    for d in range(D):
        v = lambda k: _core(P, D, (d, k))
        acc = acc + (-v(2) + 16.0 * v(1) - 30.0 * v(0) + 16.0 * v(-1) - v(-2)) / (12.0 * h * h)
    return _embed(acc, P, D)


def helmholtz(P, D, h, alpha, beta):
    """``alpha*phi + beta*L phi`` (the operator I - gamma*nu*k*L of Eq. (GePUP-IMEX b)
    has alpha = 1, beta = -gamma*nu*k; the PPE has alpha = 0, beta = 1)."""
    return alpha * P + beta * laplacian(P, D, h) if alpha != 0.0 else beta * laplacian(P, D, h)


def gradient(P, D, h, d):
    """Component d of Eq. (discreteOps a) on every core cell."""
    v = lambda k: _core(P, D, (d, k))
    return _embed((-v(2) + 8.0 * v(1) - 8.0 * v(-1) + v(-2)) / (12.0 * h), P, D)


def divergence(U, D, h):
    """Eq. (discreteOps b); ``U`` is a list of D level arrays (velocity components)."""
    acc = np.zeros(_core(U[0], D).shape)
    for d in range(D):
        v = lambda k: _core(U[d], D, (d, k))
        acc = acc + (-v(2) + 8.0 * v(1) - 8.0 * v(-1) + v(-2)) / (12.0 * h)
    return _embed(acc, U[0], D)


def face_flux_deriv(P, D, h, d, cell):
    """Eq. (cell2face), second line: <d phi/dx_d> on the high face of global-array index
    ``cell`` (a tuple of array indices, or index arrays)."""
    acc = 0.0
    for k, c in FACE_DERIV.items():
        idx = list(cell)
        idx[d] = idx[d] + k
        acc = acc + float(c) * P[tuple(idx)]
    return acc / h


def face_value(P, D, d, cell):
    """Eq. (cell2face), first line: <phi> on the high face of array index ``cell``."""
    acc = 0.0
    for k, c in FACE_VALUE.items():
        idx = list(cell)
        idx[d] = idx[d] + k
        acc = acc + float(c) * P[tuple(idx)]
    return acc


def fill_physical_ghosts(P, origin, ndom, covered, D, h, bc_types, bc_data=None, corners=False):
    """Fill the two ghost layers outside the physical domain, Eqs. (velBCHomoDiri5th) and
    (Neumann5).  Ghosts are set along each face normal only; ghost cells that are outside
    the domain in two or more dimensions (corners) are never read by the axis-aligned
    stencils and are left untouched.

    P        level array (modified in place), may carry a trailing batch axis
    origin   global index of P[0,...,0]
    ndom     number of cells of the domain at this level, per dimension
    covered  bool array over P's spatial shape: cells of the level's boxes
    bc_types list of 2*D ints, face f = 2*d + side (side 0 = low, 1 = high)
    bc_data  None (homogeneous) or dict f -> array over the face's transverse cells
             (the domain's cells at this level with dimension d removed); Dirichlet data are
             face averages of phi, Neumann data face averages of the OUTWARD normal derivative
    corners  also fill ghosts outside the domain in several dimensions by applying the
             formulas dimension after dimension to already-filled ghosts (Fig. 1(c): the
             triangle ghosts are filled after the others).  Only prolongation reads these;
             requires homogeneous data.
    """
    filled = covered.copy()
    for d in range(D):
        for side in (0, 1):
            f = 2 * d + side
            # array index of the interior cell that owns the boundary face
            g_face_cell = 0 if side == 0 else ndom[d] - 1
            a0 = g_face_cell - origin[d]
            inward = 1 if side == 0 else -1
            if a0 < 0 or a0 >= P.shape[d]:
                continue
            if not (0 <= a0 + 3 * inward < P.shape[d]):
                continue

            def sl(a):
                idx = [slice(None)] * P.ndim
                idx[d] = a
                return tuple(idx)

            owner = (filled if corners else covered)[sl(a0)[:D]]
            if not owner.any():
                continue
            interior = [P[sl(a0 + m * inward)] for m in range(4)]
            g = _face_data(bc_data, f, d, origin, P.shape[:D], ndom, D)
            if P.ndim > D and g is not None:
                g = g[..., None]
            for layer in (1, 2):
                if bc_types[f] == BC_DIRICHLET:
                    c, b = DIRICHLET[layer]
                    val = sum(float(c[m]) * interior[m] for m in range(4))
                    if g is not None:
                        val = val + float(b) * g
                else:
                    c, b = NEUMANN[layer]
                    val = sum(float(c[m]) * interior[m] for m in range(4))
                    if g is not None:
                        val = val + float(b) * h * g
                ag = a0 - layer * inward
                tgt = P[sl(ag)]
                if P.ndim > D:
                    tgt[owner, ...] = val[owner, ...]
                else:
                    tgt[owner] = val[owner]
                if corners:
                    filled[sl(ag)[:D]] |= owner


def _face_data(bc_data, f, d, origin, shape, ndom, D):
    """BC data of face f restricted to the transverse window of a level array (zero
    outside the domain; those positions are never covered)."""
    if bc_data is None or bc_data.get(f) is None:
        return None
    src = np.asarray(bc_data[f], dtype=np.float64)
    tdims = [a for a in range(D) if a != d]
    out = np.zeros([shape[a] for a in tdims])
    # overlap of [origin, origin+shape) with [0, ndom) for each transverse dim
    dst_idx, src_idx = [], []
    for t, a in enumerate(tdims):
        lo = max(origin[a], 0)
        hi = min(origin[a] + shape[a], ndom[a])
        dst_idx.append(slice(lo - origin[a], hi - origin[a]))
        src_idx.append(slice(lo, hi))
    out[tuple(dst_idx)] = src[tuple(src_idx)]
    return out
