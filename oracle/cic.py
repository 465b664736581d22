"""Coarse-fine interface conditions of the subcycled per-level solves (Sec. 6.3 "Computing
coarse-fine interface conditions", Eq. timeInterp; Sec. 6.4 "Enforcing solvability
conditions", Eq. correctingFaceAvg) -- the time interpolation of the coarse data and the
per-component correction of the interface face averages.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings (the printed passage is inconsistent with itself):
* Eq. (timeInterp) multiplies a 2 x 4 matrix I^(4)(k, eta) with a vector printed as
  phi(t_{-0}), ..., phi(t_{-3}), where t_{-i} = t^{l-1} - i k (caption of the interface
  figure, part (c)) and eta = t* - t_{-1}.  The printed matrix entries are the cubic
  Lagrange weights of the nodes eta = -2k, -k, 0, k in column order, i.e. of t_{-3},
  t_{-2}, t_{-1}, t_{-0}: the columns take the times in increasing order, the reverse of the
  printed vector.  Reading: column j multiplies phi(t_{-(3-j)}); then eta = 0 puts the unit
  weight on t_{-1}, as the definition of eta requires.  The second printed row is the
  eta-derivative of the first: applied to the data it gives d(phi)/dt, although the
  left-hand side names k d(phi)/dt.  ``time_interp_matrix`` returns the printed matrix
  (columns in printed order, nodes ``time_interp_nodes``); ``coarse_time_weights`` the same
  rows for the data in the order t_{-0}, t_{-1}, t_{-2}, t_{-3}; ``scaled=True`` multiplies
  the second row by k.
* Eq. (correctingFaceAvg): on each connected component c of the level, one shift delta_c of
  every interface face average, with -delta_c |faces_I^c| = sum over the interface faces of
  the uncorrected averages + sum over the physical faces of the given ones.
"""
import numpy as np

from . import stencil as st
from .cfi import cfi_values


def time_interp_nodes(k):
    """The times of the four coarse values, relative to eta = 0, in column order."""
    return np.array([-2.0 * k, -k, 0.0, k])


def time_interp_matrix(k, eta, scaled=False):
    """I^(4)(k, eta) of Eq. (timeInterp): row 0 the cubic Lagrange weights of the value at eta,
    row 1 their derivative in eta (times k when ``scaled``), for the four coarse values in
    column order (nodes ``time_interp_nodes(k)``)."""
    x = time_interp_nodes(k)
    M = np.zeros((2, 4))
    for j in range(4):
        others = [x[m] for m in range(4) if m != j]
        den = np.prod([x[j] - xm for xm in others])
        M[0, j] = np.prod([eta - xm for xm in others]) / den
        # derivative of the product of the three factors
        d = 0.0
        for a in range(3):
            d += np.prod([eta - others[b] for b in range(3) if b != a])
        M[1, j] = d / den
    if scaled:
        M[1] *= k
    return M


def printed_time_interp_matrix(k, eta):
    """The entries of Eq. (timeInterp) as printed (the common factor 1 / (6 k^3) applied to
    both rows), for comparison with ``time_interp_matrix``."""
    e = eta
    r0 = [-e ** 3 + k ** 2 * e, 3 * e ** 3 + 3 * k * e ** 2 - 6 * k ** 2 * e,
          -3 * e ** 3 - 6 * k * e ** 2 + 3 * k ** 2 * e + 6 * k ** 3, e ** 3 + 3 * k * e ** 2 + 2 * k ** 2 * e]
    r1 = [-3 * e ** 2 + k ** 2, 9 * e ** 2 + 6 * k * e - 6 * k ** 2, -9 * e ** 2 - 12 * k * e + 3 * k ** 2,
          3 * e ** 2 + 6 * k * e + 2 * k ** 2]
    return np.array([r0, r1]) / (6.0 * k ** 3)


def time_interpolate(values, k, eta, scaled=False):
    """[phi(t*), d(phi)/dt(t*) (times k when scaled)] from the four coarse values (arrays of
    any equal shape, in the matrix's column order)."""
    M = time_interp_matrix(k, eta, scaled)
    v = np.stack([np.asarray(a, dtype=np.float64) for a in values])
    return np.tensordot(M, v, axes=(1, 0))


def coarse_time_weights(k, eta, scaled=False):
    """The rows of I^(4)(k, eta) for the data in the order phi(t_{-0}), phi(t_{-1}),
    phi(t_{-2}), phi(t_{-3}) with t_{-i} = t^{l-1} - i k and eta = t* - t_{-1}: column j of
    the printed matrix belongs to t_{-(3-j)}."""
    return time_interp_matrix(k, eta, scaled)[:, ::-1]


def interpolate_coarse_times(values, k, eta, scaled=False):
    """[phi(t*), d(phi)/dt(t*)] from the data at t_{-0}, t_{-1}, t_{-2}, t_{-3} in that
    order."""
    M = coarse_time_weights(k, eta, scaled)
    v = np.stack([np.asarray(a, dtype=np.float64) for a in values])
    return np.tensordot(M, v, axes=(1, 0))


def correct_face_averages(interface, physical_sum):
    """Eq. (correctingFaceAvg) on one connected component: ``interface`` the uncorrected
    interface face averages (n . w), ``physical_sum`` the sum of the physical faces' given
    averages; returns (corrected averages, delta) with sum(corrected) + physical_sum = 0."""
    a = np.asarray(interface, dtype=np.float64)
    delta = -(np.sum(a) + physical_sum) / a.size
    return a + delta, delta


def correct_by_component(interface, component, physical_sums):
    """The correction on every component: ``component[i]`` labels interface face i,
    ``physical_sums[c]`` the physical-face sum of component c (0 when it has none)."""
    a = np.asarray(interface, dtype=np.float64).copy()
    lab = np.asarray(component)
    deltas = {}
    for c in np.unique(lab):
        sel = lab == c
        a[sel], deltas[int(c)] = correct_face_averages(a[sel], physical_sums.get(int(c), 0.0))
    return a, deltas


def interface_ghost_values(H, coarse_times, l, k, eta):
    """CIC-2 and CIC-3 on the CF ghost cells of level l: AMRCFI (Sec. 5.2) of each of the four
    coarse level arrays ``coarse_times`` (level l-1 at t_{-0}, t_{-1}, t_{-2}, t_{-3} in that
    order; redundant data on covered coarse cells), then Eq. (timeInterp) at t* = t_{-1} +
    eta.  Returns (cells, value, rate): the array indices of level l's CF ghosts (np.argwhere
    order), the interpolated values and their time derivatives (the printed second row)."""
    lev, crs = H.levels[l], H.levels[l - 1]
    cells = np.argwhere(lev.cf_ghost)
    g = cells + np.asarray(lev.origin)
    fine = [cfi_values(c, crs.origin, crs.ndom, g, H.ratio, H.D)[0] for c in coarse_times]
    value, rate = interpolate_coarse_times(fine, k, eta)
    return cells, value, rate


def interface_faces(H, l):
    """The coarse-fine interface faces of level l: faces between a cell of the level's boxes
    and a CF ghost cell.  Returns a list of (cell, d, s, component): the array index of the
    interior cell, the normal dimension, the side (+1: the cell's high face, outward normal
    +e_d) and the connected component of the cell's box (Sec. 5.1; components numbered in
    ascending order of their smallest box index)."""
    lev = H.levels[l]
    labels = H.components(l)
    order = sorted(set(labels))
    comp_of_box = [order.index(labels[b]) for b in range(len(labels))]
    out = []
    for d in range(H.D):
        for s in (1, -1):
            for c in np.argwhere(lev.covered):
                nb = c.copy()
                nb[d] += s
                if 0 <= nb[d] < lev.shape[d] and lev.cf_ghost[tuple(nb)]:
                    out.append((tuple(int(v) for v in c), d, s, comp_of_box[int(lev.patch[tuple(c)])]))
    return out


def interface_face_averages(H, W, l, faces=None):
    """n . <w> on the interface faces of level l (``W``: the D level-l arrays of the velocity
    components with their ghosts filled): Eq. (cell2face) on the face along its normal."""
    faces = interface_faces(H, l) if faces is None else faces
    out = np.empty(len(faces))
    for i, (c, d, s, _) in enumerate(faces):
        lowcell = list(c)
        if s < 0:
            lowcell[d] -= 1  # the face is the high face of the cell below it
        out[i] = s * st.face_value(W[d], H.D, d, tuple(lowcell))
    return out


def interface_face_values(H, X, l, faces=None):
    """<x> on the interface faces of level l (``X``: the level-l array of a field with its
    ghosts filled): Eq. (cell2face) on each face along its normal, no sign."""
    faces = interface_faces(H, l) if faces is None else faces
    out = np.empty(len(faces))
    for i, (c, d, s, _) in enumerate(faces):
        lowcell = list(c)
        if s < 0:
            lowcell[d] -= 1
        out[i] = st.face_value(X, H.D, d, tuple(lowcell))
    return out


def component_box(H, l, comp):
    """The level problem of Def. GePUP-E-OneLevel on a component that is one box: (lo, hi,
    interface flags per face 2d+side: 1 where the box face is interior to the domain, i.e. on
    the coarse-fine interface).  Raises ValueError for a component of several boxes."""
    lev = H.levels[l]
    labels = H.components(l)
    order = sorted(set(labels))
    boxes = [b for b in range(len(labels)) if order.index(labels[b]) == comp]
    if len(boxes) != 1:
        raise ValueError("component of several boxes")
    lo, hi = lev.boxes[boxes[0]]
    flags = []
    for d in range(H.D):
        flags += [1 if lo[d] > 0 else 0, 1 if hi[d] < lev.ndom[d] - 1 else 0]
    return lo, hi, flags


def box_interface_bc(H, X, l, comp):
    """Boundary data of the one-level box problem of a single-box component: for each face
    f = 2d+side of the box, an array over the box face (remaining dimensions in order) holding
    the interface face averages <x> (zeros on faces on the physical boundary)."""
    lo, hi, _ = component_box(H, l, comp)
    D = H.D
    n = [hi[e] - lo[e] + 1 for e in range(D)]
    lev = H.levels[l]
    data = {2 * d + s: np.zeros(tuple(n[e] for e in range(D) if e != d)) for d in range(D) for s in (0, 1)}
    faces = [f for f in interface_faces(H, l) if f[3] == comp]
    vals = interface_face_values(H, X, l, faces)
    for (c, d, s, _), v in zip(faces, vals):
        g = [c[e] + lev.origin[e] - lo[e] for e in range(D)]
        data[2 * d + (1 if s > 0 else 0)][tuple(g[e] for e in range(D) if e != d)] = v
    return data
