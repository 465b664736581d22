"""Coarse-fine interface conditions of the subcycled per-level solves (Sec. 6.3 "Computing
coarse-fine interface conditions", Eq. timeInterp; Sec. 6.4 "Enforcing solvability
conditions", Eq. correctingFaceAvg) -- the time interpolation of the coarse data and the
per-component correction of the interface face averages.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings (the printed passage is inconsistent with itself):
* Eq. (timeInterp) gives a 2 x 4 matrix I^(4)(k, eta) acting on the coarse values at four
  equispaced times.  Its first row is exactly the cubic Lagrange interpolation with the four
  columns at eta = -2k, -k, 0, k (in the printed column order): the printed entries put
  weight 1 on the third column at eta = 0, although the text defines eta from the time of
  the second column.  The matrix entries win.  Its second row is the eta-derivative of those
  weights: applied to the four values it gives d(phi)/dt, although the left-hand side names
  k d(phi)/dt.  The oracle returns the printed rows (value, d/dt) with the nodes in that
  order; ``time_interp_matrix(..., scaled=True)`` multiplies the second row by k to give
  the quantity the left-hand side names.
* Eq. (correctingFaceAvg): on each connected component c of the level, one shift delta_c of
  every interface face average, with -delta_c |faces_I^c| = sum over the interface faces of
  the uncorrected averages + sum over the physical faces of the given ones.
"""
import numpy as np


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
    any equal shape, in column order)."""
    M = time_interp_matrix(k, eta, scaled)
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
