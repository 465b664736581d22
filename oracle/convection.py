"""The fourth-order cell-averaged convection operator of Eq. (convOp) (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

<div(uu)>_i = (1/h) sum_d ( F<u_d, u>_{i+e_d/2} - F<u_d, u>_{i-e_d/2} ), with the face average
of a product F<phi, psi> = <phi><psi> + h^2/12 sum_{d' != d} (G_perp_{d'} phi)(G_perp_{d'} psi) at
each face, face averages <phi> from cell averages by Eq. (cell2face), and G_perp_{d'} the
central difference of face averages across the transverse direction d'.

The operator reads, for a cell, the cells two away along each face normal and one away in
each transverse direction of those (corner neighbours included).  Reading: the oracle takes
level arrays whose stencil cells all hold data (tests fill every ghost cell, corners
included, with exact cell averages); cells whose stencil leaves the array come out NaN.
"""
import numpy as np


def _shift(P, d, s):
    """Q with Q[..., k, ...] = P[..., k + s, ...] along axis d (NaN where k + s leaves P)."""
    Q = np.full(P.shape, np.nan)
    n = P.shape[d]
    src = [slice(None)] * P.ndim
    dst = [slice(None)] * P.ndim
    if s >= 0:
        src[d], dst[d] = slice(s, n), slice(0, n - s)
    else:
        src[d], dst[d] = slice(0, n + s), slice(-s, n)
    Q[tuple(dst)] = P[tuple(src)]
    return Q


def face_high(P, d):
    """<phi> on the high face (normal d) of every cell: Eq. (cell2face), first line."""
    return (7.0 * (P + _shift(P, d, 1)) - (_shift(P, d, -1) + _shift(P, d, 2))) / 12.0


def transverse_gradient(Fd, dp, h):
    """(G_perp_{d'} phi) on faces from the face averages Fd of the same orientation."""
    return (_shift(Fd, dp, 1) - _shift(Fd, dp, -1)) / (2.0 * h)


def face_product(phi, psi, d, h, D):
    """F<phi, psi> on the high face (normal d) of every cell."""
    fp, fq = face_high(phi, d), face_high(psi, d)
    out = fp * fq
    for dp in range(D):
        if dp != d:
            out = out + (h * h / 12.0) * transverse_gradient(fp, dp, h) * transverse_gradient(fq, dp, h)
    return out


def convection(U, h):
    """Eq. (convOp): the D components of <div(uu)> from the D level arrays U of <u>."""
    D = len(U)
    out = []
    for c in range(D):
        acc = np.zeros(U[0].shape)
        for d in range(D):
            f = face_product(U[d], U[c], d, h, D)
            acc = acc + (f - _shift(f, d, -1))
        out.append(acc / h)
    return out
