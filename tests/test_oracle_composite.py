"""Pins of the oracle's AMR pieces (Sec. 5) against mathematics (no GPU).

* AMRCFI: exact on cell averages of every polynomial of degree <= 4 (fifth order), not on
  degree 5, and exactly conservative (Sec. 5.2).
* Composite operators: on cell averages of a degree-4 polynomial (which are redundant by
  construction) the composite Laplacian with refluxing reproduces the cell averages of the
  exact Laplacian on every valid cell, near the physical boundary too (clipped windows).
* Pure Neumann: the composite operator annihilates constants and its columns sum to zero
  with the h^D weights (refluxing telescopes the fluxes: the discrete form of the
  solvability condition of Sec. 6.4).
* Assembly by coloured probing equals brute-force assembly by unit vectors.
"""
import itertools
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import cfi, composite as cp, solve as so
from oracle.hierarchy import Hierarchy
from paper_2506_02663_gb300.workloads import cell_average_gauss, face_average_gauss


@pytest.mark.parametrize("r", [2, 4])
def test_cfi_weights_exact_and_conservative(r):
    X0 = Fr(2, 7)

    def cavg(p, a, b):
        return ((b + X0) ** (p + 1) - (a + X0) ** (p + 1)) / ((p + 1) * (b - a))

    for pos in range(5):
        for p in range(6):
            coarse = [cavg(p, Fr(a), Fr(a + 1)) for a in range(5)]
            fine = []
            for sub in range(r):
                w = cfi.weights_1d(pos, sub, r)
                v = sum(wa * ca for wa, ca in zip(w, coarse))
                ex = cavg(p, Fr(pos) + Fr(sub, r), Fr(pos) + Fr(sub + 1, r))
                assert (v == ex) == (p <= 4), (pos, p, sub)
                fine.append(v)
            assert sum(fine) / r == coarse[pos]  # conservation, Eq. AMR_avergingDownToCrse


def _quartic(D):
    if D == 2:
        f = lambda x, y: 0.5 + x - 2 * y + 3 * x * y - x ** 2 * y ** 2 + 2 * x ** 3 * y - y ** 4 + 0.7 * x ** 4
        lap = lambda x, y: -2 * y ** 2 + 12 * x * y - 12 * y ** 2 - 2 * x ** 2 + 8.4 * x ** 2
        gx = lambda x, y: 1 + 3 * y - 2 * x * y ** 2 + 6 * x ** 2 * y + 2.8 * x ** 3
        gy = lambda x, y: -2 + 3 * x - 2 * x ** 2 * y + 2 * x ** 3 - 4 * y ** 3
        return f, lap, (gx, gy)
    f = lambda x, y, z: 1 + x * y * z + x ** 2 * z ** 2 - y ** 4 + 2 * x ** 3 * y
    lap = lambda x, y, z: 2 * z ** 2 + 2 * x ** 2 - 12 * y ** 2 + 12 * x * y
    gx = lambda x, y, z: y * z + 2 * x * z ** 2 + 6 * x ** 2 * y
    gy = lambda x, y, z: x * z - 4 * y ** 3 + 2 * x ** 3
    gz = lambda x, y, z: x * y + 2 * x ** 2 * z
    return f, lap, (gx, gy, gz)


def _fill_exact(H, func):
    F = cp.new_field(H)
    for l, lev in enumerate(H.levels):
        vals = cell_average_gauss(func, lev.ndom, lev.h, origin=lev.origin, shape=lev.shape)
        F[l][lev.covered] = vals[lev.covered]
    return F


def _face_data(H, func_of_d_side):
    data = []
    for lev in H.levels:
        data.append({2 * d + s: face_average_gauss(func_of_d_side(d, s), lev.ndom, lev.h, d, s)
                     for d in range(H.D) for s in (0, 1)})
    return data


HIER_2D = [
    # two levels, box away from the boundary
    [[((0, 0), (15, 15))], [((8, 8), (23, 23))]],
    # box touching the low x boundary and the high y boundary: clipped windows
    [[((0, 0), (15, 15))], [((0, 12), (11, 31))]],
    # two boxes on level 1 sharing a face (same-level copy ghosts) plus a level-2 box
    [[((0, 0), (15, 15))], [((4, 4), (15, 19)), ((16, 4), (27, 19))], [((16, 16), (39, 27))]],
]


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("boxes", HIER_2D)
def test_composite_laplacian_exact_on_quartic(boxes, bc):
    f, lap, grad = _quartic(2)
    H = Hierarchy(2, (16, 16), boxes, bc=[bc] * 4)
    phi = _fill_exact(H, f)
    if bc == 0:
        data = _face_data(H, lambda d, s: f)
    else:
        data = _face_data(H, lambda d, s: (lambda *x: (1.0 if s else -1.0) * grad[d](*x)))
    Y = cp.apply(H, phi, 0.0, 1.0, data)
    ex = _fill_exact(H, lap)
    scale = max(np.max(np.abs(ex[l][lev.valid])) for l, lev in enumerate(H.levels))
    for l, lev in enumerate(H.levels):
        err = np.max(np.abs(Y[l][lev.valid] - ex[l][lev.valid]))
        assert err < 1e-8 * scale, (l, err)


def test_composite_laplacian_3d_exact_on_quartic():
    f, lap, grad = _quartic(3)
    H = Hierarchy(3, (8, 8, 8), [[((0,) * 3, (7,) * 3)], [((4, 0, 6), (11, 7, 15))]], bc=[0] * 6)
    phi = _fill_exact(H, f)
    data = _face_data(H, lambda d, s: f)
    Y = cp.apply(H, phi, 0.0, 1.0, data)
    ex = _fill_exact(H, lap)
    for l, lev in enumerate(H.levels):
        assert np.max(np.abs(Y[l][lev.valid] - ex[l][lev.valid])) < 1e-8 * np.max(np.abs(ex[l][lev.valid]))


def test_composite_cfi_not_exact_for_degree_5():
    """The CF ghosts carry the degree-4 limit: a degree-5 field breaks exactness next to the
    interface (and only there), which shows the window is really used."""
    H = Hierarchy(2, (16, 16), HIER_2D[0], bc=[0, 0, 0, 0])
    f = lambda x, y: x ** 5
    P = _fill_exact(H, f)
    cp.fill_cf_ghosts(H, P, 1)
    lev = H.levels[1]
    ex = cell_average_gauss(f, lev.ndom, lev.h, origin=lev.origin, shape=lev.shape)
    err = np.abs(P[1][lev.cf_ghost] - ex[lev.cf_ghost])
    assert err.max() > 1e-9


@pytest.mark.parametrize("boxes", HIER_2D)
def test_composite_gradient_divergence_exact(boxes):
    f, lap, grad = _quartic(2)
    H = Hierarchy(2, (16, 16), boxes, bc=[0] * 4)
    phi = _fill_exact(H, f)
    data = _face_data(H, lambda d, s: f)
    G = cp.gradient(H, phi, data)
    for d in range(2):
        ex = _fill_exact(H, grad[d])
        for l, lev in enumerate(H.levels):
            assert np.max(np.abs(G[d][l][lev.valid] - ex[l][lev.valid])) < 1e-9
    # D^comp of the (quartic) gradient field: only degree <= 3 components are exact for
    # face values (Eq. cell2face), so use a cubic velocity u = (x^3 y, x y^2 - y^3)
    u = [lambda x, y: x ** 3 * y, lambda x, y: x * y ** 2 - y ** 3]
    divu = lambda x, y: 3 * x ** 2 * y + 2 * x * y - 3 * y ** 2
    U = [_fill_exact(H, u[d]) for d in range(2)]
    bcu = [_face_data(H, (lambda dd: (lambda d, s: u[dd]))(dd)) for dd in range(2)]
    Y = cp.divergence(H, U, bcu)
    ex = _fill_exact(H, divu)
    for l, lev in enumerate(H.levels):
        assert np.max(np.abs(Y[l][lev.valid] - ex[l][lev.valid])) < 1e-9


@pytest.mark.parametrize("boxes", HIER_2D)
def test_neumann_composite_null_vectors(boxes):
    H = Hierarchy(2, (16, 16), boxes, bc=[1] * 4)
    A, U = so.helmholtz_matrix(H, 0.0, 1.0)
    w = U.weights()
    scale = np.abs(A).max()
    assert np.abs(A @ np.ones(U.n)).max() < 1e-12 * scale
    assert np.abs(w @ A).max() < 1e-15 * scale
    # Dirichlet: no constant null vector
    Hd = Hierarchy(2, (16, 16), boxes, bc=[0] * 4)
    Ad, Ud = so.helmholtz_matrix(Hd, 0.0, 1.0)
    assert np.abs(Ad @ np.ones(Ud.n)).max() > 1.0


def test_assembly_matches_unit_vector_brute_force():
    H = Hierarchy(2, (8, 8), [[((0, 0), (7, 7))], [((4, 2), (11, 15))]], bc=[0, 1, 0, 1])
    A, U = so.helmholtz_matrix(H, 1.0, -0.01)
    dense = np.zeros((U.n, U.n))
    for j in range(U.n):
        e = np.zeros(U.n)
        e[j] = 1.0
        dense[:, j] = U.gather(cp.apply(H, U.scatter(e), 1.0, -0.01))
    assert np.array_equal(A.toarray(), dense)


def test_average_down_redundancy_of_exact_averages():
    """Exact cell averages are redundant: average-down of level l+1 reproduces level l."""
    f, _, _ = _quartic(2)
    H = Hierarchy(2, (16, 16), HIER_2D[2], bc=[0] * 4)
    F = _fill_exact(H, f)
    G = [a.copy() for a in F]
    cp.average_down_all(H, G)
    for l, lev in enumerate(H.levels):
        assert np.max(np.abs(G[l][lev.covered] - F[l][lev.covered])) < 1e-13
