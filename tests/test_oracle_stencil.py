"""Pins of the oracle's single-level formulas against mathematics (no GPU).

Every formula of Sec. 3 is checked in exact rational arithmetic on cell averages of
monomials: it must be exact up to the degree its stated order implies and fail one degree
above (so a dropped term, a wrong sign or a wrong index cannot pass).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import stencil as st

X0 = Fr(1, 3)  # shift so that no monomial is degenerate at the boundary face


def cavg(p, a, b):
    """Exact average of (x + X0)^p over [a, b]."""
    return ((b + X0) ** (p + 1) - (a + X0) ** (p + 1)) / ((p + 1) * (b - a))


def cell(p, k):
    """Cell k spans [k, k+1] (h = 1)."""
    return cavg(p, Fr(k), Fr(k + 1))


def value_at(p, x):
    return (x + X0) ** p


def deriv_at(p, x):
    return p * (x + X0) ** (p - 1) if p > 0 else Fr(0)


@pytest.mark.parametrize("layer", [1, 2])
def test_dirichlet_ghosts_exact_to_degree_4(layer):
    """Eq. (velBCHomoDiri5th): boundary face at x = 0, interior cells m = 0..3 span
    [-m-1, -m], ghost layer k spans [k-1, k].  Fifth order <=> exact for degree <= 4."""
    c, b = st.DIRICHLET[layer]
    for p in range(7):
        g = sum(c[m] * cell(p, -m - 1) for m in range(4)) + b * value_at(p, Fr(0))
        exact = cell(p, layer - 1)
        if p <= 4:
            assert g == exact, (layer, p)
        else:
            assert g != exact, (layer, p)


@pytest.mark.parametrize("layer", [1, 2])
def test_neumann_ghosts_exact_to_degree_4(layer):
    """Eq. (Neumann5): the datum is the outward normal derivative at the face (h = 1)."""
    c, b = st.NEUMANN[layer]
    for p in range(7):
        g = sum(c[m] * cell(p, -m - 1) for m in range(4)) + b * deriv_at(p, Fr(0))
        exact = cell(p, layer - 1)
        if p <= 4:
            assert g == exact, (layer, p)
        else:
            assert g != exact, (layer, p)


def test_face_formulas_orders():
    """Eq. (cell2face): face value exact to degree 3, face derivative to degree 4 (the
    O(h^4) remainders of the equation), face between cells 0 and 1 at x = 1."""
    for p in range(7):
        v = sum(c * cell(p, k) for k, c in st.FACE_VALUE.items())
        dv = sum(c * cell(p, k) for k, c in st.FACE_DERIV.items())
        assert (v == value_at(p, Fr(1))) == (p <= 3), p
        assert (dv == deriv_at(p, Fr(1))) == (p <= 4), p


def test_discrete_operators_orders():
    """Eq. (discreteOps): G exact to degree 4; L exact to degree 5 on cell averages
    (symmetric stencil); both reproduce cell averages of the derivative."""
    for p in range(8):
        g = sum(c * cell(p, k) for k, c in st.GRAD.items())
        lap = sum(c * cell(p, k) for k, c in st.LAPL.items())
        dex = (value_at(p, Fr(1)) - value_at(p, Fr(0)))  # average of the derivative over cell 0
        d2ex = deriv_at(p, Fr(1)) - deriv_at(p, Fr(0))
        assert (g == dex) == (p <= 4), p
        assert (lap == d2ex) == (p <= 5), p


def test_laplacian_is_difference_of_face_derivatives():
    """L = (F_{i+1/2} - F_{i-1/2}) / h with F of Eq. (cell2face): the flux form the
    refluxing step (COH-3) relies on, for arbitrary cell values."""
    vals = [Fr(3), Fr(-7), Fr(11), Fr(2), Fr(5), Fr(-1)]  # cells -2..3
    cellv = lambda k: vals[k + 2]
    lap = sum(c * cellv(k) for k, c in st.LAPL.items())
    fhi = sum(c * cellv(k) for k, c in st.FACE_DERIV.items())
    flo = sum(c * cellv(k - 1) for k, c in st.FACE_DERIV.items())
    assert lap == fhi - flo
    div = sum(c * cellv(k) for k, c in st.GRAD.items())
    uhi = sum(c * cellv(k) for k, c in st.FACE_VALUE.items())
    ulo = sum(c * cellv(k - 1) for k, c in st.FACE_VALUE.items())
    assert div == uhi - ulo


def test_neumann_ghosts_reproduce_boundary_flux_exactly():
    """With the ghosts of Eq. (Neumann5) the face derivative of Eq. (cell2face) on the
    boundary face equals the Neumann datum for ANY interior values (this is what makes the
    discrete solvability condition exact)."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        phi = [Fr(int(v)) for v in rng.integers(-50, 50, size=4)]  # cells m = 0..3
        gdat = Fr(int(rng.integers(-9, 9)))
        g1 = sum(st.NEUMANN[1][0][m] * phi[m] for m in range(4)) + st.NEUMANN[1][1] * gdat
        g2 = sum(st.NEUMANN[2][0][m] * phi[m] for m in range(4)) + st.NEUMANN[2][1] * gdat
        # face between interior cell 0 (offset 0) and ghost 1 (offset +1): cells -1..2
        seq = {-1: phi[1], 0: phi[0], 1: g1, 2: g2}
        flux = sum(c * seq[k] for k, c in st.FACE_DERIV.items())
        assert flux == gdat


def _poly2(x, y):
    return 1.0 + 2 * x - 3 * y + x * y + 4 * x ** 2 * y ** 2 - 5 * x ** 3 * y + x ** 4 - 2 * y ** 4


def _poly2_lap(x, y):
    return 8 * y ** 2 + 8 * x ** 2 - 30 * x * y + 12 * x ** 2 - 24 * y ** 2


def _cavg2(f, n, h, origin=(-2, -2), shape=None):
    """Cell averages on a grid via 4x4 Gauss (exact for these degree <= 4 polynomials)."""
    from paper_2506_02663_gb300.workloads import cell_average_gauss
    return cell_average_gauss(f, n, h, origin=origin, shape=shape)


@pytest.mark.parametrize("bc", [0, 1])
def test_level_laplacian_exact_on_quartic_2d(bc):
    """Numpy level operator with physical ghosts: exact (to roundoff) on cell averages of a
    degree-4 polynomial, Dirichlet or Neumann data given as exact face averages."""
    from paper_2506_02663_gb300.workloads import face_average_gauss
    n, h = 12, 1.0 / 12
    P = np.full((n + 4, n + 4), np.nan)
    P[2:-2, 2:-2] = _cavg2(_poly2, (n, n), h, origin=(0, 0), shape=(n, n))
    cov = np.zeros_like(P, bool)
    cov[2:-2, 2:-2] = True
    data = {}
    for d in range(2):
        for s in (0, 1):
            if bc == 0:
                data[2 * d + s] = face_average_gauss(_poly2, (n, n), h, d, s)
            else:
                sign = 1.0 if s == 1 else -1.0
                if d == 0:
                    dn = lambda x, y: sign * (2 + y + 8 * x * y ** 2 - 15 * x ** 2 * y + 4 * x ** 3)
                else:
                    dn = lambda x, y: sign * (-3 + x + 8 * x ** 2 * y - 5 * x ** 3 - 8 * y ** 3)
                data[2 * d + s] = face_average_gauss(dn, (n, n), h, d, s)
    st.fill_physical_ghosts(P, (-2, -2), (n, n), cov, 2, h, [bc] * 4, data)
    L = st.laplacian(P, 2, h)[2:-2, 2:-2]
    ex = _cavg2(_poly2_lap, (n, n), h, origin=(0, 0), shape=(n, n))
    assert np.max(np.abs(L - ex)) < 1e-9 * np.max(np.abs(ex))
