"""Pins of the oracle's transposes (no GPU).  Each transpose is checked against the FORWARD
oracle function it transposes, through the identity <M x, y> = <x, M^T y> on random
vectors; the forward functions are themselves pinned elsewhere (orders of accuracy,
Neumann invariants, brute-force assembly), so a dropped coupling, a wrong sign, a missing
average-down weight or a transposed operand in a transpose fails here."""
import math

import numpy as np
import pytest

from oracle import adjoint as ad, composite as cp, solve as so
from oracle.hierarchy import Hierarchy

CASES = {
    "two_level": (2, (16, 16), [[((0, 0), (15, 15))], [((8, 4), (23, 27))]]),
    "three_level_multibox": (2, (16, 16), [[((0, 0), (15, 15))], [((4, 4), (15, 19)), ((16, 4), (27, 19))],
                                           [((16, 16), (39, 27))]]),
    "boundary_touching": (2, (16, 16), [[((0, 0), (15, 15))], [((0, 8), (11, 31))]]),
    "three_d": (3, (8, 8, 8), [[((0, 0, 0), (7, 7, 7))], [((4, 0, 6), (11, 7, 15))]]),
}


def _hier(name, bc):
    dim, n0, boxes = CASES[name]
    return Hierarchy(dim, n0, boxes, bc=[bc] * (2 * dim))


def _all_cells(H, rng):
    """Random values on every covered cell (invalid cells independent of their children)."""
    F = cp.new_field(H)
    for l, lev in enumerate(H.levels):
        F[l][lev.covered] = rng.standard_normal(int(lev.covered.sum()))
    return F


def _dot(H, X, Y):
    return math.fsum(float(np.sum(X[l][lev.covered] * Y[l][lev.covered])) for l, lev in enumerate(H.levels))


@pytest.mark.parametrize("name", list(CASES))
def test_average_down_transpose_closed_form(name):
    H = _hier(name, 0)
    U = so.Unknowns(H)
    rng = np.random.default_rng(101)
    x = rng.standard_normal(U.n)
    Y = _all_cells(H, rng)
    lhs = _dot(H, U.scatter(x), Y)          # <E x, Y> with E from composite.average_down
    rhs = float(np.dot(x, ad.average_down_transpose(H, Y)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("bc", [0, 1])
def test_gradient_transpose_dot_identity(name, bc):
    H = _hier(name, bc)
    U = so.Unknowns(H)
    rng = np.random.default_rng(103)
    phi = U.scatter(rng.standard_normal(U.n))
    Y = [_all_cells(H, rng) for _ in range(H.D)]
    G = cp.gradient(H, phi)
    lhs = math.fsum(_dot(H, G[d], Y[d]) for d in range(H.D))
    Z = ad.gradient_transpose(H, Y)
    rhs = _dot(H, phi, Z)
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1.0)
    # the output lives on the valid cells only
    for l, lev in enumerate(H.levels):
        assert np.all(Z[l][lev.covered & ~lev.valid] == 0.0)


@pytest.mark.parametrize("name", list(CASES))
def test_divergence_transpose_dot_identity(name):
    H = _hier(name, 0)
    U = so.Unknowns(H)
    rng = np.random.default_rng(107)
    W = [U.scatter(rng.standard_normal(U.n)) for _ in range(H.D)]
    y = _all_cells(H, rng)
    lhs = _dot(H, cp.divergence(H, W, bc_types=[0] * (2 * H.D)), y)
    Z = ad.divergence_transpose(H, y, bc_types=[0] * (2 * H.D))
    rhs = math.fsum(_dot(H, W[d], Z[d]) for d in range(H.D))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1.0)


@pytest.mark.parametrize("name", ["two_level", "three_level_multibox", "three_d"])
def test_neumann_solve_transpose(name):
    """<M f, G> = <f, M^T G> with M the forward pure-Neumann solve (solvability correction,
    bordered direct solve, mean zero); M^T's output solves A^T lambda = E^T G - w (1^T E^T G)/(1^T w)
    with zero unweighted sum (the left and right null vectors of the Neumann operator are
    h^D and 1)."""
    H = _hier(name, 1)
    U = so.Unknowns(H)
    rng = np.random.default_rng(109)
    f = U.scatter(rng.standard_normal(U.n))
    Gw = _all_cells(H, rng)
    fc, _ = so.solvability_fix(H, f)
    phi, A, _ = so.solve_direct(H, fc, 0.0, 1.0)
    phi, _ = so.mean_zero(H, phi)
    lam, _, _ = ad.neumann_solve_transpose(H, Gw, A=A, U=U)
    lhs = _dot(H, phi, Gw)
    rhs = float(np.dot(U.gather(f), U.gather(lam)))
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1.0)
    g = ad.average_down_transpose(H, Gw)
    w = U.weights()
    x = U.gather(lam)
    assert abs(math.fsum(x)) <= 1e-12 * np.sum(np.abs(x))
    res = A.T @ x - (g - w * math.fsum(g) / math.fsum(w))
    assert np.max(np.abs(res)) <= 1e-10 * np.max(np.abs(g))


@pytest.mark.parametrize("name", ["two_level", "three_level_multibox", "boundary_touching", "three_d"])
def test_projection_transpose_dot_identity(name):
    """<P w, v> = <w, P^T v> over every covered cell of every component, P the forward
    oracle projection (divergence, solvability, bordered solve, mean zero, gradient)."""
    Hn = _hier(name, 1)
    rng = np.random.default_rng(113)
    W = [_all_cells(Hn, rng) for _ in range(Hn.D)]
    V = [_all_cells(Hn, rng) for _ in range(Hn.D)]
    Uw, _ = so.project(Hn, W)
    PtV, _ = ad.project_transpose(Hn, V)
    lhs = math.fsum(_dot(Hn, Uw[d], V[d]) for d in range(Hn.D))
    rhs = math.fsum(_dot(Hn, W[d], PtV[d]) for d in range(Hn.D))
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1.0)


def test_projection_transpose_is_not_the_projection():
    """The fourth-order composite projection is not symmetric (G^T != -D on the composite
    grid), so P^T v differs from P v: the transpose is a distinct computation."""
    Hn = _hier("two_level", 1)
    rng = np.random.default_rng(127)
    V = [_all_cells(Hn, rng) for _ in range(Hn.D)]
    Pv, _ = so.project(Hn, V)
    PtV, _ = ad.project_transpose(Hn, V)
    diff = max(np.nanmax(np.abs(Pv[d][l] - PtV[d][l])) for d in range(2) for l in range(2))
    assert diff > 1e-3
