"""Pins of the oracle's ERK-ESDIRK tableau (oracle/imex.py): row sums, the order conditions
up to order four of the explicit and the implicit tableau with the shared weights, the
coupling conditions between them, stiff accuracy, and fourth-order convergence of an
additive integration of a stiff linear + nonstiff nonlinear system with a known solution."""
from fractions import Fraction as F

import numpy as np

from oracle import imex


def _mv(A, v):
    return [sum(A[i][j] * v[j] for j in range(6)) for i in range(6)]


def _dot(a, v):
    return sum(x * y for x, y in zip(a, v))


def test_row_sums_stiff_accuracy_and_order_conditions():
    b, c = imex.B, imex.C
    tol = F(1, 10 ** 20)  # the explicit entries are published rational approximations
    for A in (imex.A_E, imex.A_I):
        assert all(abs(sum(A[i]) - c[i]) < tol for i in range(6))
    assert all(imex.A_E[i][j] == 0 for i in range(6) for j in range(i, 6))  # explicit
    assert all(imex.A_I[i][i] == imex.GAMMA for i in range(1, 6)) and imex.A_I[0][0] == 0
    assert imex.A_I[5] == b  # stiffly accurate
    c2 = [x * x for x in c]
    assert _dot(b, [F(1)] * 6) == 1
    assert abs(_dot(b, c) - F(1, 2)) < tol and abs(_dot(b, c2) - F(1, 3)) < tol
    assert abs(_dot(b, [x ** 3 for x in c]) - F(1, 4)) < tol
    for X in (imex.A_E, imex.A_I):
        Xc = _mv(X, c)
        assert abs(_dot(b, Xc) - F(1, 6)) < tol
        assert abs(_dot(b, [x * y for x, y in zip(c, Xc)]) - F(1, 8)) < tol
        assert abs(_dot(b, _mv(X, c2)) - F(1, 12)) < tol
        for Y in (imex.A_E, imex.A_I):  # order-4 coupling: every colouring of the tall tree
            assert abs(_dot(b, _mv(X, _mv(Y, c))) - F(1, 24)) < tol


def test_a_wrong_entry_breaks_the_conditions():
    """The pins are sharp: perturbing one explicit entry by 1e-9 violates an order condition
    by far more than the tolerance above."""
    A = [row[:] for row in imex.A_E]
    A[4][2] += F(1, 10 ** 9)
    err = abs(_dot(imex.B, _mv(A, _mv(A, imex.C))) - F(1, 24))
    assert err > F(1, 10 ** 15)


def _integrate(lam, n):
    """y' = -lam y (implicit) + y^2 + s(t) (explicit), s chosen so that y = (cos t, sin 2t)
    exactly; n steps of the additive scheme to t = 1; max error."""
    def exact(t):
        return np.array([np.cos(t), np.sin(2 * t)])

    def dexact(t):
        return np.array([-np.sin(t), 2 * np.cos(2 * t)])

    def f_i(t, y):
        return -lam * y

    def f_e(t, y):
        ye = exact(t)
        return y * y + (dexact(t) + lam * ye - ye * ye)

    def solve_i(rhs, t, kg):
        return rhs / (1.0 + kg * lam)

    k = 1.0 / n
    y, t = exact(0.0), 0.0
    for _ in range(n):
        y = imex.ark_step(y, t, k, f_e, f_i, solve_i)
        t += k
    return np.max(np.abs(y - exact(1.0)))


def test_fourth_order_additive_integration():
    """Classical order four where k lam << 1."""
    lam = np.array([1.0, 3.0])
    errs = [_integrate(lam, n) for n in (10, 20, 40)]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 3.8, (errs, orders)


def test_stiff_additive_integration_is_stable_and_converges():
    """With k lam up to 10 (the implicit part stiff) the scheme stays stable and converges,
    at a reduced order (ESDIRK stage order two under a stiff time-dependent forcing)."""
    lam = np.array([50.0, 200.0])
    errs = [_integrate(lam, n) for n in (20, 40, 80)]
    assert errs[0] < 1e-2 and errs[1] < errs[0] and errs[2] < errs[1]
    assert np.log2(errs[1] / errs[2]) > 2.0
