"""Pins of the oracle's convection operator (oracle/convection.py, Eq. convOp): exact for
linear velocities (the face average of a product of linear functions is exactly the printed
product formula), not exact for quadratic variation across a face, fourth order on the
Taylor-Green velocity against its exact cell-averaged convection, in 2-D and 3-D."""
import numpy as np
import pytest

from oracle.convection import convection


def _centres(n, h, D, ng=2):
    ax = (np.arange(-ng, n + ng) + 0.5) * h
    return np.meshgrid(*([ax] * D), indexing="ij")


@pytest.mark.parametrize("D", [2, 3])
def test_exact_for_linear_velocity(D):
    """u_c = a_c + sum_e B[c, e] x_e: cell averages are centre values, and <div(uu)> equals
    the centre value of (div u) u + (u . grad) u, a linear function."""
    rng = np.random.default_rng(D)
    a, B = rng.standard_normal(D), rng.standard_normal((D, D))
    n, h = 8, 1.0 / 8
    X = _centres(n, h, D)
    U = [a[c] + sum(B[c, e] * X[e] for e in range(D)) for c in range(D)]
    got = convection(U, h)
    div = np.trace(B)
    inner = tuple(slice(2, -2) for _ in range(D))
    for c in range(D):
        want = div * U[c] + sum(U[e] * B[c, e] for e in range(D))
        assert np.max(np.abs(got[c][inner] - want[inner])) <= 1e-12
        assert np.all(np.isnan(got[c][(slice(0, 1),) + (slice(None),) * (D - 1)]))  # outside the stencil


def test_not_exact_for_quadratic_transverse_variation():
    """u = (x y^2, 0): the product formula misses an h^4 term of the face average of
    x^2 y^4 (it is exact for fields linear across the face), so the operator is not exact,
    while the error stays at the size of that term."""
    n, h = 8, 1.0 / 8
    X, Y = _centres(n, h, 2)
    U = [X * (Y * Y + h * h / 12.0), np.zeros_like(X)]  # exact cell averages of x y^2
    got = convection(U, h)
    # div(uu) = d/dx (x^2 y^4) = 2 x y^4, cell average 2 x <y^4>
    want = 2.0 * X * (Y ** 4 + Y * Y * h * h / 2.0 + h ** 4 / 80.0)
    err = np.max(np.abs(got[0][2:-2, 2:-2] - want[2:-2, 2:-2]))
    assert 1e-9 < err < 1e-4, err
    assert np.max(np.abs(got[1][2:-2, 2:-2])) == 0.0


def _tg_averages(n, D):
    """Cell averages (two ghost layers, corners included) of the Taylor-Green velocity
    u = sin(2 pi x) cos(2 pi y) [cos(2 pi z)], v = -cos(2 pi x) sin(2 pi y) [cos(2 pi z)]
    (w = 0 in 3-D), and of its convection, by exact integrals."""
    h = 1.0 / n
    lo = (np.arange(-2, n + 2)) * h
    k = 2.0 * np.pi

    def I_sin(a):  # cell average of sin(k x) over [a, a + h]
        return (np.cos(k * a) - np.cos(k * (a + h))) / (k * h)

    def I_cos(a):
        return (np.sin(k * (a + h)) - np.sin(k * a)) / (k * h)
    S, Cc = I_sin(lo), I_cos(lo)
    if D == 2:
        u = S[:, None] * Cc[None, :]
        v = -Cc[:, None] * S[None, :]
        # (u . grad) u = (pi sin(4 pi x), pi sin(4 pi y)); div u = 0
        k2 = 2.0 * k
        s2 = (np.cos(k2 * lo) - np.cos(k2 * (lo + h))) / (k2 * h)
        cu = np.pi * np.repeat(s2[:, None], len(lo), axis=1)
        cv = np.pi * np.repeat(s2[None, :], len(lo), axis=0)
        return [u, v], [cu, cv], h
    u = S[:, None, None] * Cc[None, :, None] * Cc[None, None, :]
    v = -Cc[:, None, None] * S[None, :, None] * Cc[None, None, :]
    w = np.zeros_like(u)
    # div(uu) = (u . grad) u + (div u) u with div u = 0:
    #   x: 2 pi sin cos(x) cos^2(z) = pi sin(4 pi x) cos^2(2 pi z)
    #   y: pi sin(4 pi y) cos^2(2 pi z);  z: 0
    k2 = 2.0 * k
    s2 = (np.cos(k2 * lo) - np.cos(k2 * (lo + h))) / (k2 * h)
    c2 = 0.5 + (np.sin(k2 * (lo + h)) - np.sin(k2 * lo)) / (2.0 * k2 * h)  # average of cos^2(2 pi z)
    cu = np.pi * s2[:, None, None] * np.ones(len(lo))[None, :, None] * c2[None, None, :]
    cv = np.pi * np.ones(len(lo))[:, None, None] * s2[None, :, None] * c2[None, None, :]
    return [u, v, w], [cu, cv, np.zeros_like(u)], h


@pytest.mark.parametrize("D", [2, 3])
def test_fourth_order_on_taylor_green(D):
    errs = []
    for n in ((16, 32, 64) if D == 2 else (8, 16, 32)):
        U, C, h = _tg_averages(n, D)
        got = convection(U, h)
        inner = tuple(slice(2, -2) for _ in range(D))
        errs.append(max(float(np.max(np.abs(got[c][inner] - C[c][inner]))) for c in range(D)))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 3.8, (errs, orders)
