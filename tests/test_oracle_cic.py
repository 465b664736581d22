"""Pins of the oracle's coarse-fine interface pieces (oracle/cic.py): the time interpolation
of Eq. (timeInterp) and the per-component correction of Eq. (correctingFaceAvg), checked
against what the mathematics fixes (exactness on cubics, fourth-order convergence, the
printed entries, exact compatibility after the correction)."""
import numpy as np
import pytest

from oracle import cic


@pytest.mark.parametrize("k", [0.5, 0.1, 1e-3])
def test_time_interpolation_exact_on_cubics(k):
    """Value and derivative of every cubic in t are reproduced exactly (to rounding) from its
    values at the four nodes, at points inside and beyond the node interval."""
    rng = np.random.default_rng(11)
    x = cic.time_interp_nodes(k)
    for _ in range(20):
        c = rng.standard_normal(4)
        p = np.polynomial.Polynomial(c)
        for eta in (-1.7 * k, -0.3 * k, 0.0, 0.45 * k, 0.9 * k, 1.3 * k):
            v, dv = cic.time_interpolate([p(t) for t in x], k, eta)
            scale = np.max(np.abs(c)) * (1 + 3 * k) ** 3
            assert abs(v - p(eta)) <= 1e-12 * scale
            assert abs(dv - p.deriv()(eta)) <= 1e-12 * scale / k
        v, dvk = cic.time_interpolate([p(t) for t in x], k, 0.45 * k, scaled=True)
        assert abs(dvk - k * p.deriv()(0.45 * k)) <= 1e-12 * np.max(np.abs(c)) * 8


def test_time_interpolation_fails_on_quartics():
    """One degree higher the interpolation is no longer exact (so a dropped term or a wrong
    node would show)."""
    k, eta = 0.5, 0.3
    x = cic.time_interp_nodes(k)
    v, _ = cic.time_interpolate([t ** 4 for t in x], k, eta)
    assert abs(v - eta ** 4) > 1e-3


def test_time_interpolation_order():
    """Fourth order for the value and third for the derivative on a smooth function."""
    f, df = np.sin, np.cos
    errs = []
    for k in (0.2, 0.1, 0.05):
        t0 = 0.37
        vals = [f(t0 + t) for t in cic.time_interp_nodes(k)]
        v, dv = cic.time_interpolate(vals, k, 0.5 * k)
        errs.append((abs(v - f(t0 + 0.5 * k)), abs(dv - df(t0 + 0.5 * k))))
    o_v = np.log2(errs[1][0] / errs[2][0])
    o_d = np.log2(errs[1][1] / errs[2][1])
    assert o_v > 3.8 and o_d > 2.8, (o_v, o_d)


@pytest.mark.parametrize("k", [1.0, 0.25])
def test_time_interpolation_matches_printed_entries(k):
    """The printed matrix of Eq. (timeInterp) equals the oracle's value and d/dt rows (the
    reading stated in oracle/cic.py)."""
    for eta in (-1.5 * k, -0.2 * k, 0.0, 0.6 * k, 1.0 * k):
        assert np.allclose(cic.time_interp_matrix(k, eta), cic.printed_time_interp_matrix(k, eta),
                           rtol=0, atol=1e-12 / k)


@pytest.mark.parametrize("k", [0.5, 0.02])
def test_coarse_time_weights_follow_the_papers_time_labels(k):
    """With t_{-i} = t0 - i k and eta = t* - t_{-1}, the weights for the data in the order
    t_{-0}..t_{-3} reproduce every cubic and its derivative at t*, put the unit weight on
    t_{-1} at eta = 0 and on t_{-0} at eta = k."""
    rng = np.random.default_rng(23)
    t0 = 0.8
    times = [t0 - i * k for i in range(4)]
    for _ in range(10):
        p = np.polynomial.Polynomial(rng.standard_normal(4))
        for eta in (0.0, 0.25 * k, 0.5 * k, k):
            v, dv = cic.interpolate_coarse_times([p(t) for t in times], k, eta)
            assert abs(v - p(times[1] + eta)) <= 1e-12 * 10
            assert abs(dv - p.deriv()(times[1] + eta)) <= 1e-11 * 10 / k
    assert np.array_equal(cic.coarse_time_weights(k, 0.0)[0], [0.0, 1.0, 0.0, 0.0])
    assert np.allclose(cic.coarse_time_weights(k, k)[0], [1.0, 0.0, 0.0, 0.0], atol=1e-15)


def test_face_correction_enforces_compatibility_per_component():
    """After Eq. (correctingFaceAvg) the interface and physical face sums of every component
    vanish; one uniform shift per component; an already compatible component is unchanged."""
    rng = np.random.default_rng(13)
    a = rng.standard_normal(40)
    comp = np.repeat([0, 1, 2], [10, 18, 12])
    phys = {0: 0.75, 1: -2.0}
    a[28:] -= np.mean(a[28:])  # component 2: already compatible, no physical faces
    out, deltas = cic.correct_by_component(a, comp, phys)
    for c in (0, 1, 2):
        sel = comp == c
        assert abs(np.sum(out[sel]) + phys.get(c, 0.0)) <= 1e-13
        assert np.allclose(out[sel] - a[sel], deltas[c], rtol=0, atol=1e-15)
    assert abs(deltas[2]) <= 1e-15


def _two_level(dim=2):
    from oracle.hierarchy import Hierarchy
    if dim == 2:
        return Hierarchy(2, (16, 16), [[((0, 0), (15, 15))], [((8, 8), (23, 23))]], bc=[0] * 4)
    return Hierarchy(3, (8, 8, 8), [[((0, 0, 0), (7, 7, 7))], [((4, 4, 4), (11, 11, 11))]], bc=[0] * 6)


def _coarse_fields(H, rng, n):
    from oracle import solve as so
    U = so.Unknowns(H)
    return [U.scatter(rng.standard_normal(U.n), fill_invalid=True) for _ in range(n)]


@pytest.mark.parametrize("dim", [2, 3])
def test_interface_ghosts_compose_amrcfi_and_time_interpolation(dim):
    """Data constant in time give the AMRCFI values of that field and a zero rate; data
    linear in time (A + t B) give AMRCFI of A + t* B and the rate AMRCFI of B."""
    from oracle import composite as cp
    H = _two_level(dim)
    rng = np.random.default_rng(7)
    A, B = _coarse_fields(H, rng, 2)
    k, eta = 0.3, 0.11
    lev = H.levels[1]

    def amrcfi(F):
        G = [a.copy() for a in F]
        cp.fill_cf_ghosts(H, G, 1)
        return G[1][lev.cf_ghost]

    cells, v, r = cic.interface_ghost_values(H, [A[0]] * 4, 1, k, eta)
    assert np.array_equal(cells, np.argwhere(lev.cf_ghost))
    assert np.allclose(v, amrcfi(A), rtol=0, atol=1e-13) and np.allclose(r, 0.0, atol=1e-12)
    ts = [(1 - i) * k for i in range(4)]  # t_{-i} - t_{-1}, i = 0..3
    lin = [A[0] + t * B[0] for t in ts]
    _, v, r = cic.interface_ghost_values(H, lin, 1, k, eta)
    want = [A[l] + eta * B[l] for l in range(2)]
    assert np.allclose(v, amrcfi(want), rtol=0, atol=1e-12)
    assert np.allclose(r, amrcfi(B), rtol=0, atol=1e-11)


def test_interface_face_averages_exact_on_cubics_and_divergence_theorem():
    """Cell averages of w = (f(x), g(y)) with cubic f, g: every interface face average equals
    s f (or s g) at the face (Eq. cell2face is exact for cubics), and the face sums times the
    face length equal the integral of div w over the box."""
    H = _two_level(2)
    lev = H.levels[1]
    h = lev.h

    def f(x):
        return 2.0 * x ** 3 - x ** 2 + 0.5 * x + 1.0

    def F(x):  # antiderivative of f
        return 0.5 * x ** 4 - x ** 3 / 3.0 + 0.25 * x ** 2 + x

    def g(y):
        return -y ** 3 + 3.0 * y

    def G(y):
        return -0.25 * y ** 4 + 1.5 * y ** 2

    i = (np.arange(lev.shape[0]) + lev.origin[0]) * h
    j = (np.arange(lev.shape[1]) + lev.origin[1]) * h
    W0 = np.repeat(((F(i + h) - F(i)) / h)[:, None], lev.shape[1], axis=1)
    W1 = np.repeat(((G(j + h) - G(j)) / h)[None, :], lev.shape[0], axis=0)
    faces = cic.interface_faces(H, 1)
    assert len(faces) == 4 * 16
    vals = cic.interface_face_averages(H, [W0, W1], 1, faces)
    for (c, d, s, comp), v in zip(faces, vals):
        assert comp == 0
        xf = (c[d] + lev.origin[d] + (1 if s > 0 else 0)) * h
        want = s * (f(xf) if d == 0 else g(xf))
        assert abs(v - want) <= 1e-13
    lo, hi = 8 * h, 24 * h
    flux = (f(hi) - f(lo)) * (hi - lo) + (g(hi) - g(lo)) * (hi - lo)
    assert abs(np.sum(vals) * h - flux) <= 1e-12


def test_box_interface_data_exact_on_cubics():
    """The boundary data of a single-box component's level problem: cell averages of a cubic
    p(x, y) give, on every interface face of the box, the exact face average of p at the
    slot of that face; the multi-box component is rejected."""
    from oracle.hierarchy import Hierarchy
    H = Hierarchy(2, (32, 32), [[((0, 0), (31, 31))], [((8, 8), (19, 19)), ((40, 36), (55, 51)),
                                                       ((20, 8), (27, 15))]], bc=[0] * 4)
    lev = H.levels[1]
    h = lev.h
    with pytest.raises(ValueError):
        cic.component_box(H, 1, 0)
    lo, hi, flags = cic.component_box(H, 1, 1)
    assert (lo, hi, flags) == ((40, 36), (55, 51), [1, 1, 1, 1])

    def avg(F, a):  # cell average over [a, a + h] from the antiderivative F
        return (F(a + h) - F(a)) / h

    x = (np.arange(lev.shape[0]) + lev.origin[0]) * h
    y = (np.arange(lev.shape[1]) + lev.origin[1]) * h
    ax3 = avg(lambda t: t ** 4 / 4, x)
    ax1 = avg(lambda t: t ** 2 / 2, x)
    ay2 = avg(lambda t: t ** 3 / 3, y)
    ay1 = avg(lambda t: t ** 2 / 2, y)
    X = ax3[:, None] + 2.0 * ax1[:, None] * ay2[None, :] - ay1[None, :]
    data = cic.box_interface_bc(H, X, 1, 1)
    n = (16, 16)
    for d in range(2):
        for s in (0, 1):
            arr = data[2 * d + s]
            xf = (lo[d] + (n[d] if s else 0)) * h  # the face's coordinate
            t = np.arange(n[1 - d]) + lo[1 - d]
            tc = t * h
            if d == 0:  # face x = xf, averaged over y
                want = xf ** 3 + 2.0 * xf * avg(lambda u: u ** 3 / 3, tc) - avg(lambda u: u ** 2 / 2, tc)
            else:  # face y = xf, averaged over x
                want = avg(lambda u: u ** 4 / 4, tc) + 2.0 * avg(lambda u: u ** 2 / 2, tc) * xf ** 2 - xf
            assert np.allclose(arr, want, rtol=0, atol=1e-12)
