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
