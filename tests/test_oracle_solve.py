"""Pins of the oracle's solves (no GPU): manufactured-solution convergence order,
multigrid vs direct solve, solvability and mean-zero to machine precision, transposes,
and the composite projection (Lemma compositeProjection, O(h^4) divergence)."""
import math

import numpy as np
import pytest

from oracle import composite as cp, mg, solve as so
from oracle.hierarchy import Hierarchy
from paper_2506_02663_gb300 import workloads as wl


def _ms_errors(n):
    rhs, bc, exact = wl.ms2d(n)
    H = Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]], bc=[0] * 4)
    f = cp.new_field(H)
    f[0][H.levels[0].covered] = rhs.ravel()
    phi, _, _ = so.solve_direct(H, f, 0.0, 1.0, [bc])
    e = phi[0][H.levels[0].covered].reshape(n, n) - exact
    h = 1.0 / n
    return (np.sum(np.abs(e)) * h * h, math.sqrt(np.sum(e * e) * h * h), np.max(np.abs(e)))


def test_manufactured_solution_fourth_order():
    """Sec. 3 (Proposition cited after Eq. convOp): L is fourth-order accurate; with the
    ghost formulas the solution error converges at order ~4 in L1/L2 and >= 3.5 in Linf
    (third-order truncation on a codimension-one set near the boundary, end of Sec. 3)."""
    errs = [_ms_errors(n) for n in (16, 32, 64, 128)]
    for p in range(3):
        orders = [math.log2(errs[i][p] / errs[i + 1][p]) for i in range(len(errs) - 1)]
        assert orders[-1] > (3.8 if p < 2 else 3.5), (p, orders)


def test_direct_solution_residual_and_brute_force():
    """Sparse direct solve == dense numpy solve of the brute-force-assembled matrix."""
    H = Hierarchy(2, (8, 8), [[((0, 0), (7, 7))], [((4, 2), (11, 15))]], bc=[0, 0, 1, 0])
    U = so.Unknowns(H)
    rng = np.random.default_rng(3)
    f = U.scatter(rng.standard_normal(U.n))
    phi, A, U = so.solve_direct(H, f, 1.0, -0.05)
    dense = np.zeros((U.n, U.n))
    for j in range(U.n):
        e = np.zeros(U.n)
        e[j] = 1.0
        dense[:, j] = U.gather(cp.apply(H, U.scatter(e), 1.0, -0.05))
    x = np.linalg.solve(dense, U.gather(f))
    assert np.max(np.abs(U.gather(phi) - x)) < 1e-12 * np.max(np.abs(x))


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("ab", [(0.0, 1.0), (1.0, -1e-3)])
def test_multigrid_converges_to_direct(bc, ab):
    alpha, beta = ab
    boxes = [[((0, 0), (23, 23))], [((12, 8), (35, 31))], [((32, 24), (55, 47))]]
    H = Hierarchy(2, (24, 24), boxes, bc=[bc] * 4)
    U = so.Unknowns(H)
    f = U.scatter(np.random.default_rng(5).standard_normal(U.n))
    if so.is_pure_neumann(H, alpha):
        f, _ = so.solvability_fix(H, f)
    phi, hist = mg.solve(H, f, alpha, beta, rtol=1e-12, max_cycles=40)
    assert hist[-1] <= 1e-12 * mg.max_norm_valid(H, f)
    ref, _, _ = so.solve_direct(H, f, alpha, beta)
    if so.is_pure_neumann(H, alpha):
        phi, _ = so.mean_zero(H, phi)
    err = max(np.max(np.abs(phi[l] - ref[l])[lev.valid]) for l, lev in enumerate(H.levels))
    assert err < 1e-10 * mg.max_norm_valid(H, ref)
    # soft pin: at least a factor 3 per V-cycle on average (the paper reports ~10 for the
    # PPE with its ILU-GMRES bottom solver and ~1e4 for its Helmholtz systems)
    rate = (hist[0] / hist[-1]) ** (1.0 / (len(hist) - 1))
    assert rate > 3.0


def test_solvability_fix_and_mean_zero_machine_precision():
    H = Hierarchy(2, (16, 16), [[((0, 0), (15, 15))], [((8, 8), (23, 23))]], bc=[1] * 4)
    U = so.Unknowns(H)
    rng = np.random.default_rng(11)
    f = U.scatter(rng.standard_normal(U.n) + 3.0)
    g, m = so.solvability_fix(H, f)
    w = U.weights()
    x = U.gather(g)
    assert abs(math.fsum(x * w)) <= 1e-14 * math.fsum(np.abs(x) * w)
    assert abs(m - 3.0) < 0.2
    phi, _, _ = so.solve_direct(H, g, 0.0, 1.0)
    px = U.gather(phi)
    assert abs(math.fsum(px * w)) <= 1e-14 * math.fsum(np.abs(px) * w)


def test_solvability_with_neumann_data():
    """sum_valid h^D (L phi) = sum_boundary h^(D-1) g for any phi (telescoping), so the fix
    must make f - A phi sum to zero for the inhomogeneous data as well."""
    H = Hierarchy(2, (16, 16), [[((0, 0), (15, 15))], [((0, 8), (15, 23))]], bc=[1] * 4)
    U = so.Unknowns(H)
    rng = np.random.default_rng(12)
    data = []
    for lev in H.levels:
        data.append({f: rng.standard_normal(lev.ndom[1 - f // 2]) for f in range(4)})
    phi = U.scatter(rng.standard_normal(U.n))
    Y = U.gather(cp.apply(H, phi, 0.0, 1.0, data))
    w = U.weights()
    assert abs(math.fsum(Y * w) - so.boundary_flux_sum(H, data)) < 1e-12 * math.fsum(np.abs(Y) * w)


def test_transpose_solve():
    H = Hierarchy(2, (16, 16), [[((0, 0), (15, 15))], [((8, 4), (23, 27))]], bc=[0] * 4)
    U = so.Unknowns(H)
    g = U.scatter(np.random.default_rng(2).standard_normal(U.n))
    lam, A, U = so.solve_transpose_direct(H, g, 1.0, -0.01)
    assert np.max(np.abs(A.T @ U.gather(lam) - U.gather(g))) < 1e-12 * np.max(np.abs(U.gather(g)))
    # the composite operator is not symmetric (ghost formulas, AMRCFI, refluxing)
    assert abs(A - A.T).max() > 1e-3 * abs(A).max()


def _velocity_field(H, funcs):
    U = []
    for fn in funcs:
        F = cp.new_field(H)
        for l, lev in enumerate(H.levels):
            vals = wl.cell_average_gauss(fn, lev.ndom, lev.h, origin=lev.origin, shape=lev.shape)
            F[l][lev.covered] = vals[lev.covered]
        U.append(F)
    return U


def test_projection_lemma_and_divergence_order():
    """Eq. (comp_ProjOp), Lemma compositeProjection: P^comp of redundant data is redundant.
    The projected velocity's composite divergence decays like h^4 in the composite L1 norm
    (fourth-order P; the max norm sees the third-order boundary truncation of Sec. 3)."""
    divs = []
    for n in (16, 32):
        boxes = [[((0, 0), (n - 1, n - 1))], [((n // 2, n // 4), (3 * n // 2 - 1, 5 * n // 4 - 1))]]
        H = Hierarchy(2, (n, n), boxes, bc=[1] * 4)
        # w = divergence-free part + gradient part; both vanish on the boundary
        u0 = lambda x, y: 2 * np.pi * np.sin(np.pi * x) ** 2 * np.sin(np.pi * y) * np.cos(np.pi * y)
        u1 = lambda x, y: -2 * np.pi * np.sin(np.pi * x) * np.cos(np.pi * x) * np.sin(np.pi * y) ** 2
        g0 = lambda x, y: np.sin(np.pi * x) * x * (1 - y) * y
        W = _velocity_field(H, [lambda x, y: u0(x, y) + g0(x, y), u1])
        Uo, phi = so.project(H, W)
        # redundancy of u follows from redundancy of w (exact averages are redundant)
        for d in range(2):
            F = [a.copy() for a in Uo[d]]
            cp.average_down_all(H, F)
            lev0 = H.levels[0]
            scale = np.max(np.abs(Uo[d][0][lev0.covered]))
            assert np.max(np.abs(F[0][lev0.invalid] - Uo[d][0][lev0.invalid])) < 1e-11 * scale
        dv = cp.divergence(H, Uo, None, [0] * 4)
        divs.append(sum(np.sum(np.abs(dv[l][lev.valid])) * lev.h ** 2 for l, lev in enumerate(H.levels)))
    assert divs[0] / divs[1] > 10.0, divs
