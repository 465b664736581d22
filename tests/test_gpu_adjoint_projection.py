"""Adjoints of G^comp, D^comp, the pure-Neumann solve and the composite projection on the
GPU against the oracle's assembled transposes (element by element), and the gradient of
the differentiable chain of the adjoint2d workload (Helmholtz solve per component, then
the composite projection, J = 1/2 sum over valid cells of u^2) against central finite
differences: J is quadratic, so the differences are exact up to rounding and the solve
tolerance, at the small sizes and at the full three-level 256^2 / 308^2 / 308^2 size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as ad, composite as cp, solve as so  # noqa: E402

from _gpu_helpers import from_packed, max_abs, max_diff, to_packed  # noqa: E402
from test_gpu_parity import BCS, HIERS, _amr, _dev, _hier  # noqa: E402

pytestmark = pytest.mark.gpu


def _all_cells(H, rng):
    """Random values on every covered cell (invalid cells independent of their children)."""
    F = cp.new_field(H)
    for l, lev in enumerate(H.levels):
        F[l][lev.covered] = rng.standard_normal(int(lev.covered.sum()))
    return F


def _zeros(gh):
    return torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")


def _get(gh, H, t):
    return from_packed(gh, H, t.cpu().numpy())


@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("which", [0, 1])
def test_gradient_transpose_matches_oracle(name, which):
    amr = _amr()
    dim = HIERS[name][0]
    bc = list(BCS[dim][which])
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(201)
    Y = [_all_cells(H, rng) for _ in range(dim)]
    ref = ad.gradient_transpose(H, Y, bc_types=bc)
    out = _zeros(gh)
    amr.gradient_transpose(gh, bc, [_dev(to_packed(gh, H, y)) for y in Y], out)
    got = _get(gh, H, out)
    hmin = min(lev.h for lev in H.levels)
    scale = 4.0 / hmin * max(max_abs(H, y, "covered") for y in Y)
    assert max_diff(H, got, ref, "covered") <= 1e-13 * scale


@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("which", [0, 2])
def test_divergence_transpose_matches_oracle(name, which):
    amr = _amr()
    dim = HIERS[name][0]
    bc = list(BCS[dim][which])
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(203)
    y = _all_cells(H, rng)
    ref = ad.divergence_transpose(H, y, bc_types=bc)
    outs = [_zeros(gh) for _ in range(dim)]
    amr.divergence_transpose(gh, bc, _dev(to_packed(gh, H, y)), outs)
    hmin = min(lev.h for lev in H.levels)
    scale = 4.0 / hmin * max_abs(H, y, "covered")
    for d in range(dim):
        assert max_diff(H, _get(gh, H, outs[d]), ref[d], "covered") <= 1e-13 * scale


@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_neumann_solve_transpose_matches_oracle(name, precision):
    amr = _amr()
    dim = HIERS[name][0]
    bc = [1] * (2 * dim)
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(207)
    G = _all_cells(H, rng)
    ref, _, _ = ad.neumann_solve_transpose(H, G)
    op = amr.Operator(gh, 0.0, 1.0, bc)
    lam = _zeros(gh)
    prec = amr.FP64 if precision == "fp64" else amr.MIXED
    st = op.solve_transpose(lam, _dev(to_packed(gh, H, G)),
                            params=amr.default_params(rtol=1e-12, max_vcycles=200, precision=prec))
    got = _get(gh, H, lam)
    assert max_diff(H, got, ref) <= 1e-9 * max_abs(H, ref)
    U = so.Unknowns(H)
    x = U.gather(got)
    assert abs(np.sum(x)) <= 1e-11 * np.sum(np.abs(x))
    assert st["vcycles"] < 60


@pytest.mark.parametrize("name", list(HIERS))
def test_project_transpose_matches_oracle(name):
    amr = _amr()
    dim = HIERS[name][0]
    bcn = [1] * (2 * dim)
    vbc = [0] * (2 * dim)
    Hn, gh = _hier(name, bcn)
    rng = np.random.default_rng(211)
    V = [_all_cells(Hn, rng) for _ in range(dim)]
    ref, _ = ad.project_transpose(Hn, V, vel_bc_types=vbc)
    ppe = amr.Operator(gh, 0.0, 1.0, bcn)
    outs = [_zeros(gh) for _ in range(dim)]
    lam = _zeros(gh)
    amr.project_transpose(ppe, vbc, [_dev(to_packed(gh, Hn, v)) for v in V], outs, lam,
                          params=amr.default_params(rtol=1e-12, max_vcycles=200))
    for d in range(dim):
        got = _get(gh, Hn, outs[d])
        assert max_diff(Hn, got, ref[d], "covered") <= 1e-9 * max_abs(Hn, ref[d], "covered")


def _chain(amr, gh, helm, ppe, vbc, mask, p):
    from paper_2506_02663_gb300.autograd import AmrProject, AmrSolve

    def J(g):
        w = [AmrSolve.apply(gd, helm, p) for gd in g]
        u = AmrProject.apply(ppe, vbc, p, *w)
        return 0.5 * sum(torch.sum(mask * ud * ud) for ud in u)
    return J


def _mask(gh, H):
    return _dev(to_packed(gh, H, [lev.valid.astype(np.float64) for lev in H.levels], fill=0.0))


@pytest.mark.parametrize("name", ["two_level_ragged", "three_level_multibox", "three_d"])
def test_projection_chain_gradient_vs_dense_and_fd(name):
    """grad_g J = Helm^{-T} P^T (mask u): elementwise against the oracle's dense chain, and
    directional derivatives against central differences (relative 1e-6)."""
    amr = _amr()
    dim = HIERS[name][0]
    Hn, gh = _hier(name, [1] * (2 * dim))
    Hd, _ = _hier(name, [0] * (2 * dim))
    vbc = [0] * (2 * dim)
    beta = -0.02
    helm = amr.Operator(gh, 1.0, beta, [0] * (2 * dim))
    ppe = amr.Operator(gh, 0.0, 1.0, [1] * (2 * dim))
    p = amr.default_params(rtol=1e-13, max_vcycles=200, use_graph=1)
    rng = np.random.default_rng(223)
    U = so.Unknowns(Hd)
    Gs = [U.scatter(rng.standard_normal(U.n)) for _ in range(dim)]
    g = [_dev(to_packed(gh, Hd, G)).requires_grad_(True) for G in Gs]
    mask = _mask(gh, Hd)
    J = _chain(amr, gh, helm, ppe, vbc, mask, p)
    loss = J(g)
    loss.backward()
    grads = [x.grad.detach() for x in g]
    # dense oracle chain
    A, Ud = so.helmholtz_matrix(Hd, 1.0, beta)
    W = [so.solve_direct(Hd, G, 1.0, beta, A=A, U=Ud)[0] for G in Gs]
    Uu, _ = so.project(Hn, W)
    Vv = [[np.where(lev.valid, Uu[d][l], 0.0) for l, lev in enumerate(Hd.levels)] for d in range(dim)]
    Z, _ = ad.project_transpose(Hn, Vv)
    for d in range(dim):
        ref, _, _ = so.solve_transpose_direct(Hd, Z[d], 1.0, beta, A=A, U=Ud)
        got = _get(gh, Hd, grads[d])
        assert max_diff(Hd, got, ref) <= 1e-8 * max_abs(Hd, ref)
    eps = 1e-3
    for _ in range(3):
        v = [_dev(to_packed(gh, Hd, U.scatter(rng.standard_normal(U.n)))) for _ in range(dim)]
        with torch.no_grad():
            jp = J([x.detach() + eps * vd for x, vd in zip(g, v)])
            jm = J([x.detach() - eps * vd for x, vd in zip(g, v)])
        fd = float((jp - jm) / (2 * eps))
        adj = float(sum(torch.sum(gd * vd * mask) for gd, vd in zip(grads, v)))
        assert abs(fd - adj) <= 1e-6 * abs(fd), (fd, adj)


def test_projection_chain_full_size_fd():
    """The adjoint2d workload at full size (base 256^2, boxes [0.2,0.8]^2 and [0.35,0.65]^2
    -> 308^2 and 308^2 fine cells; seeded smoothed N(0,1) forcing, two components): the
    directional derivative of J from the adjoint agrees with central differences (eps =
    1e-3) to 1e-6 along 64 seeded random unit directions.  J is quadratic in g, so the
    central difference is exact up to rounding and the solve tolerance."""
    amr = _amr()
    from oracle.hierarchy import Hierarchy as OH
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, comps = wl.adjoint2d_forcing()
    H = OH(dim, n0, boxes, bc=[0] * 4)
    gh = amr.Hierarchy(dim, n0, boxes, h0=1.0 / n0[0])
    vbc = [0] * 4
    helm = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA, [0] * 4)
    ppe = amr.Operator(gh, 0.0, 1.0, [1] * 4)
    p = amr.default_params(rtol=1e-12, max_vcycles=200, use_graph=1)
    mask = _mask(gh, H)
    g = [torch.from_numpy(gh.pack(comps[d])).cuda().requires_grad_(True) for d in range(dim)]
    J = _chain(amr, gh, helm, ppe, vbc, mask, p)
    loss = J(g)
    loss.backward()
    grads = [x.grad.detach() for x in g]
    rng = np.random.default_rng(229)
    eps = 1e-3
    errs = []
    for _ in range(64):
        v = [mask * torch.from_numpy(rng.standard_normal(gh.nelems)).cuda() for _ in range(dim)]
        nrm = float(torch.sqrt(sum(torch.sum(vd * vd) for vd in v)))
        v = [vd / nrm for vd in v]
        with torch.no_grad():
            jp = J([x.detach() + eps * vd for x, vd in zip(g, v)])
            jm = J([x.detach() - eps * vd for x, vd in zip(g, v)])
        fd = float((jp - jm) / (2 * eps))
        adj = float(sum(torch.sum(gd * vd) for gd, vd in zip(grads, v)))
        errs.append(abs(fd - adj) / abs(fd))
    assert max(errs) <= 1e-6, (max(errs), len(errs))
