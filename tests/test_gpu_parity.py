"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element on seeded inputs.  Tolerances: operator applications within 1e-13 of the
operator's term scale (|alpha| + |beta| sum|L coefs|/h^2) * max|phi|; smoothing within
1e-12 relative; one V-cycle within 1e-10 relative; solutions within 1e-10 relative
max-norm (FP64 and mixed precision refined to the same residual)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import composite as cp, mg, solve as so  # noqa: E402
from oracle.hierarchy import Hierarchy as OH  # noqa: E402

from _gpu_helpers import from_packed, level_bc_data, max_abs, max_diff, op_scale, to_packed  # noqa: E402

pytestmark = pytest.mark.gpu

HIERS = {
    # ragged non-square base, box touching the x-low boundary
    "two_level_ragged": (2, (40, 24), [[((0, 0), (39, 23))], [((0, 8), (27, 39))]]),
    # multi-box level with a shared face + a third level
    "three_level_multibox": (2, (24, 24), [[((0, 0), (23, 23))], [((8, 8), (23, 31)), ((24, 8), (39, 31))],
                                           [((24, 24), (47, 47))]]),
    # 3-D two-level
    "three_d": (3, (12, 12, 12), [[((0, 0, 0), (11, 11, 11))], [((8, 0, 4), (19, 11, 15))]]),
}


def _amr():
    from paper_2506_02663_gb300 import amr
    return amr


def _hier(name, bc):
    dim, n0, boxes = HIERS[name]
    hi = tuple(n0[d] / n0[0] for d in range(dim))
    H = OH(dim, n0, boxes, bc=bc, hi=hi)
    gh = _amr().Hierarchy(dim, n0, boxes, h0=1.0 / n0[0])
    return H, gh


def _rand_field(H, rng, redundant=True):
    U = so.Unknowns(H)
    return U.scatter(rng.standard_normal(U.n), fill_invalid=redundant)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _bc_data(H, rng):
    out = []
    for lev in H.levels:
        out.append({2 * d + s: rng.standard_normal(tuple(lev.ndom[e] for e in range(H.D) if e != d))
                    for d in range(H.D) for s in (0, 1)})
    return out


BCS = {2: ([0, 1, 0, 0], [1, 1, 1, 1], [0, 0, 0, 0]), 3: ([0, 1, 0, 0, 1, 0], [1] * 6, [0] * 6)}


@pytest.mark.parametrize("name", list(HIERS))
def test_fill_ghosts_cfi_and_copy(name):
    dim = HIERS[name][0]
    H, gh = _hier(name, [0] * (2 * dim))
    rng = np.random.default_rng(1)
    F = _rand_field(H, rng)
    P = [a.copy() for a in F]
    cp.average_down_all(H, P)
    for l in range(1, H.lmax + 1):
        cp.fill_cf_ghosts(H, P, l)
    op = _amr().Operator(gh, 0.0, 1.0, [0] * (2 * dim))
    d = _dev(to_packed(gh, H, F, fill=np.nan))
    op.fill_ghosts(d)
    flat = d.cpu().numpy()
    maps = gh.index_maps()
    codes = maps["ghost_code"]
    base = 0
    worst = 0.0
    for p in gh.patches:
        l = p["level"]
        lev = H.levels[l]
        n = [p["hi"][e] - p["lo"][e] + 1 for e in range(dim)]
        ext = [v + 4 for v in n]
        view = gh._view(flat, p)
        cnt = int(np.prod(ext))
        c = codes[base:base + cnt].reshape(ext[::-1])  # [z][y][x]
        for idx in np.argwhere((c == 2) | (c == 3)):
            a = idx[::-1]
            g = [p["lo"][e] - 2 + a[e] for e in range(dim)]
            arr = tuple(g[e] - lev.origin[e] for e in range(dim))
            got = view[tuple(idx)]
            worst = max(worst, abs(got - P[l][arr]))
        base += cnt
    assert worst <= 1e-14 * max_abs(H, F, "covered")


@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("which", [0, 1, 2])
def test_apply_parity_with_boundary_data(name, which):
    dim = HIERS[name][0]
    bc = BCS[dim][which]
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(2 + which)
    F = _rand_field(H, rng)
    data = _bc_data(H, rng)
    for alpha, beta in ((0.0, 1.0), (1.0, -0.01)):
        ref = cp.apply(H, F, alpha, beta, data)
        op = _amr().Operator(gh, alpha, beta, bc)
        d = _dev(to_packed(gh, H, F, fill=np.nan))
        out = torch.zeros_like(d)
        op.apply(d, out, bc=_dev(gh.pack_bc(data)))
        got = from_packed(gh, H, out.cpu().numpy())
        err = max_diff(H, got, ref)
        assert np.isfinite(err)
        assert err <= 1e-13 * op_scale(H, alpha, beta, F), (err, op_scale(H, alpha, beta, F))


@pytest.mark.parametrize("name", list(HIERS))
def test_smoother_parity(name):
    dim = HIERS[name][0]
    bc = BCS[dim][0]
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(5)
    alpha, beta = 1.0, -0.02
    op = _amr().Operator(gh, alpha, beta, bc)
    for l in range(H.lmax + 1):
        X = _rand_field(H, rng, redundant=False)
        B = _rand_field(H, rng, redundant=False)
        diag = mg.jacobi_diagonal(H, l, alpha, beta)
        Xr = X[l].copy()
        for _ in range(3):
            Xr = mg.jacobi(H, l, Xr, B[l], diag, alpha, beta, 2.0 / 3.0)
        dx = _dev(to_packed(gh, H, X))
        db = _dev(to_packed(gh, H, B))
        op.smooth(l, 3, 2.0 / 3.0, dx, db)
        got = from_packed(gh, H, dx.cpu().numpy())
        lev = H.levels[l]
        err = float(np.max(np.abs(got[l][lev.covered] - Xr[lev.covered])))
        assert err <= 1e-12 * float(np.max(np.abs(Xr[lev.covered]))), (l, err)


@pytest.mark.parametrize("name", ["two_level_ragged", "three_level_multibox"])
@pytest.mark.parametrize("bcw", [0, 1])
def test_one_vcycle_parity(name, bcw):
    dim = HIERS[name][0]
    bc = [bcw] * (2 * dim)
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(9)
    alpha, beta = (0.0, 1.0)
    F = _rand_field(H, rng)
    if bcw == 1:
        F, _ = so.solvability_fix(H, F)
    phi = _rand_field(H, rng)
    ref = mg.CompositeMG(H, alpha, beta).vcycle(phi, F)
    op = _amr().Operator(gh, alpha, beta, bc)
    dphi = _dev(to_packed(gh, H, phi))
    op.vcycle(dphi, _dev(to_packed(gh, H, F)))
    got = from_packed(gh, H, dphi.cpu().numpy())
    err = max_diff(H, got, ref)
    assert err <= 1e-10 * max_abs(H, ref), err


SOLVE_CASES = [
    ("two_level_ragged", 0, (1.0, -0.01)),
    ("two_level_ragged", 1, (0.0, 1.0)),
    ("three_level_multibox", 0, (0.0, 1.0)),
    ("three_level_multibox", 1, (0.0, 1.0)),
    ("three_d", 0, (1.0, -0.01)),
    ("three_d", 1, (0.0, 1.0)),
]


@pytest.mark.parametrize("name,bcw,ab", SOLVE_CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_parity(name, bcw, ab, precision):
    amr = _amr()
    dim = HIERS[name][0]
    bc = [bcw] * (2 * dim)
    H, gh = _hier(name, bc)
    alpha, beta = ab
    rng = np.random.default_rng(11)
    F = _rand_field(H, rng)
    Fc = F
    if so.is_pure_neumann(H, alpha):
        Fc, _ = so.solvability_fix(H, F)
    ref, _, _ = so.solve_direct(H, Fc, alpha, beta)
    if so.is_pure_neumann(H, alpha):
        ref, _ = so.mean_zero(H, ref)
    op = amr.Operator(gh, alpha, beta, bc)
    dphi = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
    st = op.solve(dphi, _dev(to_packed(gh, H, F)),
                  params=amr.default_params(rtol=1e-12, max_vcycles=200, precision=precision))
    got = from_packed(gh, H, dphi.cpu().numpy())
    err = max_diff(H, got, ref)
    assert err <= 1e-10 * max_abs(H, ref), (err, st)


def test_solvability_fix_and_mean_zero_parity():
    amr = _amr()
    H, gh = _hier("three_level_multibox", [1, 1, 1, 1])
    rng = np.random.default_rng(13)
    F = _rand_field(H, rng)
    F = [a + 2.5 for a in F]
    data = _bc_data(H, rng)
    ref, m = so.solvability_fix(H, F, beta=1.0, bc_data=data)
    op = amr.Operator(gh, 0.0, 1.0, [1, 1, 1, 1])
    d = _dev(to_packed(gh, H, F))
    mg_ = op.solvability_fix(d, bc=_dev(gh.pack_bc(data)))
    assert abs(mg_ - m) <= 1e-14 * abs(m)
    got = from_packed(gh, H, d.cpu().numpy())
    assert max_diff(H, got, ref) <= 1e-14 * max_abs(H, ref)
    phi = _rand_field(H, rng)
    phi = [a + 1.0 for a in phi]
    refz, mean = so.mean_zero(H, phi)
    dp = _dev(to_packed(gh, H, phi))
    mm = amr.mean_zero(gh, dp)
    assert abs(mm - mean) <= 1e-14 * abs(mean)
    gotz = from_packed(gh, H, dp.cpu().numpy())
    assert max_diff(H, gotz, refz) <= 1e-13 * max_abs(H, phi)


@pytest.mark.parametrize("name", list(HIERS))
def test_gradient_divergence_parity(name):
    amr = _amr()
    dim = HIERS[name][0]
    H, gh = _hier(name, [1] * (2 * dim))
    rng = np.random.default_rng(17)
    phi = _rand_field(H, rng)
    G = cp.gradient(H, phi)
    dphi = _dev(to_packed(gh, H, phi))
    grads = [torch.zeros_like(dphi) for _ in range(dim)]
    amr.gradient(gh, [1] * (2 * dim), dphi, grads)
    scale = max_abs(H, phi, "covered") * 16.0 / (12 * min(l.h for l in H.levels))
    for d in range(dim):
        got = from_packed(gh, H, grads[d].cpu().numpy())
        assert max_diff(H, got, G[d]) <= 1e-13 * scale
    U = [_rand_field(H, rng) for _ in range(dim)]
    Y = cp.divergence(H, U, None, [0] * (2 * dim))
    du = [_dev(to_packed(gh, H, u)) for u in U]
    out = torch.zeros_like(du[0])
    amr.divergence(gh, [0] * (2 * dim), du, out)
    got = from_packed(gh, H, out.cpu().numpy())
    scale = max(max_abs(H, u, "covered") for u in U) * 16.0 * dim / (12 * min(l.h for l in H.levels))
    assert max_diff(H, got, Y) <= 1e-13 * scale


def test_projection_parity():
    amr = _amr()
    H, gh = _hier("two_level_ragged", [1, 1, 1, 1])
    rng = np.random.default_rng(19)
    W = [_rand_field(H, rng) for _ in range(2)]
    Uref, phiref = so.project(H, W)
    ppe = amr.Operator(gh, 0.0, 1.0, [1, 1, 1, 1])
    dw = [_dev(to_packed(gh, H, w)) for w in W]
    du = [torch.zeros_like(dw[0]) for _ in range(2)]
    dphi = torch.zeros_like(dw[0])
    amr.project(ppe, [0, 0, 0, 0], dw, du, dphi, params=amr.default_params(rtol=1e-13, max_vcycles=200))
    for d in range(2):
        got = from_packed(gh, H, du[d].cpu().numpy())
        assert max_diff(H, got, Uref[d], "covered") <= 1e-10 * max_abs(H, Uref[d]), d
    gphi = from_packed(gh, H, dphi.cpu().numpy())
    assert max_diff(H, gphi, phiref) <= 1e-10 * max_abs(H, phiref)


def test_manufactured_solution_order_on_gpu():
    """The 64^2 manufactured-solution workload with inhomogeneous Dirichlet data, solved to
    1e-12: fourth-order convergence of the GPU solution against exact cell averages."""
    amr = _amr()
    from paper_2506_02663_gb300 import workloads as wl
    errs = []
    for n in (32, 64, 128):
        rhs, bcd, exact = wl.ms2d(n)
        gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
        op = amr.Operator(gh, 0.0, 1.0, [0, 0, 0, 0])
        dphi = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        st = op.solve(dphi, _dev(gh.pack([[rhs]])), bc=_dev(gh.pack_bc([bcd])),
                      params=amr.default_params(rtol=1e-12, max_vcycles=100))
        got = gh.unpack(dphi.cpu().numpy())[0][0]
        errs.append(np.sum(np.abs(got - exact)) / n ** 2)
        if n == 64:
            assert st["final_res"] <= 1e-12 * st["rhs_norm"]
    assert np.log2(errs[0] / errs[1]) > 3.8 and np.log2(errs[1] / errs[2]) > 3.8, errs


def test_status_codes_and_nan_corners():
    amr = _amr()
    H, gh = _hier("two_level_ragged", [0, 0, 0, 0])
    rng = np.random.default_rng(23)
    F = _rand_field(H, rng)
    op = amr.Operator(gh, 0.0, 1.0, [0, 0, 0, 0])
    # corners and pitch padding poisoned with NaN: never read by any kernel
    dphi = _dev(to_packed(gh, H, cp.new_field(H), fill=np.nan))
    st = op.solve(dphi, _dev(to_packed(gh, H, F, fill=np.nan)), params=amr.default_params(rtol=1e-10, zero_initial=0))
    assert st["status"] == amr.AMR_OK and np.isfinite(st["final_res"])
    # iteration cap reported as NOT_CONVERGED with valid statistics
    d2 = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
    st = op.solve(d2, _dev(to_packed(gh, H, F)), params=amr.default_params(rtol=1e-14, max_vcycles=1),
                  allow_not_converged=True)
    assert st["status"] == amr.AMR_ERR_NOT_CONVERGED and st["vcycles"] == 1
    # a NaN in the right-hand side is detected by the residual norm
    Fn = to_packed(gh, H, F)
    Fn[gh.patches[0]["offset"] + 3 * gh.patches[0]["sy"] + 3] = np.nan
    with pytest.raises(amr.AmrError) as ei:
        op.solve(torch.zeros_like(d2), _dev(Fn))
    assert ei.value.status == amr.AMR_ERR_NONFINITE
    # bad parameters are rejected on the host before any launch
    with pytest.raises(amr.AmrError) as ei:
        op.solve(d2, _dev(Fn), params=amr.default_params(nu1=-1))
    assert ei.value.status == amr.AMR_ERR_INVALID_ARG


def _bumps2d_gpu(scale=1):
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = wl.bumps2d_rhs(scale)
    return dim, n0, boxes, rhs


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_bumps2d_residual_property(precision):
    """The two-level 256^2 workload at full size in the bench's launch configuration: the
    oracle's own composite operator confirms the GPU solution's residual (PPE and
    Helmholtz), i.e. a property that holds at any size."""
    amr = _amr()
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = _bumps2d_gpu()
    gh = amr.Hierarchy(dim, n0, boxes)
    f = _dev(gh.pack(rhs))
    for bc, (alpha, beta) in (([1, 1, 1, 1], (0.0, 1.0)), ([0, 0, 0, 0], (1.0, wl.HELMHOLTZ_BETA))):
        H = OH(dim, n0, boxes, bc=bc)
        op = amr.Operator(gh, alpha, beta, bc)
        dphi = torch.zeros_like(f)
        st = op.solve(dphi, f, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=precision))
        phi = from_packed(gh, H, dphi.cpu().numpy())
        F = from_packed(gh, H, f.cpu().numpy())
        if so.is_pure_neumann(H, alpha):
            F, m = so.solvability_fix(H, F)
            assert abs(m - st["removed_mean"]) <= 1e-14 * max(abs(m), 1e-300) + 1e-300
        R = cp.residual(H, phi, F, alpha, beta)
        assert max_abs(H, R) <= 1.05e-10 * max_abs(H, F), (max_abs(H, R), st)


@pytest.mark.parametrize("name,bcw,ab", [("two_level_ragged", 1, (0.0, 1.0)), ("three_level_multibox", 0, (1.0, -0.01)),
                                         ("three_d", 1, (0.0, 1.0))])
@pytest.mark.parametrize("precision", [0, 1])
def test_graph_solve_matches_host_loop(name, bcw, ab, precision):
    """The captured solve (one CUDA graph with a device-side while loop over V-cycles)
    performs the same V-cycles as the host-driven loop: same count, same residual history
    to rounding, same solution; relaunching the cached graph reproduces it."""
    amr = _amr()
    dim = HIERS[name][0]
    bc = [bcw] * (2 * dim)
    H, gh = _hier(name, bc)
    alpha, beta = ab
    rng = np.random.default_rng(29)
    F = _rand_field(H, rng)
    op = amr.Operator(gh, alpha, beta, bc)
    f = _dev(to_packed(gh, H, F))
    p0 = amr.default_params(rtol=1e-11, max_vcycles=100, precision=precision)
    p1 = amr.default_params(rtol=1e-11, max_vcycles=100, precision=precision, use_graph=1)
    a = torch.zeros_like(f)
    s0 = op.solve(a, f, params=p0)
    for _ in range(2):
        b = torch.zeros_like(f)
        s1 = op.solve(b, f, params=p1)
        assert s1["vcycles"] == s0["vcycles"], (s0, s1)
        for x, y in zip(s0["res_history"], s1["res_history"]):
            assert abs(x - y) <= 1e-6 * abs(x) + 1e-300
        ga = from_packed(gh, H, a.cpu().numpy())
        gb = from_packed(gh, H, b.cpu().numpy())
        assert max_diff(H, ga, gb) <= 1e-12 * max_abs(H, ga)
    # the iteration cap is reported the same way through the graph
    s2 = op.solve(torch.zeros_like(f), f, params=amr.default_params(rtol=1e-15, max_vcycles=2, use_graph=1,
                                                                   precision=precision), allow_not_converged=True)
    assert s2["status"] == amr.AMR_ERR_NOT_CONVERGED and s2["vcycles"] == 2


@pytest.mark.parametrize("name,bcw,ab", [("two_level_ragged", 1, (0.0, 1.0)), ("three_level_multibox", 0, (1.0, -0.01)),
                                         ("three_d", 0, (0.0, 1.0))])
@pytest.mark.parametrize("precision", [0, 1])
def test_fused_coarse_vcycle_matches_per_grid_kernels(name, bcw, ab, precision):
    """The one-block coarse V-cycle runs the same per-cell arithmetic as the per-grid
    kernels: solves with and without it agree to rounding."""
    amr = _amr()
    dim = HIERS[name][0]
    bc = [bcw] * (2 * dim)
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(37)
    F = _rand_field(H, rng)
    op = amr.Operator(gh, ab[0], ab[1], bc)
    f = _dev(to_packed(gh, H, F))
    out = []
    for fuse in (0, 1):
        x = torch.zeros_like(f)
        st = op.solve(x, f, params=amr.default_params(rtol=1e-11, max_vcycles=100, precision=precision,
                                                      fuse_coarse=fuse))
        out.append((from_packed(gh, H, x.cpu().numpy()), st))
    assert out[0][1]["vcycles"] == out[1][1]["vcycles"]
    assert max_diff(H, out[0][0], out[1][0]) <= 1e-12 * max_abs(H, out[0][0])


@pytest.mark.parametrize("name,bcw,ab", [("two_level_ragged", 1, (0.0, 1.0)), ("three_level_multibox", 0, (1.0, -0.01)),
                                         ("two_level_ragged", 0, (1.0, -0.5))])
def test_temporal_blocking_matches_per_sweep_legs(name, bcw, ab):
    """The blocked down/up legs of the level-0 multigrid (shared-memory tiles with halos) run
    the per-sweep kernels' per-cell arithmetic: one FP64 V-cycle agrees to rounding, and
    solves in both precisions take the same V-cycles to the same solution."""
    amr = _amr()
    dim = HIERS[name][0]
    bc = [bcw] * (2 * dim)
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(39)
    F = _rand_field(H, rng)
    if so.is_pure_neumann(H, ab[0]):
        F, _ = so.solvability_fix(H, F)
    op = amr.Operator(gh, ab[0], ab[1], bc)
    f = _dev(to_packed(gh, H, F))
    outs = []
    for blk in (0, 1):
        x = torch.zeros_like(f)
        op.vcycle(x, f, params=amr.default_params(precision=amr.FP64, temporal_blocking=blk))
        outs.append(from_packed(gh, H, x.cpu().numpy()))
    assert max_diff(H, outs[0], outs[1]) <= 1e-12 * max_abs(H, outs[0])
    for precision in (amr.FP64, amr.MIXED):
        res = []
        for blk in (0, 1):
            x = torch.zeros_like(f)
            st = op.solve(x, f, params=amr.default_params(rtol=1e-11, max_vcycles=100, precision=precision,
                                                          temporal_blocking=blk))
            res.append((from_packed(gh, H, x.cpu().numpy()), st["vcycles"]))
        assert abs(res[0][1] - res[1][1]) <= (0 if precision == amr.FP64 else 1)
        assert max_diff(H, res[0][0], res[1][0]) <= 1e-9 * max_abs(H, res[0][0])


def test_3d_large_grid_smoother_and_apply_parity():
    """A 72^3 single-level grid (blocks far from every face as well as face blocks): three
    FP64 weighted-Jacobi sweeps and the operator with boundary data against the oracle."""
    amr = _amr()
    n = 72
    bc = [0, 1, 0, 0, 1, 0]
    H = OH(3, (n, n, n), [[((0, 0, 0), (n - 1, n - 1, n - 1))]], bc=bc)
    gh = amr.Hierarchy(3, (n, n, n), [[((0, 0, 0), (n - 1, n - 1, n - 1))]], h0=1.0 / n)
    rng = np.random.default_rng(61)
    alpha, beta = 1.0, -0.02
    op = amr.Operator(gh, alpha, beta, bc)
    X = _rand_field(H, rng, redundant=False)
    B = _rand_field(H, rng, redundant=False)
    diag = mg.jacobi_diagonal(H, 0, alpha, beta)
    Xr = X[0].copy()
    for _ in range(3):
        Xr = mg.jacobi(H, 0, Xr, B[0], diag, alpha, beta, 2.0 / 3.0)
    dx = _dev(to_packed(gh, H, X))
    op.smooth(0, 3, 2.0 / 3.0, dx, _dev(to_packed(gh, H, B)))
    got = from_packed(gh, H, dx.cpu().numpy())
    cov = H.levels[0].covered
    assert float(np.max(np.abs(got[0][cov] - Xr[cov]))) <= 1e-12 * float(np.max(np.abs(Xr[cov])))
    data = _bc_data(H, rng)
    ref = cp.apply(H, X, alpha, beta, data)
    out = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
    op.apply(_dev(to_packed(gh, H, X)), out, bc=_dev(gh.pack_bc(data)))
    got = from_packed(gh, H, out.cpu().numpy())
    assert max_diff(H, got, ref) <= 1e-13 * op_scale(H, alpha, beta, X)


@pytest.fixture
def tile_rows():
    amr = _amr()
    yield amr.set_tile_rows
    amr.set_tile_rows(0)


@pytest.fixture
def bulk_sweep():
    amr = _amr()
    yield amr.set_bulk_sweep
    amr.set_bulk_sweep(1)


@pytest.mark.parametrize("n", [(64, 48, 40), (64, 64, 40)])
@pytest.mark.parametrize("rows", [2, 4])
def test_3d_zchunk_operator_parity(n, rows, tile_rows, bulk_sweep):
    """Single-level grids whose x, y extents are multiples of the z-chunked kernel's tile
    (32 x 16 with two rows per thread, 32 x 32 with four; 48 rows fall back to two), so
    blocks sit at every face and z chunks end inside the grid: three FP64 weighted-Jacobi
    sweeps, the homogeneous operator and the residual against the oracle (the bulk-copy
    kernel, which would take these grids, switched off)."""
    amr = _amr()
    tile_rows(rows)
    bulk_sweep(0)
    box = [[((0, 0, 0), tuple(v - 1 for v in n))]]
    bc = [0, 1, 0, 0, 1, 0]
    H = OH(3, n, box, bc=bc, hi=tuple(v / n[0] for v in n))
    gh = amr.Hierarchy(3, n, box, h0=1.0 / n[0])
    rng = np.random.default_rng(67)
    alpha, beta = 1.0, -0.02
    op = amr.Operator(gh, alpha, beta, bc)
    X = _rand_field(H, rng, redundant=False)
    B = _rand_field(H, rng, redundant=False)
    diag = mg.jacobi_diagonal(H, 0, alpha, beta)
    Xr = X[0].copy()
    for _ in range(3):
        Xr = mg.jacobi(H, 0, Xr, B[0], diag, alpha, beta, 2.0 / 3.0)
    dx = _dev(to_packed(gh, H, X))
    op.smooth(0, 3, 2.0 / 3.0, dx, _dev(to_packed(gh, H, B)))
    got = from_packed(gh, H, dx.cpu().numpy())
    cov = H.levels[0].covered
    assert float(np.max(np.abs(got[0][cov] - Xr[cov]))) <= 1e-12 * float(np.max(np.abs(Xr[cov])))
    ref = cp.apply(H, X, alpha, beta, None)
    out = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
    op.apply(_dev(to_packed(gh, H, X)), out)
    got = from_packed(gh, H, out.cpu().numpy())
    assert max_diff(H, got, ref) <= 1e-13 * op_scale(H, alpha, beta, X)
    res = torch.zeros_like(out)
    op.residual(_dev(to_packed(gh, H, X)), _dev(to_packed(gh, H, B)), res)
    got = from_packed(gh, H, res.cpu().numpy())
    refr = [B[l] - ref[l] for l in range(len(ref))]
    assert max_diff(H, got, refr) <= 1e-13 * op_scale(H, alpha, beta, X)


def _level_ops(amr, op, gh, H, X, B):
    """Three FP64 weighted-Jacobi sweeps, the operator and the residual through the C ABI."""
    dx = _dev(to_packed(gh, H, X))
    op.smooth(0, 3, 2.0 / 3.0, dx, _dev(to_packed(gh, H, B)))
    out = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
    op.apply(_dev(to_packed(gh, H, X)), out)
    res = torch.zeros_like(out)
    op.residual(_dev(to_packed(gh, H, X)), _dev(to_packed(gh, H, B)), res)
    return [from_packed(gh, H, t.cpu().numpy()) for t in (dx, out, res)]


@pytest.mark.parametrize("n,bc", [((64, 48, 40), [0, 1, 0, 0, 1, 0]), ((128, 32, 16), [1, 0, 1, 1, 0, 1]),
                                  ((64, 16, 64), [1, 1, 0, 1, 0, 0])])
def test_3d_bulk_sweep_operator_parity(n, bc, bulk_sweep):
    """The bulk-copy pipelined 3-D level operator, forced (64 x 16 tiles, z chunks of at least
    eight planes, ghost values written into the staged planes at every face of both types) on single-level grids with one or two
    tiles across x and several across y: three FP64 weighted-Jacobi sweeps, the operator and
    the residual against the oracle, and against the z-chunked kernel (the same operations
    per cell) to 1e-14."""
    amr = _amr()
    box = [[((0, 0, 0), tuple(v - 1 for v in n))]]
    H = OH(3, n, box, bc=bc, hi=tuple(v / n[0] for v in n))
    gh = amr.Hierarchy(3, n, box, h0=1.0 / n[0])
    rng = np.random.default_rng(71)
    alpha, beta = 1.0, -0.02
    op = amr.Operator(gh, alpha, beta, bc)
    X = _rand_field(H, rng, redundant=False)
    B = _rand_field(H, rng, redundant=False)
    bulk_sweep(2)
    got = _level_ops(amr, op, gh, H, X, B)
    amr.check_kernel_flags()
    bulk_sweep(0)
    zc = _level_ops(amr, op, gh, H, X, B)
    diag = mg.jacobi_diagonal(H, 0, alpha, beta)
    Xr = X[0].copy()
    for _ in range(3):
        Xr = mg.jacobi(H, 0, Xr, B[0], diag, alpha, beta, 2.0 / 3.0)
    cov = H.levels[0].covered
    sx = float(np.max(np.abs(Xr[cov])))
    assert float(np.max(np.abs(got[0][0][cov] - Xr[cov]))) <= 1e-12 * sx
    assert float(np.max(np.abs(got[0][0][cov] - zc[0][0][cov]))) <= 1e-14 * sx
    ref = cp.apply(H, X, alpha, beta, None)
    scale = op_scale(H, alpha, beta, X)
    assert max_diff(H, got[1], ref) <= 1e-13 * scale
    assert max_diff(H, got[1], zc[1]) <= 1e-14 * scale
    refr = [B[l] - ref[l] for l in range(len(ref))]
    assert max_diff(H, got[2], refr) <= 1e-13 * scale
    assert max_diff(H, got[2], zc[2]) <= 1e-14 * scale


@pytest.mark.parametrize("bcw,ab", [(0, (1.0, -0.01)), (1, (0.0, 1.0))])
@pytest.mark.parametrize("n", [(64, 32, 32), (32, 32, 16)])
@pytest.mark.parametrize("fuse", [2, 0])
def test_3d_coarse_cluster_vcycle_and_transpose(n, bcw, ab, fuse):
    """Single-level grids whose multigrid ends in grids of at most 32^3 cells: 64 x 32 x 32
    (the cluster takes 32 x 16 x 16 -> 16 x 8 x 8 -> 8 x 4 x 4) and 32 x 32 x 16 (the cluster
    takes the level itself).  fuse_coarse = 2 runs those grids as one cluster launch, 0 as
    per-grid launches.  One FP64 V-cycle against the oracle's V-cycle; mixed and FP64 solves
    whose residual the oracle recomputes; and on the smaller grid the adjoint solve, whose
    level-0 V-cycles take the same path, checked by the residual of the oracle's assembled
    transposed system."""
    amr = _amr()
    box = [[((0, 0, 0), tuple(v - 1 for v in n))]]
    bc = [0, 1, 0, 0, 1, 0] if bcw == 0 else [1] * 6
    alpha, beta = ab
    H = OH(3, n, box, bc=bc, hi=tuple(v / n[0] for v in n))
    gh = amr.Hierarchy(3, n, box, h0=1.0 / n[0])
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(79)
    F = _rand_field(H, rng, redundant=False)
    if so.is_pure_neumann(H, alpha):
        F, _ = so.solvability_fix(H, F)
    phi = _rand_field(H, rng, redundant=False)
    ref = mg.CompositeMG(H, alpha, beta).vcycle(phi, F)
    dphi = _dev(to_packed(gh, H, phi))
    op.vcycle(dphi, _dev(to_packed(gh, H, F)), params=amr.default_params(fuse_coarse=fuse))
    got = from_packed(gh, H, dphi.cpu().numpy())
    assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref)
    for prec in (0, 1):
        x = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        st = op.solve(x, _dev(to_packed(gh, H, F)), params=amr.default_params(
            rtol=1e-10, max_vcycles=100, precision=prec, use_graph=1, fuse_coarse=fuse))
        R = cp.residual(H, from_packed(gh, H, x.cpu().numpy()), F, alpha, beta)
        assert max_abs(H, R) <= 1.05e-10 * max_abs(H, F), (prec, st)
    if alpha != 0.0 and n == (32, 32, 16) and fuse == 2:
        U = so.Unknowns(H)
        A, _ = so.helmholtz_matrix(H, alpha, beta)
        g = rng.standard_normal(U.n)
        dl = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        op.solve_transpose(dl, _dev(to_packed(gh, H, U.scatter(g, fill_invalid=False))),
                           params=amr.default_params(rtol=1e-12, max_vcycles=100, fuse_coarse=fuse))
        lam = U.gather(from_packed(gh, H, dl.cpu().numpy()))
        assert np.max(np.abs(g - A.T @ lam)) <= 2e-12 * np.max(np.abs(g))


@pytest.mark.parametrize("bcw,ab", [(0, (1.0, -0.01)), (1, (0.0, 1.0))])
def test_3d_bulk_sweep_two_level_vcycle_and_solve(bcw, ab, bulk_sweep):
    """Two-level 3-D hierarchy whose base (64 x 32 x 16, covered cells masked in the residual)
    and fine box (64 x 32 x 16 fine cells, coarse-fine ghosts stored in the halo) both take
    the bulk-copy kernel: one FP64 V-cycle against the oracle's V-cycle, then mixed-precision
    solves to 1e-10 with the bulk-copy and the z-chunked kernels (same V-cycle count, same
    solution to 1e-12), the residual recomputed by the oracle's composite operator."""
    amr = _amr()
    n0 = (64, 32, 16)
    boxes = [[((0, 0, 0), (63, 31, 15))], [((32, 16, 8), (95, 47, 23))]]
    bc = [bcw] * 6
    alpha, beta = ab
    H = OH(3, n0, boxes, bc=bc, hi=(1.0, 0.5, 0.25))
    gh = amr.Hierarchy(3, n0, boxes, h0=1.0 / 64)
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(73)
    F = _rand_field(H, rng)
    if bcw == 1:
        F, _ = so.solvability_fix(H, F)
    phi = _rand_field(H, rng)
    bulk_sweep(2)
    ref = mg.CompositeMG(H, alpha, beta).vcycle(phi, F)
    dphi = _dev(to_packed(gh, H, phi))
    df = _dev(to_packed(gh, H, F))
    op.vcycle(dphi, df)
    got = from_packed(gh, H, dphi.cpu().numpy())
    assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref)
    sols = []
    for on in (2, 0):
        bulk_sweep(on)
        x = torch.zeros_like(df)
        st = op.solve(x, df, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=1, use_graph=1))
        sols.append((from_packed(gh, H, x.cpu().numpy()), st["vcycles"]))
    assert sols[0][1] == sols[1][1]
    assert max_diff(H, sols[0][0], sols[1][0]) <= 1e-12 * max_abs(H, sols[1][0])
    R = cp.residual(H, sols[0][0], F, alpha, beta)
    assert max_abs(H, R) <= 1.05e-10 * max_abs(H, F)


@pytest.mark.parametrize("precision", [0, 1])
def test_3d_bulk_restriction_matches_generic(bulk_sweep, precision):
    """The residual restriction of the multigrid down leg by the bulk-copy kernel (128 x 64 x
    32 grid with every face type; its next grid 64 x 32 x 16 also takes it): one V-cycle, in
    FP64 and in the FP32 correction cycle of mixed precision, bit for bit equal to the
    z-chunked kernels with the generic restriction (same children order and arithmetic), and
    the FP64 one equal to the oracle's V-cycle to 1e-10."""
    amr = _amr()
    n = (128, 64, 32)
    box = [[((0, 0, 0), tuple(v - 1 for v in n))]]
    bc = [0, 1, 1, 0, 0, 1]
    alpha, beta = 1.0, -0.02
    H = OH(3, n, box, bc=bc, hi=tuple(v / n[0] for v in n))
    gh = amr.Hierarchy(3, n, box, h0=1.0 / n[0])
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(97)
    F = _rand_field(H, rng, redundant=False)
    phi = _rand_field(H, rng, redundant=False)
    got = {}
    for on in (2, 0):
        bulk_sweep(on)
        dphi = _dev(to_packed(gh, H, phi))
        if precision == 0:
            op.vcycle(dphi, _dev(to_packed(gh, H, F)))
        else:  # two refinement steps, each one FP32 correction V-cycle
            op.solve(dphi, _dev(to_packed(gh, H, F)), allow_not_converged=True,
                     params=amr.default_params(rtol=1e-30, max_vcycles=2, precision=1, use_graph=0))
        got[on] = dphi.cpu().numpy()
    assert np.array_equal(got[2], got[0])
    if precision == 0:
        ref = mg.CompositeMG(H, alpha, beta).vcycle(phi, F)
        g = from_packed(gh, H, got[2])
        assert max_diff(H, g, ref) <= 1e-10 * max_abs(H, ref)


@pytest.fixture
def fx_switch():
    amr = _amr()
    yield amr.set_fx_residual
    amr.set_fx_residual(1)


@pytest.mark.parametrize("bulk", [0, 2])
def test_3d_fixed_point_residual(fx_switch, bulk_sweep, bulk):
    """The 3-D FP64 residual with exact fixed-point stencil sums (the default on tile-multiple
    single-patch levels) against the oracle and the plain FP64 kernel on a 64 x 64 x 40 grid
    with Dirichlet and Neumann faces, in both forms: the z-chunked kernel (bulk = 0) and the
    bulk-copy kernel whose converter warps rewrite the staged planes as integers (bulk = 2;
    five z chunks, so chunks on both z faces and between them).  A smooth field that meets
    the boundary conditions and a rough one (whose layer-2 Dirichlet ghost values reach about
    50 times the interior values) both stay in the frame, so the fixed-point result is the
    one returned (it differs from the plain kernel's in rounding only); phi = 0 (the
    refinement loop's first residual) gives f exactly."""
    amr = _amr()
    bulk_sweep(bulk)
    n = (64, 64, 40)
    box = [[((0, 0, 0), tuple(v - 1 for v in n))]]
    bc = [0, 1, 0, 0, 1, 0]
    hi = tuple(v / n[0] for v in n)
    H = OH(3, n, box, bc=bc, hi=hi)
    gh = amr.Hierarchy(3, n, box, h0=1.0 / n[0])
    alpha, beta = 1.0, -0.02
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(73)
    B = _rand_field(H, rng, redundant=False)
    h = 1.0 / n[0]
    xc, yc, zc = np.meshgrid(*[(np.arange(m) + 0.5) * h for m in n], indexing="ij")
    lev = H.levels[0]
    smooth = np.zeros(lev.shape)
    smooth[lev.box_slice(*box[0][0])] = (np.sin(0.5 * np.pi * xc) * np.sin(np.pi * yc) *
                                         np.cos(0.5 * np.pi * zc / hi[2]) * 3.7)
    cases = {"smooth": [smooth], "rough": _rand_field(H, rng, redundant=False), "zero": [np.zeros(lev.shape)]}
    for name, X in cases.items():
        dx, df = _dev(to_packed(gh, H, X)), _dev(to_packed(gh, H, B))
        got = {}
        for on in (1, 0):
            fx_switch(on)
            res = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
            op.residual(dx, df, res)
            got[on] = res.cpu().numpy()
        fx_switch(1)
        ref = cp.apply(H, X, alpha, beta, None)
        refr = [B[0] - ref[0]]
        for on in (1, 0):
            g = from_packed(gh, H, got[on])
            assert max_diff(H, g, refr) <= 1e-13 * op_scale(H, alpha, beta, X) + 1e-300, (name, on)
        if name == "zero":
            assert np.array_equal(got[1], got[0])
        else:
            assert not np.array_equal(got[1], got[0]), name


def test_3d_fixed_point_residual_fallback(fx_switch):
    """Two z-chunked levels (base 32 x 32 x 16, a 32 x 16 x 16 fine box) whose fine level
    holds values a thousand times smaller than the coarse level around it: its coarse-fine
    ghost values leave the fine level's frame, so the gated FP64 kernel recomputes that level
    (bit for bit the plain kernel's result), while the base level keeps the fixed-point
    result; the composite residual matches the oracle either way."""
    amr = _amr()
    n0 = (32, 32, 16)
    boxes = [[((0, 0, 0), (31, 31, 15))], [((16, 16, 8), (47, 31, 23))]]
    bc = [0, 1, 0, 0, 1, 0]
    alpha, beta = 1.0, -0.01
    H = OH(3, n0, boxes, bc=bc, hi=tuple(v / n0[0] for v in n0))
    gh = amr.Hierarchy(3, n0, boxes, h0=1.0 / n0[0])
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(79)
    X = _rand_field(H, rng)
    X[1] = X[1] * 1e-3
    B = _rand_field(H, rng)
    ref = cp.residual(H, X, B, alpha, beta)
    got = {}
    for on in (1, 0):
        fx_switch(on)
        res = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        op.residual(_dev(to_packed(gh, H, X)), _dev(to_packed(gh, H, B)), res)
        got[on] = from_packed(gh, H, res.cpu().numpy())
    fx_switch(1)
    for on in (1, 0):
        assert max_diff(H, got[on], ref) <= 1e-13 * op_scale(H, alpha, beta, X), on
    v0, v1 = H.levels[0].valid, H.levels[1].valid
    assert np.array_equal(got[1][1][v1], got[0][1][v1])
    assert not np.array_equal(got[1][0][v0], got[0][0][v0])


def test_3d_fixed_point_residual_forms_agree(fx_switch, bulk_sweep):
    """The two fixed-point forms (z-chunked, bulk-copy) on a 128 x 64 x 48 grid with every
    face type: both within 1e-13 of the oracle's residual, and bit for bit equal (the same
    frame, the same exact sums, ghost values and multiply-adds)."""
    amr = _amr()
    n = (128, 64, 48)
    box = [[((0, 0, 0), tuple(v - 1 for v in n))]]
    bc = [1, 0, 0, 1, 0, 1]
    hi = tuple(v / n[0] for v in n)
    H = OH(3, n, box, bc=bc, hi=hi)
    gh = amr.Hierarchy(3, n, box, h0=1.0 / n[0])
    alpha, beta = 1.0, -0.03
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(83)
    X = _rand_field(H, rng, redundant=False)
    B = _rand_field(H, rng, redundant=False)
    dx, df = _dev(to_packed(gh, H, X)), _dev(to_packed(gh, H, B))
    got = {}
    for bulk in (0, 2):
        bulk_sweep(bulk)
        res = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        op.residual(dx, df, res)
        got[bulk] = from_packed(gh, H, res.cpu().numpy())
    ref = cp.residual(H, X, B, alpha, beta)
    scale = op_scale(H, alpha, beta, X)
    for bulk in (0, 2):
        assert max_diff(H, got[bulk], ref) <= 1e-13 * scale, bulk
    assert max_diff(H, got[0], got[2]) == 0.0


def test_3d_fixed_point_residual_fallback_bulk(fx_switch, bulk_sweep):
    """The out-of-frame fallback behind the bulk-copy form: base 64 x 32 x 16 and a 64 x 16 x
    16 fine box (both bulk-copy levels) whose values are a thousand times smaller than the
    coarse level around it; its coarse-fine ghost values leave its frame, the converter warps
    raise the flag and the gated FP64 kernel recomputes the fine level (bit for bit the plain
    kernel's result), while the base level keeps the fixed-point result; the composite
    residual matches the oracle either way."""
    amr = _amr()
    bulk_sweep(2)
    n0 = (64, 32, 16)
    boxes = [[((0, 0, 0), (63, 31, 15))], [((32, 16, 8), (95, 31, 23))]]
    bc = [0, 1, 1, 0, 0, 1]
    alpha, beta = 1.0, -0.01
    H = OH(3, n0, boxes, bc=bc, hi=tuple(v / n0[0] for v in n0))
    gh = amr.Hierarchy(3, n0, boxes, h0=1.0 / n0[0])
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(89)
    X = _rand_field(H, rng)
    X[1] = X[1] * 1e-3
    B = _rand_field(H, rng)
    ref = cp.residual(H, X, B, alpha, beta)
    got = {}
    for on in (1, 0):
        fx_switch(on)
        res = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        op.residual(_dev(to_packed(gh, H, X)), _dev(to_packed(gh, H, B)), res)
        got[on] = from_packed(gh, H, res.cpu().numpy())
    fx_switch(1)
    for on in (1, 0):
        assert max_diff(H, got[on], ref) <= 1e-13 * op_scale(H, alpha, beta, X), on
    v0, v1 = H.levels[0].valid, H.levels[1].valid
    assert np.array_equal(got[1][1][v1], got[0][1][v1])
    assert not np.array_equal(got[1][0][v0], got[0][0][v0])


@pytest.mark.parametrize("precision", [0, 1])
def test_bumps3d_quarter_size_residual_property(precision):
    """The 3-D workload at a quarter of its size (base 64^3, a 32^3 fine box over
    [0.375,0.625]^3, Gaussian-bump right-hand side; both levels take the z-chunked kernels
    and the fixed-point FP64 residual): the PPE and the Helmholtz solves to 1e-10, whose
    residual, recomputed by the oracle's composite operator, meets the tolerance."""
    amr = _amr()
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = wl.bumps3d_rhs(scale=4)
    gh = amr.Hierarchy(dim, n0, boxes)
    f = _dev(gh.pack(rhs))
    for bc, (alpha, beta) in (([1] * 6, (0.0, 1.0)), ([0] * 6, (1.0, wl.HELMHOLTZ_BETA))):
        H = OH(dim, n0, boxes, bc=bc)
        op = amr.Operator(gh, alpha, beta, bc)
        dphi = torch.zeros_like(f)
        st = op.solve(dphi, f, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=precision))
        phi = from_packed(gh, H, dphi.cpu().numpy())
        F = from_packed(gh, H, f.cpu().numpy())
        if so.is_pure_neumann(H, alpha):
            F, _ = so.solvability_fix(H, F)
        R = cp.residual(H, phi, F, alpha, beta)
        assert max_abs(H, R) <= 1.05e-10 * max_abs(H, F), (bc[0], max_abs(H, R) / max_abs(H, F), st)


def test_3d_large_grid_prolongation_vcycle_parity():
    """A single-level 128^3 Helmholtz problem with Dirichlet and Neumann faces: its multigrid
    prolongs from a 64^3 grid, so every V-cycle takes the large-grid prolongation (four fine
    cells per thread along z, the domain-face layer in its own launch) that the 256^3
    workload runs.  One FP64 V-cycle against the oracle's V-cycle (Sec. 6.5: linear
    interpolation, homogeneous extension at the faces), then a mixed-precision solve whose
    residual the oracle's operator recomputes."""
    amr = _amr()
    n = 128
    bc = [0, 1, 1, 0, 0, 1]
    box = [[((0, 0, 0), (n - 1, n - 1, n - 1))]]
    H = OH(3, (n, n, n), box, bc=bc)
    gh = amr.Hierarchy(3, (n, n, n), box, h0=1.0 / n)
    alpha, beta = 1.0, -0.01
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(67)
    F = _rand_field(H, rng, redundant=False)
    phi = _rand_field(H, rng, redundant=False)
    ref = mg.CompositeMG(H, alpha, beta).vcycle(phi, F)
    dphi = _dev(to_packed(gh, H, phi))
    df = _dev(to_packed(gh, H, F))
    op.vcycle(dphi, df)
    got = from_packed(gh, H, dphi.cpu().numpy())
    assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref)
    dphi = torch.zeros_like(df)
    st = op.solve(dphi, df, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=1, use_graph=1))
    R = cp.residual(H, from_packed(gh, H, dphi.cpu().numpy()), F, alpha, beta)
    assert max_abs(H, R) <= 1.05e-10 * max_abs(H, F), (max_abs(H, R) / max_abs(H, F), st)


@pytest.mark.parametrize("precision", [0, 1])
def test_bumps3d_full_size_residual_property(precision):
    """The 3-D workload at full size (base 256^3, a 128^3 fine box over [0.375,0.625]^3) in
    the bench's launch configuration (captured solve graph): the pure-Neumann PPE and one
    velocity component's Helmholtz system solved to 1e-10, each residual recomputed by the
    oracle's composite operator (a property that holds at any size)."""
    amr = _amr()
    from paper_2506_02663_gb300 import workloads as wl
    for comp, bc, (alpha, beta) in ((0, [1] * 6, (0.0, 1.0)), (1, [0] * 6, (1.0, wl.HELMHOLTZ_BETA))):
        dim, n0, boxes, rhs = wl.bumps3d_rhs(component=comp)
        gh = amr.Hierarchy(dim, n0, boxes)
        f = _dev(gh.pack(rhs))
        H = OH(dim, n0, boxes, bc=bc)
        op = amr.Operator(gh, alpha, beta, bc)
        dphi = torch.zeros_like(f)
        st = op.solve(dphi, f, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=precision,
                                                         use_graph=1))
        phi = from_packed(gh, H, dphi.cpu().numpy())
        del dphi
        F = from_packed(gh, H, f.cpu().numpy())
        if so.is_pure_neumann(H, alpha):
            F, m = so.solvability_fix(H, F)
            assert abs(m - st["removed_mean"]) <= 1e-13 * max(abs(m), 1e-300) + 1e-300
        R = cp.residual(H, phi, F, alpha, beta)
        assert max_abs(H, R) <= 1.05e-10 * max_abs(H, F), (bc[0], max_abs(H, R) / max_abs(H, F), st)
        op.close()
        gh.close()


@pytest.mark.parametrize("bcw,ab", [(0, (1.0, -0.01)), (1, (0.0, 1.0))])
@pytest.mark.parametrize("rows", [2, 4])
def test_3d_zchunk_two_level_vcycle_and_solve(bcw, ab, rows, tile_rows):
    """Two-level 3-D hierarchy whose levels both run the z-chunked kernel (base 32 x 32 x 16,
    one ratio-2 box of 32 x 16 x 16 fine cells, covered cells on the base): one FP64 V-cycle
    against the oracle's, and mixed- and FP64 solves to 1e-10 whose residual, recomputed by
    the oracle, meets the tolerance."""
    amr = _amr()
    tile_rows(rows)
    n0 = (32, 32, 16)
    boxes = [[((0, 0, 0), (31, 31, 15))], [((16, 16, 8), (47, 31, 23))]]
    bc = [bcw] * 6
    alpha, beta = ab
    H = OH(3, n0, boxes, bc=bc, hi=tuple(v / n0[0] for v in n0))
    gh = amr.Hierarchy(3, n0, boxes, h0=1.0 / n0[0])
    rng = np.random.default_rng(71)
    F = _rand_field(H, rng)
    if so.is_pure_neumann(H, alpha):
        F, _ = so.solvability_fix(H, F)
    phi = _rand_field(H, rng)
    ref = mg.CompositeMG(H, alpha, beta).vcycle(phi, F)
    op = amr.Operator(gh, alpha, beta, bc)
    dphi = _dev(to_packed(gh, H, phi))
    op.vcycle(dphi, _dev(to_packed(gh, H, F)))
    got = from_packed(gh, H, dphi.cpu().numpy())
    assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref)
    for precision in (amr.FP64, amr.MIXED):
        x = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        st = op.solve(x, _dev(to_packed(gh, H, F)),
                      params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=precision))
        sol = from_packed(gh, H, x.cpu().numpy())
        r = cp.residual(H, sol, F, alpha, beta)
        fmax = max_abs(H, F)
        rmax = max(float(np.max(np.abs(r[l][lev.valid]))) for l, lev in enumerate(H.levels))
        assert rmax <= 1.5e-10 * fmax, (precision, rmax / fmax, st)


SQUARE_CASES = {
    # level-0 pyramid 64, 32, 16, 8, 4: the whole level-0 V-cycle in the one-block kernel
    "single64": (2, (64, 64), [[((0, 0), (63, 63))]]),
    # 96, then 48, 24, 12, 6 in the one-block kernel
    "single96": (2, (96, 96), [[((0, 0), (95, 95))]]),
    # two levels over a 64^2 base
    "two_level64": (2, (64, 64), [[((0, 0), (63, 63))], [((32, 40), (87, 95))]]),
}


@pytest.mark.parametrize("name", list(SQUARE_CASES))
@pytest.mark.parametrize("bcw,ab", [(0, (1.0, -0.01)), (1, (0.0, 1.0))])
def test_square_coarse_block_solves(name, bcw, ab):
    """Square level-0 pyramids run the compile-time-size one-block coarse V-cycle (ghost values
    evaluated where the stencil reads them): mixed-precision solves reach the oracle's direct
    solution to 1e-10 and take the same number of V-cycles (+-1) as the per-sweep kernels."""
    amr = _amr()
    dim, n0, boxes = SQUARE_CASES[name]
    bc = [bcw] * (2 * dim)
    alpha, beta = ab
    H = OH(dim, n0, boxes, bc=bc, hi=(1.0, 1.0))
    gh = amr.Hierarchy(dim, n0, boxes, h0=1.0 / n0[0])
    rng = np.random.default_rng(73)
    F = _rand_field(H, rng)
    Fc = F
    if so.is_pure_neumann(H, alpha):
        Fc, _ = so.solvability_fix(H, F)
    ref, _, _ = so.solve_direct(H, Fc, alpha, beta)
    if so.is_pure_neumann(H, alpha):
        ref, _ = so.mean_zero(H, ref)
    op = amr.Operator(gh, alpha, beta, bc)
    f = _dev(to_packed(gh, H, F))
    counts = []
    for blk in (1, 0):
        x = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        st = op.solve(x, f, params=amr.default_params(rtol=1e-12, max_vcycles=200, precision=amr.MIXED,
                                                      temporal_blocking=blk))
        got = from_packed(gh, H, x.cpu().numpy())
        assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref), (blk, st)
        counts.append(st["vcycles"])
    assert abs(counts[0] - counts[1]) <= 1, counts


@pytest.mark.parametrize("bcw,ab", [(0, (1.0, -1e-4)), (1, (0.0, 1.0))])
def test_blocked_legs_large_tiles(bcw, ab):
    """A 1024^2 single level takes the blocked legs with 32^2 tiles: mixed-precision solves
    with and without temporal blocking take the same V-cycles (+-1) and agree to 1e-9, and
    the oracle's residual of the blocked solution meets the tolerance."""
    amr = _amr()
    n = 1024
    box = [[((0, 0), (n - 1, n - 1))]]
    bc = [bcw] * 4
    alpha, beta = ab
    H = OH(2, (n, n), box, bc=bc, hi=(1.0, 1.0))
    gh = amr.Hierarchy(2, (n, n), box, h0=1.0 / n)
    rng = np.random.default_rng(79)
    F = _rand_field(H, rng)
    if so.is_pure_neumann(H, alpha):
        F, _ = so.solvability_fix(H, F)
    op = amr.Operator(gh, alpha, beta, bc)
    f = _dev(to_packed(gh, H, F))
    sols, counts = [], []
    for blk in (1, 0):
        x = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        st = op.solve(x, f, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=amr.MIXED,
                                                      temporal_blocking=blk))
        sols.append(from_packed(gh, H, x.cpu().numpy()))
        counts.append(st["vcycles"])
    assert abs(counts[0] - counts[1]) <= 1, counts
    assert max_diff(H, sols[0], sols[1]) <= 1e-9 * max_abs(H, sols[1])
    r = cp.residual(H, sols[0], F, alpha, beta)
    rmax = float(np.max(np.abs(r[0][H.levels[0].valid])))
    assert rmax <= 1.5e-10 * max_abs(H, F), rmax / max_abs(H, F)


def test_manufactured_solution_matches_golden_values():
    """The 64^2 manufactured-solution solve on the GPU against the stored oracle values of
    tests/golden/ms2d.json: sampled cells to 1e-10 of max|phi| and the error norms against
    the exact cell averages to 1e-4 relative (a 1e-10 |phi| deviation moves norms of about
    2e-6 by at most that much)."""
    import json
    import os
    amr = _amr()
    from paper_2506_02663_gb300 import workloads as wl
    golden = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ms2d.json")))
    n = golden["n"]
    rhs, bcd, exact = wl.ms2d(n)
    gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
    op = amr.Operator(gh, 0.0, 1.0, [0, 0, 0, 0])
    for precision in (amr.FP64, amr.MIXED):
        dphi = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        op.solve(dphi, _dev(gh.pack([[rhs]])), bc=_dev(gh.pack_bc([bcd])),
                 params=amr.default_params(rtol=1e-12, max_vcycles=100, precision=precision))
        got = gh.unpack(dphi.cpu().numpy())[0][0]
        scale = float(np.max(np.abs(got)))
        for (i, j), v in zip(golden["cells_ij"], golden["phi"]):
            assert abs(got[i, j] - v) <= 1e-10 * scale, (precision, i, j)
        e = got - exact
        h = 1.0 / n
        errs = (np.sum(np.abs(e)) * h * h, np.sqrt(np.sum(e * e) * h * h), np.max(np.abs(e)))
        for a, b in zip(errs, golden["err_l1_l2_linf"]):
            assert abs(a - b) <= 1e-4 * b, (precision, a, b)


def test_amr2d_composite_solves_match_golden_values():
    """The two-level 32^2 + ratio-2 box workload (Gaussian-bump right-hand side) on the GPU
    against the stored oracle values of tests/golden/amr2d.json: the pure-Neumann PPE
    (solvability fix, mean-zero result) and the Dirichlet Helmholtz system, FP64 and mixed
    precision, sampled valid cells of both levels to 1e-10 of max|phi|."""
    import json
    import os
    amr = _amr()
    from paper_2506_02663_gb300 import workloads as wl
    golden = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "amr2d.json")))
    dim, n0, boxes, rhs = wl.bumps2d_rhs(scale=8)
    assert list(n0) == golden["n0"]
    gh = amr.Hierarchy(dim, n0, boxes)
    f = _dev(gh.pack(rhs))
    for name, bc, alpha, beta in (("ppe", [1] * 4, 0.0, 1.0), ("helmholtz", [0] * 4, 1.0, wl.HELMHOLTZ_BETA)):
        H = OH(dim, n0, boxes, bc=bc)
        op = amr.Operator(gh, alpha, beta, bc)
        scale = golden[name]["max_abs"]
        for precision in (amr.FP64, amr.MIXED):
            dphi = torch.zeros_like(f)
            op.solve(dphi, f, params=amr.default_params(rtol=1e-12, max_vcycles=100, precision=precision))
            got = from_packed(gh, H, dphi.cpu().numpy())
            for l, i, j, v in golden[name]["samples_level_index_value"]:
                assert abs(got[l][i, j] - v) <= 1e-10 * scale, (name, precision, l, i, j, got[l][i, j], v)


def test_amr3d_composite_solves_match_golden_values():
    """The 3-D workload at 1/8 size (32^3 base, 16^3 fine box over [0.375, 0.625]^3) against
    the stored oracle values of tests/golden/amr3d.json (direct solves of the composite
    systems): the pure-Neumann PPE (solvability fix, mean-zero result) and a velocity
    component's Dirichlet Helmholtz system, FP64 and mixed precision, sampled valid cells of
    both levels to 1e-10 of max|phi|."""
    import json
    import os
    amr = _amr()
    from paper_2506_02663_gb300 import workloads as wl
    golden = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "amr3d.json")))
    for name, comp, bc, alpha, beta in (("ppe", 0, [1] * 6, 0.0, 1.0), ("helmholtz", 1, [0] * 6, 1.0, wl.HELMHOLTZ_BETA)):
        dim, n0, boxes, rhs = wl.bumps3d_rhs(scale=8, component=comp)
        assert list(n0) == golden["n0"]
        gh = amr.Hierarchy(dim, n0, boxes)
        f = _dev(gh.pack(rhs))
        H = OH(dim, n0, boxes, bc=bc)
        op = amr.Operator(gh, alpha, beta, bc)
        scale = golden[name]["max_abs"]
        for precision in (amr.FP64, amr.MIXED):
            dphi = torch.zeros_like(f)
            op.solve(dphi, f, params=amr.default_params(rtol=1e-12, max_vcycles=100, precision=precision))
            got = from_packed(gh, H, dphi.cpu().numpy())
            for l, i, j, k, v in golden[name]["samples_level_index_value"]:
                assert abs(got[l][i, j, k] - v) <= 1e-10 * scale, (name, precision, l, i, j, k, got[l][i, j, k], v)
        op.close()
        gh.close()


@pytest.mark.parametrize("bc,ab", [([0, 1, 1, 0, 0, 1], (1.0, -0.02)), ([0] * 6, (0.0, 1.0))])
@pytest.mark.parametrize("two_level", [False, True])
def test_3d_cube_coarse_fp32_vcycle(bc, ab, two_level):
    """The one-block coarse V-cycle of 3-D pyramids ending 16^3, 8^3, 4^3 (FP32, the default
    coarse end of such pyramids): one mixed-precision step from zero (one FP32 V-cycle on f)
    against the oracle's FP64 V-cycle to FP32 accuracy, on a 32^3 base (pyramid 32, 16, 8, 4)
    alone and with a fine box; then solves to 1e-10 with it and with the cluster coarse end
    (fuse_coarse = 2): the same V-cycle count (within one), both meeting the tolerance by the
    oracle's composite residual."""
    amr = _amr()
    n0 = (32, 32, 32)
    boxes = [[((0, 0, 0), (31, 31, 31))]]
    if two_level:
        boxes.append([((16, 16, 16), (47, 47, 47))])
    alpha, beta = ab
    H = OH(3, n0, boxes, bc=bc, hi=(1.0, 1.0, 1.0))
    gh = amr.Hierarchy(3, n0, boxes, h0=1.0 / 32)
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(103)
    F = _rand_field(H, rng)
    df = _dev(to_packed(gh, H, F))
    x = torch.zeros_like(df)
    op.solve(x, df, allow_not_converged=True,
             params=amr.default_params(rtol=1e-30, max_vcycles=1, precision=1, use_graph=0))
    ref = mg.CompositeMG(H, alpha, beta).vcycle(cp.new_field(H), F)
    got = from_packed(gh, H, x.cpu().numpy())
    assert max_diff(H, got, ref) <= 2e-5 * max_abs(H, ref)
    out = []
    for fuse in (0, 2):
        y = torch.zeros_like(df)
        st = op.solve(y, df, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=1, use_graph=1,
                                                         fuse_coarse=fuse))
        out.append((from_packed(gh, H, y.cpu().numpy()), st["vcycles"]))
    assert abs(out[0][1] - out[1][1]) <= 1
    for sol, _ in out:
        R = cp.residual(H, sol, F, alpha, beta)
        assert max_abs(H, R) <= 1.05e-10 * max_abs(H, F)


@pytest.mark.parametrize("precision", [0, 1])
def test_3d_bulk_amr_restriction_matches_generic(bulk_sweep, precision):
    """The restriction of a single-patch fine level's residual into the coarse level by the
    bulk-copy kernel (base 64 x 32 x 16, a 64 x 32 x 16 fine box; both levels bulk-copy): one
    FP64 V-cycle and two mixed refinement steps bit for bit those of the z-chunked kernels with
    the generic restriction, and the FP64 V-cycle equal to the oracle's to 1e-10."""
    amr = _amr()
    n0 = (64, 32, 16)
    boxes = [[((0, 0, 0), (63, 31, 15))], [((32, 16, 8), (95, 47, 23))]]
    bc = [0, 1, 0, 0, 1, 0]
    alpha, beta = 1.0, -0.02
    H = OH(3, n0, boxes, bc=bc, hi=(1.0, 0.5, 0.25))
    gh = amr.Hierarchy(3, n0, boxes, h0=1.0 / 64)
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(107)
    F = _rand_field(H, rng)
    phi = _rand_field(H, rng)
    got = {}
    for on in (2, 0):
        bulk_sweep(on)
        dphi = _dev(to_packed(gh, H, phi))
        if precision == 0:
            op.vcycle(dphi, _dev(to_packed(gh, H, F)))
        else:
            op.solve(dphi, _dev(to_packed(gh, H, F)), allow_not_converged=True,
                     params=amr.default_params(rtol=1e-30, max_vcycles=2, precision=1, use_graph=0))
        got[on] = from_packed(gh, H, dphi.cpu().numpy())
    assert max_diff(H, got[2], got[0]) == 0.0
    if precision == 0:
        ref = mg.CompositeMG(H, alpha, beta).vcycle(phi, F)
        assert max_diff(H, got[2], ref) <= 1e-10 * max_abs(H, ref)
