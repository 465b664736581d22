"""GPU parity of the interface conditions of a subcycled level solve (Sec. 6.3 CIC-2/3,
Eq. timeInterp; Sec. 6.4, Eq. correctingFaceAvg) through the C ABI against the oracle
(oracle/cic.py): the CF ghosts at an intermediate time and their time derivative, and the
corrected normal face averages with their per-component shifts.  Tolerances: 1e-13 of the
largest input times the sum of |weights| (the value and the derivative rows of I^(4)); the
faces within 1e-13 of max|w|."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cic, composite as cp, solve as so  # noqa: E402
from oracle.hierarchy import Hierarchy as OH  # noqa: E402

from _gpu_helpers import from_packed, to_packed  # noqa: E402

pytestmark = pytest.mark.gpu

HIERS = {
    "three_level_multibox": (2, (24, 24), [[((0, 0), (23, 23))], [((8, 8), (23, 31)), ((24, 8), (39, 31))],
                                           [((24, 24), (47, 47))]]),
    "two_components": (2, (32, 32), [[((0, 0), (31, 31))],
                                     [((8, 8), (19, 19)), ((40, 36), (55, 51)), ((20, 8), (27, 15))]]),
    "boundary_box": (2, (16, 16), [[((0, 0), (15, 15))], [((0, 12), (11, 31))]]),
    "three_d_two_components": (3, (12, 12, 12), [[((0, 0, 0), (11, 11, 11))],
                                                 [((2, 2, 2), (7, 7, 7)), ((14, 14, 12), (21, 21, 19))]]),
    "three_d_box": (3, (16, 16, 16), [[((0, 0, 0), (15, 15, 15))], [((8, 8, 8), (23, 23, 23))]]),
}


def _amr():
    from paper_2506_02663_gb300 import amr
    return amr


def _hier(name):
    dim, n0, boxes = HIERS[name]
    H = OH(dim, n0, boxes, bc=[0] * (2 * dim))
    gh = _amr().Hierarchy(dim, n0, boxes, h0=1.0 / n0[0])
    return H, gh


def _rand(H, rng):
    U = so.Unknowns(H)
    return U.scatter(rng.standard_normal(U.n), fill_invalid=True)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _cf_slots(gh, H, l):
    """(flat index into the packed field, level-l array index) of every stored CF ghost of
    level l (ghost code 3)."""
    dim = H.D
    codes = gh.index_maps()["ghost_code"]
    lev = H.levels[l]
    out = []
    base = 0
    for p in gh.patches:
        n = [p["hi"][e] - p["lo"][e] + 1 for e in range(dim)]
        ext = [v + 4 for v in n]
        cnt = int(np.prod(ext))
        if p["level"] == l:
            c = codes[base:base + cnt].reshape(ext[::-1])
            for idx in np.argwhere(c == 3):
                a = idx[::-1]
                g = [p["lo"][e] - 2 + a[e] for e in range(dim)]
                flat = p["offset"] + int(a[0]) + int(a[1]) * p["sy"] + (int(a[2]) * p["sz"] if dim == 3 else 0)
                out.append((flat, tuple(g[e] - lev.origin[e] for e in range(dim))))
        base += cnt
    return out


@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("k,eta", [(0.25, 0.1), (0.01, 0.0), (0.5, 0.5), (1.0, -1.5), (0.125, 0.125)])
def test_interface_ghosts_match_oracle(name, k, eta):
    H, gh = _hier(name)
    amr = _amr()
    rng = np.random.default_rng(31)
    Ft = [_rand(H, rng) for _ in range(4)]
    dt = [_dev(to_packed(gh, H, F)) for F in Ft]
    sentinel = 7.25
    value = torch.full_like(dt[0], sentinel)
    rate = torch.full_like(dt[0], sentinel)
    amr.Operator(gh, 0.0, 1.0, [0] * (2 * H.D))  # device copy of the hierarchy
    M = cic.coarse_time_weights(k, eta)
    big = max(float(np.max(np.abs(F[l][H.levels[l].covered]))) for F in Ft for l in range(len(H.levels)))
    touched = np.zeros(dt[0].numel(), bool)
    for l in range(1, len(H.levels)):
        amr.cic_ghosts(gh, l, dt, k, eta, value, rate)
        torch.cuda.synchronize()
        cells, rv, rr = cic.interface_ghost_values(H, [F[l - 1] for F in Ft], l, k, eta)
        lev = H.levels[l]
        V = np.full(lev.shape, np.nan)
        R = np.full(lev.shape, np.nan)
        V[tuple(cells.T)] = rv
        R[tuple(cells.T)] = rr
        gv, gr = value.cpu().numpy(), rate.cpu().numpy()
        slots = _cf_slots(gh, H, l)
        assert slots
        for flat, a in slots:
            touched[flat] = True
            assert abs(gv[flat] - V[a]) <= 1e-13 * big * np.sum(np.abs(M[0])), (flat, a)
            assert abs(gr[flat] - R[a]) <= 1e-13 * big * np.sum(np.abs(M[1])), (flat, a)
    # nothing but the CF ghosts is written
    gv, gr = value.cpu().numpy(), rate.cpu().numpy()
    assert np.all(gv[~touched] == sentinel) and np.all(gr[~touched] == sentinel)


def test_interface_ghosts_at_a_coarse_time_are_amrcfi_of_that_time():
    """eta = 0 puts the unit weight on t_{-1} (the second coarse field): the ghosts then equal
    the AMRCFI values amr_fill_ghosts gives that field; the rate output is optional."""
    H, gh = _hier("three_level_multibox")
    amr = _amr()
    rng = np.random.default_rng(5)
    Ft = [_rand(H, rng) for _ in range(4)]
    dt = [_dev(to_packed(gh, H, F)) for F in Ft]
    op = amr.Operator(gh, 0.0, 1.0, [0] * 4)
    ref = dt[1].clone()
    op.fill_ghosts(ref)
    value = dt[1].clone()
    for l in range(1, len(H.levels)):
        amr.cic_ghosts(gh, l, dt, 0.3, 0.0, value, None)
    torch.cuda.synchronize()
    a, b = value.cpu().numpy(), ref.cpu().numpy()
    big = float(np.max(np.abs(b)))
    for l in range(1, len(H.levels)):
        for flat, _ in _cf_slots(gh, H, l):
            assert abs(a[flat] - b[flat]) <= 1e-14 * big


@pytest.mark.parametrize("name", list(HIERS))
def test_interface_face_averages_match_oracle(name):
    H, gh = _hier(name)
    amr = _amr()
    D = H.D
    rng = np.random.default_rng(17)
    k, eta = 0.2, 0.07
    W = [_rand(H, rng) for _ in range(D)]
    Wt = [[_rand(H, rng) for _ in range(4)] for _ in range(D)]  # coarse time levels per component
    op = amr.Operator(gh, 0.0, 1.0, [0] * (2 * D))
    wd = [_dev(to_packed(gh, H, W[d])) for d in range(D)]
    wtd = [[_dev(to_packed(gh, H, F)) for F in Wt[d]] for d in range(D)]
    for d in range(D):
        op.fill_ghosts(wd[d])
    for l in range(1, len(H.levels)):
        for d in range(D):
            amr.cic_ghosts(gh, l, wtd[d], k, eta, wd[d], None)
        info = amr.cic_faces(gh, l)
        nf, nc = len(info["face"]), info["ncomponents"]
        phys = rng.standard_normal(nc)
        faces = torch.zeros(nf, dtype=torch.float64, device="cuda")
        delta = torch.zeros(nc, dtype=torch.float64, device="cuda")
        amr.cic_face_averages(gh, l, wd, faces, phys=_dev(phys), delta=delta)
        torch.cuda.synchronize()
        # oracle: the level's arrays with CF ghosts from the time interpolation
        lev = H.levels[l]
        P = []
        for d in range(D):
            A = [a.copy() for a in W[d]]
            cp.average_down_all(H, A)
            cells, v, _ = cic.interface_ghost_values(H, [F[l - 1] for F in Wt[d]], l, k, eta)
            A[l][tuple(cells.T)] = v
            P.append(A[l])
        ref_faces = cic.interface_faces(H, l)
        raw = cic.interface_face_averages(H, P, l, ref_faces)
        comp = np.array([f[3] for f in ref_faces])
        corr, deltas = cic.correct_by_component(raw, comp, {c: float(phys[c]) for c in range(nc)})
        key = {(tuple(int(c[e] + lev.origin[e]) for e in range(D)), 2 * dd + (1 if s > 0 else 0)): i
               for i, (c, dd, s, _) in enumerate(ref_faces)}
        gf = faces.cpu().numpy()
        scale = max(float(np.max(np.abs(a[np.isfinite(a)]))) for a in P)
        assert nf == len(ref_faces)
        for i in range(nf):
            j = key[(tuple(int(v) for v in info["cell"][i]), int(info["face"][i]))]
            assert abs(gf[i] - corr[j]) <= 1e-13 * scale, (i, gf[i], corr[j])
        gd = delta.cpu().numpy()
        for c in range(nc):
            assert abs(gd[c] - deltas[c]) <= 1e-13 * scale
            sel = info["component"] == c
            assert abs(np.sum(gf[sel]) + phys[c]) <= 1e-12 * scale * max(1, int(sel.sum()))


def test_interface_face_averages_deterministic_and_level_without_interface():
    """Two calls give bitwise equal faces; a level covering the whole domain has no interface
    faces and its one component gets delta = 0."""
    amr = _amr()
    H, gh = _hier("two_components")
    rng = np.random.default_rng(3)
    W = [_dev(to_packed(gh, H, _rand(H, rng))) for _ in range(2)]
    op = amr.Operator(gh, 0.0, 1.0, [0] * 4)
    for w in W:
        op.fill_ghosts(w)
    nf = len(amr.cic_faces(gh, 1)["face"])
    a = torch.zeros(nf, dtype=torch.float64, device="cuda")
    b = torch.zeros(nf, dtype=torch.float64, device="cuda")
    amr.cic_face_averages(gh, 1, W, a)
    amr.cic_face_averages(gh, 1, W, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    dim, n0, boxes = 2, (16, 16), [[((0, 0), (15, 15))], [((0, 0), (31, 31))]]
    g2 = amr.Hierarchy(dim, n0, boxes)
    amr.Operator(g2, 0.0, 1.0, [0] * 4)
    H2 = OH(dim, n0, boxes, bc=[0] * 4)
    w2 = [_dev(to_packed(g2, H2, _rand(H2, rng))) for _ in range(2)]
    delta = torch.full((1,), 3.0, dtype=torch.float64, device="cuda")
    info = amr.cic_faces(g2, 1)
    assert len(info["face"]) == 0 and info["ncomponents"] == 1
    amr.cic_face_averages(g2, 1, w2, None, delta=delta)
    torch.cuda.synchronize()
    assert float(delta[0]) == 0.0


def test_full_size_3d_sampled():
    """The 3-D workload's geometry (256^3 base, 128^3 refined box) in the launch configuration
    the bench times: sampled CF ghosts against the oracle's AMRCFI of each coarse time and its
    time interpolation, sampled faces against Eq. (cell2face) on the filled fields plus the
    returned shift, and the per-component sum property on every face."""
    from oracle import stencil as st
    from oracle.cfi import cfi_values
    from paper_2506_02663_gb300 import workloads as wl
    amr = _amr()
    dim, n0, boxes = wl.hierarchy_boxes("bumps3d", 1)
    gh = amr.Hierarchy(dim, n0, boxes)
    op = amr.Operator(gh, 0.0, 1.0, [1] * 6)
    n = gh.nelems
    g = torch.Generator(device="cuda").manual_seed(11)
    coarse = [torch.randn(n, dtype=torch.float64, device="cuda", generator=g) for _ in range(4)]
    vel = [torch.randn(n, dtype=torch.float64, device="cuda", generator=g) for _ in range(3)]
    for x in coarse + vel:
        op.fill_ghosts(x)  # average-down: redundant data on covered coarse cells
    k, eta = 1.0 / 256.0, 0.3 / 256.0
    rate = torch.empty_like(vel[0])
    for d in range(3):
        amr.cic_ghosts(gh, 1, coarse, k, eta, vel[d], rate if d == 0 else None)
    info = amr.cic_faces(gh, 1)
    nf, nc = len(info["face"]), info["ncomponents"]
    assert nf == 6 * 128 * 128 and nc == 1
    phys = torch.tensor([0.37], dtype=torch.float64, device="cuda")
    faces = torch.empty(nf, dtype=torch.float64, device="cuda")
    delta = torch.empty(1, dtype=torch.float64, device="cuda")
    amr.cic_face_averages(gh, 1, vel, faces, phys=phys, delta=delta)
    torch.cuda.synchronize()
    p0, p1 = gh.patches[0], gh.patches[1]
    C = [gh.interior(x.cpu().numpy(), p0).transpose() for x in coarse]
    gv, gr = vel[0].cpu().numpy(), rate.cpu().numpy()
    M = cic.coarse_time_weights(k, eta)
    # sampled CF ghosts of level 1
    maps = gh.index_maps()
    n0pad = (256 + 4) ** 3
    sel = np.nonzero(maps["cfi_cell"] >= n0pad)[0]
    rng = np.random.default_rng(2)
    pick = rng.choice(sel, 300, replace=False)
    a = np.stack(np.unravel_index(maps["cfi_cell"][pick] - n0pad, (132, 132, 132)), axis=1)[:, ::-1]  # x, y, z
    gcell = a + np.asarray(p1["lo"]) - 2
    vals = [cfi_values(c, (0, 0, 0), (256, 256, 256), gcell, 2, 3)[0] for c in C]
    want_v = sum(M[0][i] * vals[i] for i in range(4))
    want_r = sum(M[1][i] * vals[i] for i in range(4))
    flat = p1["offset"] + a[:, 0] + a[:, 1] * p1["sy"] + a[:, 2] * p1["sz"]
    big = max(float(np.max(np.abs(c))) for c in C)
    assert np.max(np.abs(gv[flat] - want_v)) <= 1e-13 * big * np.sum(np.abs(M[0]))
    assert np.max(np.abs(gr[flat] - want_r)) <= 1e-13 * big * np.sum(np.abs(M[1]))
    # sampled faces against Eq. (cell2face) plus the shift; the sum property on all faces
    P = [gh._view(x.cpu().numpy(), p1)[:, :, :132].transpose() for x in vel]
    gf = faces.cpu().numpy()
    dl = float(delta[0])
    scale = max(float(np.max(np.abs(x))) for x in P)
    for i in rng.choice(nf, 300, replace=False):
        d, s = int(info["face"][i]) // 2, 1 if int(info["face"][i]) % 2 else -1
        cell = list(info["cell"][i] - (np.asarray(p1["lo"]) - 2))
        if s < 0:
            cell[d] -= 1
        raw = s * st.face_value(P[d], 3, d, tuple(cell))
        assert abs(gf[i] - (raw + dl)) <= 1e-13 * scale
    assert abs(np.sum(gf) + 0.37) <= 1e-12 * scale * nf


@pytest.mark.parametrize("name,comp", [("two_components", 1), ("three_d_two_components", 0),
                                       ("three_d_two_components", 1), ("three_d_box", 0)])
def test_level_problem_of_a_single_box_component(name, comp):
    """Def. GePUP-E-OneLevel on a single-box component: CF ghosts at t* from four coarse times
    (amr_cic_ghosts), their interface face averages as the box problem's Dirichlet data
    (amr_cic_interface_bc, against the oracle's), then the Helmholtz problem on the box solved
    by amr_solve against the oracle's direct solve with the oracle's data."""
    H, gh = _hier(name)
    amr = _amr()
    D = H.D
    rng = np.random.default_rng(41)
    k, eta = 0.2, 0.05
    X = _rand(H, rng)
    Xt = [_rand(H, rng) for _ in range(4)]
    op = amr.Operator(gh, 0.0, 1.0, [0] * (2 * D))
    xd = _dev(to_packed(gh, H, X))
    xtd = [_dev(to_packed(gh, H, F)) for F in Xt]
    op.fill_ghosts(xd)
    amr.cic_ghosts(gh, 1, xtd, k, eta, xd, None)
    lo, hi, flags = amr.cic_component_box(gh, 1, comp)
    olo, ohi, oflags = cic.component_box(H, 1, comp)
    assert (lo, hi, flags) == (tuple(olo), tuple(ohi), oflags)
    n = tuple(hi[e] - lo[e] + 1 for e in range(D))
    h = H.levels[1].h
    boxes_b = [[((0,) * D, tuple(v - 1 for v in n))]]
    gb = amr.Hierarchy(D, n, boxes_b, h0=h)
    Hb = OH(D, n, boxes_b, bc=[0] * (2 * D), hi=tuple(v * h for v in n))
    bc = torch.zeros(gb.bc_offsets[-1], dtype=torch.float64, device="cuda")
    amr.cic_interface_bc(gh, 1, comp, xd, bc)
    torch.cuda.synchronize()
    A = [a.copy() for a in X]
    cp.average_down_all(H, A)
    cells, v, _ = cic.interface_ghost_values(H, [F[0] for F in Xt], 1, k, eta)
    A[1][tuple(cells.T)] = v
    data = cic.box_interface_bc(H, A[1], 1, comp)
    scale = float(np.max(np.abs(A[1][np.isfinite(A[1])])))  # cells the oracle leaves undefined hold NaN
    assert np.max(np.abs(bc.cpu().numpy() - gb.pack_bc([data]))) <= 1e-13 * scale
    alpha, beta = 1.0, -0.01
    Fb = so.Unknowns(Hb).scatter(rng.standard_normal(so.Unknowns(Hb).n))
    ref, _, _ = so.solve_direct(Hb, Fb, alpha, beta, bc_data=[data])
    opb = amr.Operator(gb, alpha, beta, [0] * (2 * D))
    phi = torch.zeros(gb.nelems, dtype=torch.float64, device="cuda")
    st = opb.solve(phi, _dev(to_packed(gb, Hb, Fb)), bc=bc,
                   params=amr.default_params(rtol=1e-12, max_vcycles=60, precision=amr.FP64))
    assert st["status"] == 0
    got = from_packed(gb, Hb, phi.cpu().numpy())
    lev = Hb.levels[0]
    assert np.max(np.abs(got[0][lev.valid] - ref[0][lev.valid])) <= 1e-10 * np.max(np.abs(ref[0][lev.valid]))
