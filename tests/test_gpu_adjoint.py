"""Adjoint (transposed) operator and solve on the GPU against the oracle's assembled
composite matrix: (A^comp)^T y elementwise, the dot-product identity through the ABI alone,
and A^{-T} g against the oracle's direct transposed solve.  Finite-difference check of the
autograd gradient of a quadratic loss of a Helmholtz solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import solve as so  # noqa: E402

from _gpu_helpers import from_packed, max_abs, max_diff, to_packed  # noqa: E402
from test_gpu_parity import BCS, HIERS, _amr, _dev, _hier, _rand_field  # noqa: E402

pytestmark = pytest.mark.gpu


def _valid_vec(H, F):
    U = so.Unknowns(H)
    return U, U.gather(F)


@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("ab", [(1.0, -0.01), (0.0, 1.0)])
def test_apply_transpose_matches_assembled_matrix(name, which, ab):
    amr = _amr()
    dim = HIERS[name][0]
    bc = BCS[dim][which]
    H, gh = _hier(name, bc)
    alpha, beta = ab
    A, U = so.helmholtz_matrix(H, alpha, beta)
    rng = np.random.default_rng(41)
    Y = _rand_field(H, rng)
    y = U.gather(Y)
    ref = A.T @ y
    op = amr.Operator(gh, alpha, beta, bc)
    out = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
    op.apply_transpose(_dev(to_packed(gh, H, Y, fill=np.nan)), out)
    got = U.gather(from_packed(gh, H, out.cpu().numpy()))
    scale = abs(A).max() * np.max(np.abs(y)) * 8
    assert np.max(np.abs(got - ref)) <= 1e-13 * scale


@pytest.mark.parametrize("name", list(HIERS))
def test_dot_product_identity_through_the_abi(name):
    """<A x, y> = <x, A^T y> over the valid cells, both sides computed by the library."""
    amr = _amr()
    dim = HIERS[name][0]
    bc = BCS[dim][0]
    H, gh = _hier(name, bc)
    U = so.Unknowns(H)
    rng = np.random.default_rng(43)
    X, Y = _rand_field(H, rng), _rand_field(H, rng)
    op = amr.Operator(gh, 1.0, -0.02, bc)
    ax = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
    aty = torch.zeros_like(ax)
    op.apply(_dev(to_packed(gh, H, X)), ax)
    op.apply_transpose(_dev(to_packed(gh, H, Y)), aty)
    x, y = U.gather(X), U.gather(Y)
    lhs = float(np.dot(U.gather(from_packed(gh, H, ax.cpu().numpy())), y))
    rhs = float(np.dot(x, U.gather(from_packed(gh, H, aty.cpu().numpy()))))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs) + 1.0)


@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_transpose_matches_direct(name, precision):
    amr = _amr()
    dim = HIERS[name][0]
    bc = BCS[dim][0]
    H, gh = _hier(name, bc)
    rng = np.random.default_rng(47)
    # zero on invalid cells: the ABI hands invalid-cell weight to the children first
    # (transposed average-down), which the oracle's plain A^{-T} g does not do
    G = _rand_field(H, rng, redundant=False)
    for alpha, beta in ((1.0, -0.01), (0.0, 1.0)):
        ref, A, U = so.solve_transpose_direct(H, G, alpha, beta)
        op = amr.Operator(gh, alpha, beta, bc)
        lam = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
        st = op.solve_transpose(lam, _dev(to_packed(gh, H, G)),
                                params=amr.default_params(rtol=1e-12, max_vcycles=200, precision=precision))
        got = from_packed(gh, H, lam.cpu().numpy())
        assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref), (alpha, st)


def _valid_mask_tensor(gh, H):
    m = [lev.valid.astype(np.float64) for lev in H.levels]
    return _dev(to_packed(gh, H, m, fill=0.0))


def test_solve_transpose_hands_invalid_weight_to_children():
    """g with weight on invalid cells: the ABI solves A^T lambda = E^T g (E = the map from
    unknowns to composite data whose invalid cells are averages), checked against the oracle
    with E^T applied by hand."""
    amr = _amr()
    from oracle import composite as cp
    H, gh = _hier("three_level_multibox", [0, 0, 0, 0])
    rng = np.random.default_rng(59)
    G = _rand_field(H, rng)  # invalid cells hold the average of their children
    Et = [a.copy() for a in G]
    for l in range(H.lmax):
        lev, fine = H.levels[l], H.levels[l + 1]
        for lo, hi in fine.boxes:
            fs = fine.box_slice(lo, hi)
            par = np.repeat(np.repeat(Et[l][lev.box_slice(tuple(v // 2 for v in lo), tuple(v // 2 for v in hi))], 2, 0), 2, 1)
            Et[l + 1][fs] = Et[l + 1][fs] + par / 4.0
    ref, _, _ = so.solve_transpose_direct(H, Et, 1.0, -0.01)
    op = amr.Operator(gh, 1.0, -0.01, [0, 0, 0, 0])
    lam = torch.zeros(gh.nelems, dtype=torch.float64, device="cuda")
    op.solve_transpose(lam, _dev(to_packed(gh, H, G)), params=amr.default_params(rtol=1e-12, max_vcycles=200))
    got = from_packed(gh, H, lam.cpu().numpy())
    assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref)


@pytest.mark.parametrize("name", ["two_level_ragged", "three_level_multibox", "three_d"])
def test_autograd_gradient_vs_finite_differences_and_dense(name):
    """J(f) = 1/2 sum_valid phi^2 with A phi = f (Helmholtz).  J is quadratic in f, so central
    differences are exact up to rounding and the solve tolerance: the adjoint gradient must
    agree to 1e-6 on random directions, and with the dense reference A^{-T} phi elementwise."""
    amr = _amr()
    from paper_2506_02663_gb300.autograd import AmrSolve
    dim = HIERS[name][0]
    bc = BCS[dim][0]
    H, gh = _hier(name, bc)
    alpha, beta = 1.0, -0.01
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(53)
    F = _rand_field(H, rng)
    f = _dev(to_packed(gh, H, F)).requires_grad_(True)
    mask = _valid_mask_tensor(gh, H)
    p = amr.default_params(rtol=1e-13, max_vcycles=200, use_graph=1)

    def J(ff):
        phi = AmrSolve.apply(ff, op, p)
        return 0.5 * torch.sum(mask * phi * phi)

    loss = J(f)
    loss.backward()
    g = f.grad.detach()
    # dense reference gradient: A^{-T} phi on the valid cells
    phi, A, U = so.solve_direct(H, F, alpha, beta)
    lam, _, _ = so.solve_transpose_direct(H, phi, alpha, beta, A=A, U=U)
    got = from_packed(gh, H, g.cpu().numpy())
    assert max_diff(H, got, lam) <= 1e-9 * max_abs(H, lam)
    eps = 1e-3
    for _ in range(4):
        v = _dev(to_packed(gh, H, _rand_field(H, rng)))
        with torch.no_grad():
            fd = (J(f.detach() + eps * v) - J(f.detach() - eps * v)) / (2 * eps)
        ad = torch.sum(g * v * mask)
        assert abs(float(fd) - float(ad)) <= 1e-6 * abs(float(fd)), (float(fd), float(ad))
