"""GPU: mixed precision with several FP32 correction cycles per FP64 residual
(cycles_per_refinement).  In exact arithmetic c cycles of one refinement step (each later
cycle on the FP32 composite residual of the correction so far) give the iterate of c steps
of one cycle, so the solve needs the same number of V-cycles, rounded up to a multiple of c,
and reaches the same residual bound; the oracle's composite residual checks the solution."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import composite as cp, solve as so  # noqa: E402
from oracle.hierarchy import Hierarchy as OH  # noqa: E402

from _gpu_helpers import from_packed, max_abs, max_diff, to_packed  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    # 3-D two-level, both levels bulk-copy and fixed-point eligible
    "3d": (3, (64, 32, 16), [[((0, 0, 0), (63, 31, 15))], [((32, 16, 8), (95, 47, 23))]]),
    # 2-D three-level with a two-box level
    "2d": (2, (32, 32), [[((0, 0), (31, 31))], [((8, 8), (23, 39)), ((24, 8), (39, 39))], [((24, 24), (55, 55))]]),
}


def _amr():
    from paper_2506_02663_gb300 import amr
    return amr


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("bcw,ab", [(0, (1.0, -0.01)), (1, (0.0, 1.0))])
@pytest.mark.parametrize("graph", [1, 0])
def test_cycles_per_refinement(case, bcw, ab, graph):
    amr = _amr()
    dim, n0, boxes = CASES[case]
    bc = [bcw] * (2 * dim)
    alpha, beta = ab
    hi = tuple(n0[d] / n0[0] for d in range(dim))
    H = OH(dim, n0, boxes, bc=bc, hi=hi)
    gh = amr.Hierarchy(dim, n0, boxes, h0=1.0 / n0[0])
    op = amr.Operator(gh, alpha, beta, bc)
    rng = np.random.default_rng(101)
    U = so.Unknowns(H)
    F = U.scatter(rng.standard_normal(U.n), fill_invalid=True)
    if bcw == 1:
        F, _ = so.solvability_fix(H, F)
    df = torch.from_numpy(np.ascontiguousarray(to_packed(gh, H, F))).cuda()
    out = {}
    for c in (1, 2, 3):
        x = torch.zeros_like(df)
        st = op.solve(x, df, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=1, use_graph=graph,
                                                         cycles_per_refinement=c))
        out[c] = (from_packed(gh, H, x.cpu().numpy()), st["vcycles"])
    n1 = out[1][1]
    for c in (2, 3):
        sol, n = out[c]
        assert n % c == 0 and abs(n - -(-n1 // c) * c) <= c, (c, n, n1)
        R = cp.residual(H, sol, F, alpha, beta)
        assert max_abs(H, R) <= 1.05e-10 * max_abs(H, F), c
        assert max_diff(H, sol, out[1][0]) <= 1e-8 * max_abs(H, out[1][0]), c


def test_cycles_per_refinement_bounds():
    amr = _amr()
    gh = amr.Hierarchy(2, (16, 16), [[((0, 0), (15, 15))]])
    op = amr.Operator(gh, 1.0, -0.01, [0] * 4)
    f = torch.ones(gh.nelems, dtype=torch.float64, device="cuda")
    for c in (0, 5):
        with pytest.raises(Exception):
            op.solve(torch.zeros_like(f), f, params=amr.default_params(precision=1, cycles_per_refinement=c))
