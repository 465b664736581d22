"""Batched solves (uneven single-level Helmholtz problems, the batch workload's shape at
reduced sizes): concurrent captured solves give the same answers as one-by-one solves and
as the oracle's direct solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import composite as cp, solve as so  # noqa: E402
from oracle.hierarchy import Hierarchy as OH  # noqa: E402

from _gpu_helpers import from_packed, max_abs, max_diff, to_packed  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_solve_matches_individual_and_oracle(precision):
    from paper_2506_02663_gb300 import amr, workloads as wl
    probs = wl.batch2d_problems(nprob=10, sizes=(16, 24, 32, 48, 64))
    hs, ops, fs, Hs = [], [], [], []
    for pr in probs:
        n = pr["n"]
        box = [[((0, 0), (n - 1, n - 1))]]
        gh = amr.Hierarchy(2, (n, n), box)
        hs.append(gh)
        ops.append(amr.Operator(gh, pr["alpha"], pr["beta"] * 256.0, [0, 0, 0, 0]))
        fs.append(torch.from_numpy(gh.pack([[pr["rhs"]]])).cuda())
        Hs.append(OH(2, (n, n), box, bc=[0, 0, 0, 0]))
    p = amr.default_params(rtol=1e-12, max_vcycles=100, precision=precision)
    phis = [torch.zeros_like(f) for f in fs]
    stats, status = amr.batch_solve(ops, phis, fs, params=p)
    assert all(s == 0 for s in status)
    for k, (op, f) in enumerate(zip(ops, fs)):
        x = torch.zeros_like(f)
        st = op.solve(x, f, params=amr.default_params(rtol=1e-12, max_vcycles=100, precision=precision, use_graph=1))
        assert st["vcycles"] == stats[k]["vcycles"]
        assert torch.max(torch.abs(x - phis[k])).item() <= 1e-13 * torch.max(torch.abs(x)).item()
    for k in (0, 3, 9):
        H = Hs[k]
        F = cp.new_field(H)
        F[0][H.levels[0].covered] = probs[k]["rhs"].ravel()
        ref, _, _ = so.solve_direct(H, F, probs[k]["alpha"], probs[k]["beta"] * 256.0)
        got = from_packed(hs[k], H, phis[k].cpu().numpy())
        assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref)
