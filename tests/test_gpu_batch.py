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


def _batch(amr, sizes, nprob, beta_scale, shared=False):
    from paper_2506_02663_gb300 import workloads as wl
    probs = wl.batch2d_problems(nprob=nprob, sizes=sizes)
    hs, ops, fs = [], [], []
    for k, pr in enumerate(probs):
        n = pr["n"]
        box = [[((0, 0), (n - 1, n - 1))]]
        if shared and k > 0 and probs[k - 1]["n"] == n:
            gh = hs[-1]
        else:
            gh = amr.Hierarchy(2, (n, n), box)
        hs.append(gh)
        ops.append(amr.Operator(gh, pr["alpha"], pr["beta"] * beta_scale, [0, 0, 0, 0]))
        fs.append(torch.from_numpy(gh.pack([[pr["rhs"]]])).cuda())
    return probs, hs, ops, fs


@pytest.mark.parametrize("sizes,nprob,shared", [((48, 64, 96, 128, 192, 256), 14, False), ((64, 96), 6, True)])
def test_worklist_batch_matches_individual_and_oracle(sizes, nprob, shared):
    """Batches of single-level problems whose level-0 pyramids end in the square one-block
    coarse V-cycle run as one captured graph with one launch per phase over a work list
    (problems sharing a hierarchy included): every problem takes the V-cycles of its own
    captured solve and reaches the same solution, and small ones match the oracle's direct
    solve; a second call reuses the graph."""
    from paper_2506_02663_gb300 import amr
    probs, hs, ops, fs = _batch(amr, sizes, nprob, 256.0, shared)
    p = amr.default_params(rtol=1e-12, max_vcycles=100, precision=amr.MIXED)
    phis = [torch.zeros_like(f) for f in fs]
    for rep in range(2):
        for x in phis:
            x.fill_(1.0)  # zero_initial clears the guess
        stats, status = amr.batch_solve(ops, phis, fs, params=p)
        assert all(s == 0 for s in status), status
    for k, (op, f) in enumerate(zip(ops, fs)):
        x = torch.zeros_like(f)
        st = op.solve(x, f, params=amr.default_params(rtol=1e-12, max_vcycles=100, precision=amr.MIXED, use_graph=1))
        assert st["vcycles"] == stats[k]["vcycles"], (k, st["vcycles"], stats[k]["vcycles"])
        assert torch.max(torch.abs(x - phis[k])).item() <= 1e-13 * torch.max(torch.abs(x)).item()
    for k in range(nprob):
        if probs[k]["n"] > 96:
            continue
        n = probs[k]["n"]
        H = OH(2, (n, n), [[((0, 0), (n - 1, n - 1))]], bc=[0, 0, 0, 0])
        F = cp.new_field(H)
        F[0][H.levels[0].covered] = probs[k]["rhs"].ravel()
        ref, _, _ = so.solve_direct(H, F, probs[k]["alpha"], probs[k]["beta"] * 256.0)
        got = from_packed(hs[k], H, phis[k].cpu().numpy())
        assert max_diff(H, got, ref) <= 1e-10 * max_abs(H, ref)
        break


def test_worklist_batch_large_tiles():
    """A batch mixing 32^2-tile grids (1024^2) with small ones: the work-list graph splits each
    leg's launch by tile edge and still matches the problems' own captured solves."""
    from paper_2506_02663_gb300 import amr
    probs, hs, ops, fs = _batch(amr, (64, 1024), 4, 1.0)
    p = amr.default_params(rtol=1e-10, max_vcycles=100, precision=amr.MIXED)
    phis = [torch.zeros_like(f) for f in fs]
    stats, status = amr.batch_solve(ops, phis, fs, params=p)
    assert all(s == 0 for s in status), status
    for k, (op, f) in enumerate(zip(ops, fs)):
        x = torch.zeros_like(f)
        st = op.solve(x, f, params=amr.default_params(rtol=1e-10, max_vcycles=100, precision=amr.MIXED, use_graph=1))
        assert st["vcycles"] == stats[k]["vcycles"]
        assert torch.max(torch.abs(x - phis[k])).item() <= 1e-13 * torch.max(torch.abs(x)).item()
