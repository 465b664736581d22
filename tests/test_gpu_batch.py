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


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_solve_host_matches_device_batch(precision):
    """amr_batch_solve_host (host buffers, copies inside the call) gives the device batch's
    solutions and statistics, on both batch paths: single-level 2-D problems (work list) and
    two-level 3-D problems (concurrent captured solves)."""
    from paper_2506_02663_gb300 import amr, workloads as wl
    p = amr.default_params(rtol=1e-12, max_vcycles=100, precision=precision)
    cases = []
    probs = wl.batch2d_problems(nprob=4, sizes=(64, 96))
    for pr in probs:
        n = pr["n"]
        gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
        cases.append((gh, amr.Operator(gh, pr["alpha"], pr["beta"] * 256.0, [0, 0, 0, 0]), gh.pack([[pr["rhs"]]])))
    for comp in (1, 2):
        dim, n0, boxes, rhs = wl.bumps3d_rhs(scale=8, component=comp)
        gh = amr.Hierarchy(dim, n0, boxes)
        cases.append((gh, amr.Operator(gh, 1.0, -0.01, [0] * 6), gh.pack(rhs)))
    for group in (cases[:4], cases[4:]):
        ops = [c[1] for c in group]
        fs = [torch.from_numpy(c[2]).cuda() for c in group]
        phis = [torch.zeros_like(f) for f in fs]
        st_d, status_d = amr.batch_solve(ops, phis, fs, params=p)
        fh = [torch.from_numpy(c[2]).pin_memory().numpy() for c in group]
        ph = [np.zeros_like(c[2]) for c in group]  # pageable
        for _ in range(2):  # the second call reuses the operators' device buffers
            st_h, status_h = amr.batch_solve_host(ops, ph, fh, params=p)
            assert status_h == status_d and all(s == 0 for s in status_h)
            for k in range(len(group)):
                assert st_h[k]["vcycles"] == st_d[k]["vcycles"]
                ref = phis[k].cpu().numpy()
                assert np.max(np.abs(ph[k] - ref)) <= 1e-13 * np.max(np.abs(ref))
    with pytest.raises(amr.AmrError) as ei:
        amr.batch_solve_host([cases[0][1], cases[0][1]], [np.zeros_like(cases[0][2])] * 2, [cases[0][2]] * 2, params=p)
    assert ei.value.status == amr.AMR_ERR_INVALID_ARG
    for gh, op, _ in cases:
        op.close()
        gh.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scale,bulk", [(8, 1), (4, 2)])
def test_stacked_batch_matches_separate_solves(precision, scale, bulk):
    """Three Helmholtz problems on hierarchies of one 3-D geometry (the 3-D workload at 1/8 and
    1/4 size: 32^3 or 64^3 base with a ratio-2 box; three independent bump right-hand sides)
    and one operator: with stacked batches on, amr_batch_solve stacks them (one replica of
    every patch per problem, one launch per phase).  Each problem's V-cycle count and solution equal those of its own
    solve (the per-cell arithmetic and the per-replica norms are the same), and equal those
    of the unstacked batch; on the 64^3 base the bulk-copy kernel runs on the replicas."""
    from paper_2506_02663_gb300 import amr, workloads as wl
    amr.set_bulk_sweep(bulk)
    try:
        p = amr.default_params(rtol=1e-10, max_vcycles=100, precision=precision, use_graph=1)
        ghs, ops, fs = [], [], []
        for comp in (1, 2, 3):
            dim, n0, boxes, rhs = wl.bumps3d_rhs(scale=scale, component=comp)
            gh = amr.Hierarchy(dim, n0, boxes)
            ghs.append(gh)
            ops.append(amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA * 64, [0] * 6))
            fs.append(torch.from_numpy(gh.pack(rhs)).cuda())
        ref = []
        for op, f in zip(ops, fs):
            x = torch.zeros_like(f)
            st = op.solve(x, f, params=p)
            ref.append((x, st["vcycles"]))
        results = {}
        for on in (1, 0):
            amr.set_stacked_batches(on)
            phis = [torch.full_like(f, 7.0) for f in fs]  # zero_initial: overwritten
            for _ in range(2):  # the second call reuses the stacked hierarchy and graph
                stats, status = amr.batch_solve(ops, phis, fs, params=p)
                assert all(s == 0 for s in status)
            results[on] = (phis, stats)
        for on in (1, 0):
            phis, stats = results[on]
            for k in range(3):
                assert stats[k]["vcycles"] == ref[k][1], (on, k, stats[k]["vcycles"], ref[k][1])
                scale_k = torch.max(torch.abs(ref[k][0])).item()
                assert torch.max(torch.abs(phis[k] - ref[k][0])).item() <= 1e-13 * scale_k, (on, k)
                assert stats[k]["final_res"] <= 1e-10 * stats[k]["rhs_norm"]
        amr.check_kernel_flags()
    finally:
        amr.set_stacked_batches(0)
        amr.set_bulk_sweep(1)
    for op in ops:
        op.close()
    for gh in ghs:
        gh.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_stored_oracle_solutions(precision):
    """The four stored problems of the batch workload (tests/golden/batch2d.json: the oracle's
    direct solutions at seeded cells), solved together by amr_batch_solve to 1e-12: every
    sample within 1e-10 of max|phi|."""
    import json
    import os
    from paper_2506_02663_gb300 import amr, workloads as wl
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch2d.json")))
    probs = wl.batch2d_problems()
    keys = sorted(gold["problems"], key=int)
    hs, ops, fs = [], [], []
    for k in keys:
        pr = probs[int(k)]
        n = pr["n"]
        gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
        hs.append(gh)
        ops.append(amr.Operator(gh, pr["alpha"], pr["beta"], [0, 0, 0, 0]))
        fs.append(torch.from_numpy(gh.pack([[pr["rhs"]]])).cuda())
    phis = [torch.zeros_like(f) for f in fs]
    stats, status = amr.batch_solve(ops, phis, fs, params=amr.default_params(rtol=1e-12, max_vcycles=100,
                                                                              precision=precision))
    assert all(s == 0 for s in status), status
    for k, gh, x in zip(keys, hs, phis):
        e = gold["problems"][k]
        per = gh.unpack(x.cpu().numpy())[0][0]
        for i, j, v in e["samples_index_value"]:
            assert abs(float(per[i - 2, j - 2]) - v) <= 1e-10 * e["max_abs"], (k, i, j)


def test_stacked_batch_host_buffers():
    """amr_batch_solve_host on the stacked path (three Helmholtz problems of one 3-D geometry,
    stacked batches on): the copies around the stacked solve give the device batch's
    solutions and V-cycle counts."""
    from paper_2506_02663_gb300 import amr, workloads as wl
    p = amr.default_params(rtol=1e-10, max_vcycles=100, precision=1)
    ghs, ops, fs = [], [], []
    for comp in (1, 2, 3):
        dim, n0, boxes, rhs = wl.bumps3d_rhs(scale=8, component=comp)
        gh = amr.Hierarchy(dim, n0, boxes)
        ghs.append(gh)
        ops.append(amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA * 64, [0] * 6))
        fs.append(gh.pack(rhs))
    amr.set_stacked_batches(1)
    try:
        dphis = [torch.zeros(len(f), dtype=torch.float64, device="cuda") for f in fs]
        st_d, status_d = amr.batch_solve(ops, dphis, [torch.from_numpy(f).cuda() for f in fs], params=p)
        ph = [np.zeros_like(f) for f in fs]
        st_h, status_h = amr.batch_solve_host(ops, ph, fs, params=p)
        assert status_h == status_d and all(s == 0 for s in status_h)
        for k in range(3):
            assert st_h[k]["vcycles"] == st_d[k]["vcycles"]
            ref = dphis[k].cpu().numpy()
            assert np.max(np.abs(ph[k] - ref)) <= 1e-13 * np.max(np.abs(ref))
    finally:
        amr.set_stacked_batches(0)
    for op in ops:
        op.close()
    for gh in ghs:
        gh.close()
