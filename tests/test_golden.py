"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py from the
oracle alone): the oracle still reproduces them, and they carry the fourth-order
convergence Sec. 3 states for the discretisation."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402

GOLDEN = json.load(open(os.path.join(HERE, "golden", "ms2d.json")))


def test_golden_orders_are_fourth_order():
    """Sec. 3: fourth-order L1 / L2 convergence of the solution error (third-order truncation
    on the boundary layer leaves the max norm at >= 3.5)."""
    last = GOLDEN["observed_orders_l1_l2_linf"]["64->128"]
    assert last[0] > 3.8 and last[1] > 3.8 and last[2] > 3.5, last


def test_oracle_reproduces_golden_values():
    n = GOLDEN["n"]
    sol, err = make_golden.ms_solution(n)
    scale = float(np.max(np.abs(sol)))
    for (i, j), v in zip(GOLDEN["cells_ij"], GOLDEN["phi"]):
        assert abs(sol[i, j] - v) <= 1e-12 * scale
    for a, b in zip(err, GOLDEN["err_l1_l2_linf"]):
        assert abs(a - b) <= 1e-9 * b


AMR2D = json.load(open(os.path.join(HERE, "golden", "amr2d.json")))


def test_oracle_reproduces_amr2d_golden_values():
    """The two-level composite solves (coarse-fine ghosts of Sec. 5.2, refluxing, the
    solvability fix and mean-zero of Sec. 6.4) still give the stored values."""
    (_, n0, boxes), sols = make_golden.amr2d_solutions()
    assert list(n0) == AMR2D["n0"]
    assert json.loads(json.dumps(boxes)) == AMR2D["boxes"]
    for name, (H, phi) in sols.items():
        scale = AMR2D[name]["max_abs"]
        for l, i, j, v in AMR2D[name]["samples_level_index_value"]:
            assert H.levels[l].valid[i, j]
            assert abs(phi[l][i, j] - v) <= 1e-12 * scale, (name, l, i, j)


def test_oracle_reproduces_batch2d_golden_values():
    """The stored batch-workload solutions (four seeded problems) are reproduced by the
    oracle's direct solve, and each is the discrete solution: the oracle's residual of the
    stored problem vanishes to rounding at the sampled cells' level."""
    from oracle import composite as cp, solve as so
    from oracle.hierarchy import Hierarchy
    from paper_2506_02663_gb300 import workloads as wl
    gold = json.load(open(os.path.join(HERE, "golden", "batch2d.json")))
    probs = wl.batch2d_problems()
    for k, e in gold["problems"].items():
        pr = probs[int(k)]
        n = pr["n"]
        assert n == e["n"]
        H = Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]], bc=[0] * 4)
        F = cp.new_field(H)
        F[0][H.levels[0].covered] = pr["rhs"].ravel()
        phi, _, _ = so.solve_direct(H, F, pr["alpha"], pr["beta"])
        for s in e["samples_index_value"]:
            assert abs(phi[0][s[0], s[1]] - s[2]) <= 1e-12 * e["max_abs"]
        R = cp.residual(H, phi, F, pr["alpha"], pr["beta"])
        assert np.max(np.abs(R[0][H.levels[0].valid])) <= 1e-9 * np.max(np.abs(F[0][H.levels[0].valid]))
