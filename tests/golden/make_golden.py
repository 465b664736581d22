"""Writes the stored expected values under tests/golden/ from the FP64 oracle alone (no
GPU, no library): ``python tests/golden/make_golden.py``.

ms2d.json: the 64^2 manufactured-solution Poisson problem (phi = sin 2 pi x sin 3 pi y +
x^2 y on the unit square, Dirichlet face averages, right-hand side = cell averages of the
Laplacian, the paper's Sec. 3 discretisation): the discrete solution at 32 seeded cells,
its error norms against the exact cell averages, and the errors and observed orders for
n = 16, 32, 64, 128 (the fourth-order claim of Sec. 3).

amr2d.json: the bench's two-level workload at 1/8 size (32^2 base, ratio-2 box over
[0.25, 0.75]^2, Gaussian-bump right-hand side): the composite discrete solution of the
pure-Neumann PPE after the solvability fix and mean-zero (Sec. 6.4), and of the Helmholtz
system alpha = 1, beta = -0.25 * 1e-3 / 256 with homogeneous Dirichlet data (Eq. comp. of
Sec. 5 with AMRCFI ghosts and refluxing), at 24 seeded valid cells of each level.

amr3d.json: the 3-D workload at 1/8 size (32^3 base, ratio-2 box over [0.375, 0.625]^3,
i.e. 16^3 fine cells, Gaussian-bump right-hand sides): the composite discrete solution of
the pure-Neumann PPE (right-hand side component 0) after the solvability fix and mean-zero,
and of the Helmholtz system of velocity component 1 (alpha = 1, beta = -0.25 * 1e-3 / 256,
homogeneous Dirichlet), at 24 seeded valid cells of each level.  Each direct solve takes a
few minutes: ``python tests/golden/make_golden.py amr3d`` writes this file alone.

batch2d.json: four problems of the batch workload (``python tests/golden/make_golden.py
batch2d``), directly solved, 24 seeded cells each."""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import composite as cp, solve as so  # noqa: E402
from oracle.hierarchy import Hierarchy  # noqa: E402
from paper_2506_02663_gb300 import workloads as wl  # noqa: E402  (seeded inputs only)


def ms_solution(n):
    rhs, bc, exact = wl.ms2d(n)
    H = Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]], bc=[0] * 4)
    f = cp.new_field(H)
    f[0][H.levels[0].covered] = rhs.ravel()
    phi, _, _ = so.solve_direct(H, f, 0.0, 1.0, [bc])
    sol = phi[0][H.levels[0].covered].reshape(n, n)
    e = sol - exact
    h = 1.0 / n
    return sol, (float(np.sum(np.abs(e)) * h * h), float(math.sqrt(np.sum(e * e) * h * h)), float(np.max(np.abs(e))))


def main():
    n = 64
    sol, err = ms_solution(n)
    g = np.random.default_rng(20250603 + 1)
    cells = g.integers(0, n, size=(32, 2))
    errs = {m: ms_solution(m)[1] for m in (16, 32, 64, 128)}
    ms = sorted(errs)
    orders = {f"{ms[i]}->{ms[i + 1]}": [math.log2(errs[ms[i]][k] / errs[ms[i + 1]][k]) for k in range(3)]
              for i in range(len(ms) - 1)}
    out = {
        "source": "oracle.solve.solve_direct on workloads.ms2d (paper Sec. 3 discretisation, Dirichlet "
                  "Eq. velBCHomoDiri5th); written by tests/golden/make_golden.py",
        "n": n,
        "cells_ij": cells.tolist(),  # (i, j): x index, y index of the n x n interior array [i, j]
        "phi": [float(sol[i, j]) for i, j in cells],
        "err_l1_l2_linf": list(err),
        "errors_by_n": {str(m): list(v) for m, v in errs.items()},
        "observed_orders_l1_l2_linf": orders,
    }
    with open(os.path.join(HERE, "ms2d.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote ms2d.json")
    amr2d()


def amr2d_solutions():
    dim, n0, boxes, rhs = wl.bumps2d_rhs(scale=8)
    out = {}
    for name, bc, alpha, beta in (("ppe", [1] * 4, 0.0, 1.0), ("helmholtz", [0] * 4, 1.0, wl.HELMHOLTZ_BETA)):
        H = Hierarchy(dim, n0, boxes, bc=bc)
        F = cp.new_field(H)
        for l, lev in enumerate(H.levels):
            for k, (lo, hi) in enumerate(lev.boxes):
                F[l][lev.box_slice(lo, hi)] = rhs[l][k]
        if so.is_pure_neumann(H, alpha):
            F, _ = so.solvability_fix(H, F)
        phi, _, _ = so.solve_direct(H, F, alpha, beta)
        if so.is_pure_neumann(H, alpha):
            phi, _ = so.mean_zero(H, phi)
        out[name] = (H, phi)
    return (dim, n0, boxes), out


def amr2d():
    (dim, n0, boxes), sols = amr2d_solutions()
    g = np.random.default_rng(20250603 + 2)
    res = {"source": "oracle.solve.solve_direct (+ solvability_fix, mean_zero) on workloads.bumps2d_rhs(scale=8); "
                     "written by tests/golden/make_golden.py",
           "n0": list(n0), "boxes": boxes}
    _write_samples(res, sols, g, "amr2d.json")


def amr3d_solutions():
    out = {}
    for name, comp, bc, alpha, beta in (("ppe", 0, [1] * 6, 0.0, 1.0),
                                        ("helmholtz", 1, [0] * 6, 1.0, wl.HELMHOLTZ_BETA)):
        dim, n0, boxes, rhs = wl.bumps3d_rhs(scale=8, component=comp)
        H = Hierarchy(dim, n0, boxes, bc=bc)
        F = cp.new_field(H)
        for l, lev in enumerate(H.levels):
            for k, (lo, hi) in enumerate(lev.boxes):
                F[l][lev.box_slice(lo, hi)] = rhs[l][k]
        if so.is_pure_neumann(H, alpha):
            F, _ = so.solvability_fix(H, F)
        phi, _, _ = so.solve_direct(H, F, alpha, beta)
        if so.is_pure_neumann(H, alpha):
            phi, _ = so.mean_zero(H, phi)
        out[name] = (H, phi)
    return (dim, n0, boxes), out


def amr3d():
    (dim, n0, boxes), sols = amr3d_solutions()
    g = np.random.default_rng(20250603 + 5)
    res = {"source": "oracle.solve.solve_direct (+ solvability_fix, mean_zero) on workloads.bumps3d_rhs(scale=8, "
                     "component=0 for the PPE, 1 for the Helmholtz system); written by tests/golden/make_golden.py",
           "n0": list(n0), "boxes": boxes}
    _write_samples(res, sols, g, "amr3d.json")


def batch2d():
    """batch2d.json: four problems of the batch workload (the first three of size 64^2 and the
    first of size 96^2 in its seeded order), each solved directly: 24 seeded cells and
    max|phi| per problem."""
    probs = wl.batch2d_problems()
    picks = [k for k, pr in enumerate(probs) if pr["n"] == 64][:3] + [k for k, pr in enumerate(probs) if pr["n"] == 96][:1]
    g = np.random.default_rng(20250603 + 3)
    res = {"source": "oracle.solve.solve_direct on workloads.batch2d_problems() entries (alpha, beta as given, "
                     "homogeneous Dirichlet); written by tests/golden/make_golden.py", "problems": {}}
    for k in picks:
        pr = probs[k]
        n = pr["n"]
        H = Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]], bc=[0] * 4)
        F = cp.new_field(H)
        F[0][H.levels[0].covered] = pr["rhs"].ravel()
        phi, _, _ = so.solve_direct(H, F, pr["alpha"], pr["beta"])
        lev = H.levels[0]
        idx = np.argwhere(lev.valid)
        pick = idx[g.choice(len(idx), size=24, replace=False)]
        res["problems"][str(k)] = {
            "n": n, "samples_index_value": [[int(v) for v in c] + [float(phi[0][tuple(c)])] for c in pick],
            "max_abs": float(np.max(np.abs(phi[0][lev.valid])))}
    with open(os.path.join(HERE, "batch2d.json"), "w") as fh:
        json.dump(res, fh, indent=1)
    print("wrote batch2d.json")


def _write_samples(res, sols, g, fname):
    for name, (H, phi) in sols.items():
        samples = []
        for l, lev in enumerate(H.levels):
            idx = np.argwhere(lev.valid)
            pick = idx[g.choice(len(idx), size=24, replace=False)]
            samples += [[l] + [int(v) for v in c] + [float(phi[l][tuple(c)])] for c in pick]
        res[name] = {"samples_level_index_value": samples,
                     "max_abs": float(max(np.max(np.abs(phi[l][lev.valid])) for l, lev in enumerate(H.levels)))}
    with open(os.path.join(HERE, fname), "w") as fh:
        json.dump(res, fh, indent=1)
    print("wrote", fname)


if __name__ == "__main__":
    if sys.argv[1:] == ["amr3d"]:
        amr3d()
    elif sys.argv[1:] == ["batch2d"]:
        batch2d()
    else:
        main()
        batch2d()
        amr3d()
