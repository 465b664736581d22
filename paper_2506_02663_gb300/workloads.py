"""Seeded synthetic inputs for the five workloads (shared by tests, smoke and bench).

This module holds no arithmetic of the method: it only draws random numbers, evaluates
analytic functions and averages them over cells and faces by quadrature or in closed form.
Both the CUDA path's tests and the oracle's tests take their inputs from here.

Workloads (the paper evaluates its solver only inside full flow simulations, so these are
synthetic stand-ins with the shapes the paper's tests use: unit-square/cube domains,
refinement ratio 2, smooth right-hand sides):

* ``ms2d``     single-level 2-D Poisson, Dirichlet data of the manufactured solution
               phi = sin(2 pi x) sin(3 pi y) + x^2 y, RHS = 4x4 Gauss cell averages of Lap phi.
* ``bumps2d``  two-level 2-D hierarchy, base 256^2, one ratio-2 box over [0.25,0.75]^2,
               RHS = cell averages of a seeded sum of 8 Gaussian bumps (analytic, erf).
* ``batch2d``  96 independent single-level Helmholtz problems of uneven square sizes with
               seeded random Fourier-mode right-hand sides (|k| <= 16, |k|^-2 spectrum).
* ``adjoint2d`` three-level 2-D hierarchy (base 256^2, boxes [0.2,0.8]^2, [0.35,0.65]^2)
               with a seeded, smoothed N(0,1) forcing.
* ``bumps3d``  3-D base 256^3 with one ratio-2 box over [0.375,0.625]^3, Gaussian bumps.

Box coordinates are snapped outward to the coarse cells that contain them.
Seeds: ``numpy.random.default_rng(20250603 + workload_id)``.
"""
import math

import numpy as np

SEED0 = 20250603

_GL4_X = np.array([-0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526])
_GL4_W = np.array([0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538])


def rng(workload_id):
    return np.random.default_rng(SEED0 + workload_id)


# ----------------------------------------------------------------------------- geometry
def snapped_box(lo_x, hi_x, n_coarse, dim, ratio=2):
    """Fine-level box (inclusive, fine index space) covering [lo_x, hi_x]^dim, snapped
    outward to coarse cells of a level with ``n_coarse`` cells per dimension."""
    clo = int(math.floor(lo_x * n_coarse + 1e-12))
    chi = int(math.ceil(hi_x * n_coarse - 1e-12)) - 1
    return (tuple([ratio * clo] * dim), tuple([ratio * chi + ratio - 1] * dim))


def hierarchy_boxes(name, scale=1):
    """(dim, n0, boxes per level) for a named workload; ``scale`` divides the base size
    (used for the small parity cases)."""
    if name == "bumps2d":
        n = 256 // scale
        return 2, (n, n), [[((0, 0), (n - 1, n - 1))], [snapped_box(0.25, 0.75, n, 2)]]
    if name == "adjoint2d":
        n = 256 // scale
        b1 = snapped_box(0.2, 0.8, n, 2)
        # level-2 box: [0.35, 0.65] snapped to level-1 cells
        b2 = snapped_box(0.35, 0.65, 2 * n, 2)
        return 2, (n, n), [[((0, 0), (n - 1, n - 1))], [b1], [b2]]
    if name == "bumps3d":
        n = 256 // scale
        return 3, (n, n, n), [[((0,) * 3, (n - 1,) * 3)], [snapped_box(0.375, 0.625, n, 3)]]
    if name == "ms2d":
        n = 64 // scale
        return 2, (n, n), [[((0, 0), (n - 1, n - 1))]]
    raise KeyError(name)


def level_boxes_cells(boxes_l):
    return sum(int(np.prod([hi[d] - lo[d] + 1 for d in range(len(lo))])) for lo, hi in boxes_l)


# ----------------------------------------------------------------------------- quadrature
def cell_average_gauss(func, n, h, lo=None, origin=None, shape=None):
    """4x4 (or 4^3) Gauss-Legendre cell averages of func(x, y[, z]) over the cells
    origin + [0, shape) of a grid with spacing h.  Returns an array with axis d = dim d."""
    D = len(n)
    lo = lo if lo is not None else (0.0,) * D
    origin = origin if origin is not None else (0,) * D
    shape = shape or n
    axes = []
    for d in range(D):
        c = lo[d] + (np.arange(shape[d]) + origin[d] + 0.5) * h
        axes.append((c[:, None] + 0.5 * h * _GL4_X[None, :]))  # (n_d, 4)
    out = np.zeros(tuple(shape))
    for qi in np.ndindex(*([4] * D)):
        pts = np.meshgrid(*[axes[d][:, qi[d]] for d in range(D)], indexing="ij")
        w = np.prod([_GL4_W[qi[d]] for d in range(D)]) / 2.0 ** D
        out += w * func(*pts)
    return out


def face_average_gauss(func, n, h, d, side, lo=None):
    """4-point (per transverse dimension) Gauss face averages of func on the domain face
    (d, side) of a grid with n cells per dimension; array over the transverse cells."""
    D = len(n)
    lo = lo if lo is not None else (0.0,) * D
    tdims = [e for e in range(D) if e != d]
    xf = lo[d] + (0.0 if side == 0 else n[d] * h)
    axes = [lo[e] + (np.arange(n[e]) + 0.5)[:, None] * h + 0.5 * h * _GL4_X[None, :] for e in tdims]
    out = np.zeros(tuple(n[e] for e in tdims))
    for qi in np.ndindex(*([4] * (D - 1))):
        grids = np.meshgrid(*[axes[t][:, qi[t]] for t in range(D - 1)], indexing="ij")
        args = [None] * D
        args[d] = np.full(grids[0].shape, xf)
        for t, e in enumerate(tdims):
            args[e] = grids[t]
        w = np.prod([_GL4_W[qi[t]] for t in range(D - 1)]) / 2.0 ** (D - 1)
        out += w * func(*args)
    return out


# ----------------------------------------------------------------------------- ms2d
def ms_phi(x, y):
    return np.sin(2 * np.pi * x) * np.sin(3 * np.pi * y) + x * x * y


def ms_lap(x, y):
    return -13.0 * np.pi ** 2 * np.sin(2 * np.pi * x) * np.sin(3 * np.pi * y) + 2.0 * y


def ms2d(n):
    """Manufactured-solution Poisson problem on n x n cells: (rhs, dirichlet face data,
    exact cell averages of phi).  Face data: dict face -> array."""
    h = 1.0 / n
    rhs = cell_average_gauss(ms_lap, (n, n), h)
    exact = cell_average_gauss(ms_phi, (n, n), h)
    bc = {2 * d + s: face_average_gauss(ms_phi, (n, n), h, d, s) for d in range(2) for s in (0, 1)}
    return rhs, bc, exact


# ----------------------------------------------------------------------------- bumps
def bump_params(workload_id, nbumps=8, dim=2, component=0):
    """Centres, widths and amplitudes of the bumps; ``component`` > 0 draws an independent
    set (seeded by (SEED0 + workload_id, component)) for the other right-hand sides of one
    workload, e.g. the velocity components' Helmholtz systems."""
    g = rng(workload_id) if component == 0 else np.random.default_rng([SEED0 + workload_id, component])
    c = g.uniform(0.0, 1.0, size=(nbumps, dim))
    w = g.uniform(0.03, 0.1, size=nbumps)
    a = g.standard_normal(nbumps)
    return c, w, a


def _erf_int(a, b, c, w):
    """int_a^b exp(-(x-c)^2/w^2) dx."""
    from scipy.special import erf
    return 0.5 * math.sqrt(math.pi) * w * (erf((b - c) / w) - erf((a - c) / w))


def bumps_cell_averages(params, h, origin, shape):
    """Exact cell averages of sum_j a_j exp(-|x-c_j|^2 / w_j^2) over cells origin+[0,shape)."""
    c, w, a = params
    D = len(origin)
    out = np.zeros(tuple(shape))
    for j in range(len(a)):
        fac = []
        for d in range(D):
            lo = (np.arange(shape[d]) + origin[d]) * h
            fac.append(_erf_int(lo, lo + h, c[j, d], w[j]) / h)
        term = fac[0]
        for d in range(1, D):
            term = np.multiply.outer(term, fac[d])
        out += a[j] * term
    return out


def level_rhs(params_fn, dim, n0, boxes, ratio=2):
    """Per level, per box, cell averages (axis d = dim d) of an analytic RHS."""
    out = []
    for l, bl in enumerate(boxes):
        h = 1.0 / (n0[0] * ratio ** l)
        out.append([params_fn(h, lo, tuple(hi[d] - lo[d] + 1 for d in range(dim))) for lo, hi in bl])
    return out


def bumps2d_rhs(scale=1):
    dim, n0, boxes = hierarchy_boxes("bumps2d", scale)
    p = bump_params(2, 8, 2)
    return dim, n0, boxes, level_rhs(lambda h, o, s: bumps_cell_averages(p, h, o, s), dim, n0, boxes)


def bumps3d_rhs(scale=1, component=0):
    """Right-hand side of the 3-D workload: component 0 for the pressure Poisson equation,
    1..3 for the three velocity components' Helmholtz systems (independent bump sets)."""
    dim, n0, boxes = hierarchy_boxes("bumps3d", scale)
    p = bump_params(5, 8, 3, component)
    return dim, n0, boxes, level_rhs(lambda h, o, s: bumps_cell_averages(p, h, o, s), dim, n0, boxes)


# ----------------------------------------------------------------------------- batch2d
BATCH_SIZES = (64, 96, 128, 192, 256, 384, 512)


def batch2d_problems(nprob=96, sizes=BATCH_SIZES, kmax=16, workload_id=3):
    """List of dicts {n, alpha, beta, rhs}: alpha = 1, beta = -gamma*nu*k with gamma = 0.25,
    k = 1/256 and nu log-uniform in [1e-4, 1e-2]; rhs = exact cell averages of
    sum_{|k|<=kmax} a_k |k|^-2 sin(pi kx x) sin(pi ky y), a_k ~ N(0,1)."""
    g = rng(workload_id)
    ns = g.choice(np.asarray(sizes), size=nprob)
    nus = np.exp(g.uniform(math.log(1e-4), math.log(1e-2), size=nprob))
    modes = [(kx, ky) for kx in range(1, kmax + 1) for ky in range(1, kmax + 1) if kx * kx + ky * ky <= kmax * kmax]
    out = []
    for p in range(nprob):
        n = int(ns[p])
        a = g.standard_normal(len(modes))
        h = 1.0 / n
        edges = np.arange(n + 1) * h
        rhs = np.zeros((n, n))
        for (kx, ky), ak in zip(modes, a):
            # cell average of sin(pi k x) over [x_i, x_i + h] = (cos(pi k x_i) - cos(pi k x_{i+1}))/(pi k h)
            fx = (np.cos(np.pi * kx * edges[:-1]) - np.cos(np.pi * kx * edges[1:])) / (np.pi * kx * h)
            fy = (np.cos(np.pi * ky * edges[:-1]) - np.cos(np.pi * ky * edges[1:])) / (np.pi * ky * h)
            rhs += ak / (kx * kx + ky * ky) * np.outer(fx, fy)
        out.append({"n": n, "alpha": 1.0, "beta": -0.25 * float(nus[p]) / 256.0, "rhs": rhs})
    return out


# ----------------------------------------------------------------------------- adjoint2d
def adjoint2d_forcing(scale=1, sweeps=3, omega=2.0 / 3.0):
    """Two forcing components per level and box: N(0,1) cell values smoothed by ``sweeps``
    passes of g <- (1-omega) g + omega * mean of the 2D face neighbours (zero outside the
    domain), each level on its own grid (this is input generation, not the solver)."""
    dim, n0, boxes = hierarchy_boxes("adjoint2d", scale)
    g = rng(4)
    comps = []
    for _ in range(dim):
        lev = []
        for l, bl in enumerate(boxes):
            n = n0[0] * 2 ** l
            full = np.zeros((n, n))
            mask = np.zeros((n, n), bool)
            for lo, hi in bl:
                mask[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1] = True
            full[mask] = g.standard_normal(int(mask.sum()))
            for _s in range(sweeps):
                p = np.pad(full, 1)
                nb = (p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:]) / 4.0
                full = np.where(mask, (1 - omega) * full + omega * nb, 0.0)
            lev.append([full[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1].copy() for lo, hi in bl])
        comps.append(lev)
    return dim, n0, boxes, comps


HELMHOLTZ_BETA = -0.25 * 1e-3 / 256.0  # -gamma * nu * k with gamma = 0.25, nu = 1e-3, k = 1/256
