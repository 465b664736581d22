"""Marshalling between oracle composite fields (level arrays) and the library's packed
composite layout, for the GPU parity tests."""
import numpy as np


def to_packed(gh, H, F, fill=0.0):
    per = []
    for l, lev in enumerate(H.levels):
        per.append([F[l][lev.box_slice(lo, hi)] for lo, hi in lev.boxes])
    return gh.pack(per, fill=fill)


def from_packed(gh, H, flat):
    per = gh.unpack(flat)
    out = []
    for l, lev in enumerate(H.levels):
        a = np.full(lev.shape, np.nan)
        for k, (lo, hi) in enumerate(lev.boxes):
            a[lev.box_slice(lo, hi)] = per[l][k]
        out.append(a)
    return out


def max_diff(H, A, B, mask="valid"):
    m = 0.0
    for l, lev in enumerate(H.levels):
        sel = lev.valid if mask == "valid" else lev.covered
        if sel.any():
            m = max(m, float(np.max(np.abs(A[l][sel] - B[l][sel]))))
    return m


def max_abs(H, A, mask="valid"):
    m = 0.0
    for l, lev in enumerate(H.levels):
        sel = lev.valid if mask == "valid" else lev.covered
        if sel.any():
            m = max(m, float(np.max(np.abs(A[l][sel]))))
    return m


def op_scale(H, alpha, beta, phi):
    """Bound on |A phi| terms: (|alpha| + |beta| * sum|L coefs| / h_min^2) * max|phi|, with
    a factor for the one-sided ghost coefficients near physical faces."""
    hmin = min(lev.h for lev in H.levels)
    return (abs(alpha) + abs(beta) * 8.0 * 64.0 / 12.0 * H.D / hmin ** 2) * max_abs(H, phi, "covered")


def level_bc_data(H, funcs):
    """Per level: dict face -> array of face data from funcs(d, side) -> callable."""
    from paper_2506_02663_gb300.workloads import face_average_gauss
    out = []
    for lev in H.levels:
        out.append({2 * d + s: face_average_gauss(funcs(d, s), lev.ndom, lev.h, d, s)
                    for d in range(H.D) for s in (0, 1)})
    return out
