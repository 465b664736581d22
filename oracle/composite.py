"""Composite data and composite operators of Sec. 5.2-5.3 (oracle; test infrastructure).

A composite field is a list of level arrays (see ``hierarchy.Level``); values live on the
covered cells of each level, NaN elsewhere until ghosts are filled.

* Eq. (AMR_avergingDownToCrse): ``average_down``.
* COH-1: ``fill_ghosts`` -- same-level data are implicit in a level array, AMRCFI for CF
  ghosts (``cfi.py``), Eqs. (velBCHomoDiri5th)/(Neumann5) for physical ghosts.
* COH-2: the level operators of ``stencil.py``.
* COH-3: ``reflux`` -- on each coarse valid cell that shares a face with the invalid region,
  the coarse flux through that face is replaced by the mean of the fine fluxes through the
  r^(D-1) fine faces that tile it (fluxes of Eq. (cell2face)).
* COH-4: ``average_down`` of the result.
* Eq. (comp_ProjOp) and Lemma compositeProjection: ``project`` -- no COH-4 on the result.
"""
import numpy as np

from . import stencil as st
from .cfi import cfi_values


def new_field(H, batch=(), fill=0.0):
    """Composite field: covered cells set to ``fill``, everything else NaN."""
    F = []
    for lev in H.levels:
        a = np.full(lev.shape + tuple(batch), np.nan)
        a[lev.covered] = fill
        F.append(a)
    return F


def average_down(H, F, l):
    """Eq. (AMR_avergingDownToCrse): every cell of level l under level l+1 receives the
    mean of its r^D children."""
    r, D = H.ratio, H.D
    lev, fine = H.levels[l], H.levels[l + 1]
    for lo, hi in fine.boxes:
        fs = fine.box_slice(lo, hi)
        block = F[l + 1][fs]
        acc = 0.0
        for offs in np.ndindex(*([r] * D)):
            idx = tuple(slice(offs[d], None, r) for d in range(D))
            acc = acc + block[idx]
        clo = tuple(v // r for v in lo)
        chi = tuple(v // r for v in hi)
        F[l][lev.box_slice(clo, chi)] = acc / r ** D


def average_down_all(H, F):
    for l in range(H.lmax - 1, -1, -1):
        average_down(H, F, l)


def fill_cf_ghosts(H, F, l):
    """AMRCFI values on every CF ghost cell of level l >= 1 from level l-1 (which must
    already hold redundant data on its invalid region)."""
    lev, crs = H.levels[l], H.levels[l - 1]
    cells = np.argwhere(lev.cf_ghost)
    if cells.size == 0:
        return
    g = cells + np.asarray(lev.origin)
    vals, _ = cfi_values(F[l - 1], crs.origin, crs.ndom, g, H.ratio, H.D)
    F[l][tuple(cells.T)] = vals


def fill_ghosts(H, F, l, bc_data=None, cf_zero=False, bc_types=None):
    """COH-1 for level l: CF ghosts (AMRCFI, or zero when ``cf_zero``), then physical
    ghosts (corners outside the domain in two dimensions stay untouched)."""
    lev = H.levels[l]
    if l > 0:
        if cf_zero:
            F[l][lev.cf_ghost] = 0.0
        else:
            fill_cf_ghosts(H, F, l)
    st.fill_physical_ghosts(F[l], lev.origin, lev.ndom, lev.covered, H.D, lev.h,
                            bc_types if bc_types is not None else H.bc, bc_data)


def _mask(Y, lev):
    Y[~lev.covered] = np.nan
    return Y


def cf_faces(H, l):
    """Coarse CF faces of level l < lmax: list of (d, s, cells) where ``cells`` (n, D) are
    array indices of valid cells whose neighbour c + s*e^d is invalid (s = +1: the face is
    the cell's high face)."""
    lev = H.levels[l]
    out = []
    for d in range(H.D):
        for s in (1, -1):
            nb = np.zeros(lev.shape, bool)
            src = [slice(None)] * H.D
            dst = [slice(None)] * H.D
            if s == 1:
                dst[d], src[d] = slice(0, -1), slice(1, None)
            else:
                dst[d], src[d] = slice(1, None), slice(0, -1)
            nb[tuple(dst)] = lev.invalid[tuple(src)]
            cells = np.argwhere(lev.valid & nb)
            if len(cells):
                out.append((d, s, cells))
    return out


def _flux(P, D, h, d, cells, kind):
    if kind == "deriv":
        return st.face_flux_deriv(P, D, h, d, tuple(cells.T))
    return st.face_value(P, D, d, tuple(cells.T))


def reflux(H, P, Y, coef, kind):
    """COH-3.  ``P`` holds ghost-filled composite data, ``Y`` the per-level results.
    kind 'deriv': Laplacian fluxes (face normal derivative), result += coef*s*(Fbar-Fc)/h;
    kind 'value': divergence fluxes (face values of the d-th component, P is then the list
    of component fields), result += coef*s*(Ubar-Uc)/h."""
    r, D = H.ratio, H.D
    for l in range(H.lmax - 1, -1, -1):
        lev, fine = H.levels[l], H.levels[l + 1]
        for d, s, cells in cf_faces(H, l):
            Pc = P[l] if kind == "deriv" else P[d][l]
            Pf = P[l + 1] if kind == "deriv" else P[d][l + 1]
            # coarse flux through the face: high face of c (s=+1) or of c-e^d (s=-1)
            owner = cells.copy()
            if s == -1:
                owner[:, d] -= 1
            Fc = _flux(Pc, D, lev.h, d, owner, kind)
            # fine faces tiling it: the face at fine index r*(c_d + 1) (s=+1) or r*c_d (s=-1)
            gc = cells + np.asarray(lev.origin)
            Fsum = 0.0
            tdims = [e for e in range(D) if e != d]
            for offs in np.ndindex(*([r] * (D - 1))):
                gf = np.empty_like(gc)
                for t, e in enumerate(tdims):
                    gf[:, e] = r * gc[:, e] + offs[t]
                # high face of fine cell gf_d, gf_d = r*(c_d+1) - 1 (s=+1) or r*c_d - 1 (s=-1)
                gf[:, d] = r * (gc[:, d] + 1) - 1 if s == 1 else r * gc[:, d] - 1
                af = gf - np.asarray(fine.origin)
                Fsum = Fsum + _flux(Pf, D, fine.h, d, af, kind)
            Fbar = Fsum / r ** (D - 1)
            idx = tuple(cells.T)
            Y[l][idx] = Y[l][idx] + coef * s * (Fbar - Fc) / lev.h


def _prepared(H, F, bc_data, bc_types=None):
    """COH-1 on a copy of F: average down, then ghosts level by level."""
    P = [a.copy() for a in F]
    average_down_all(H, P)
    for l in range(H.lmax + 1):
        fill_ghosts(H, P, l, None if bc_data is None else bc_data[l], bc_types=bc_types)
    return P


def apply(H, phi, alpha, beta, bc_data=None):
    """Composite alpha*phi + beta*L^comp phi (COH-1..4).  bc_data: None (homogeneous) or a
    list over levels of per-face dicts (see stencil.fill_physical_ghosts)."""
    P = _prepared(H, phi, bc_data)
    Y = [_mask(st.helmholtz(P[l], H.D, lev.h, alpha, beta), lev) for l, lev in enumerate(H.levels)]
    reflux(H, P, Y, beta, "deriv")
    average_down_all(H, Y)
    return Y


def residual(H, phi, f, alpha, beta, bc_data=None):
    """f - A^comp phi on covered cells (meaningful on valid cells)."""
    Y = apply(H, phi, alpha, beta, bc_data)
    return [_mask(f[l] - Y[l], lev) for l, lev in enumerate(H.levels)]


def gradient(H, phi, bc_data=None, bc_types=None):
    """G^comp: COH-1, 2, 4 (G is not in divergence form; no refluxing)."""
    P = _prepared(H, phi, bc_data, bc_types)
    G = []
    for d in range(H.D):
        Gd = [_mask(st.gradient(P[l], H.D, lev.h, d), lev) for l, lev in enumerate(H.levels)]
        average_down_all(H, Gd)
        G.append(Gd)
    return G


def divergence(H, U, bc_data=None, bc_types=None):
    """D^comp: COH-1..4 with refluxing of the face values of Eq. (cell2face)."""
    Ps = [_prepared(H, U[d], None if bc_data is None else bc_data[d], bc_types) for d in range(H.D)]
    Y = []
    for l, lev in enumerate(H.levels):
        Y.append(_mask(st.divergence([Ps[d][l] for d in range(H.D)], H.D, lev.h), lev))
    reflux(H, Ps, Y, 1.0, "value")
    average_down_all(H, Y)
    return Y
