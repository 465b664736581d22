"""Thin Python binding of libamr4 (ctypes).  Argument marshalling only: every step of the
solver runs in the library's CUDA kernels.  The library must have been built
(``__graft_entry__.build()``); importing this module without it raises ImportError --
there is no fallback path.

Field arguments are torch CUDA tensors (float64, contiguous, ``numel == nelems``) holding
a composite field in the library's padded layout (``Hierarchy.pack`` / ``unpack`` convert
from and to per-box numpy arrays whose axis d is the paper's dimension d).
"""
import ctypes as C
import os

import numpy as np

from .build import LIB

if not os.path.exists(LIB):
    raise ImportError(f"libamr4 is not built ({LIB} missing); run __graft_entry__.build()")
_lib = C.CDLL(LIB)

AMR_OK, AMR_ERR_INVALID_ARG, AMR_ERR_NESTING, AMR_ERR_REFINEMENT, AMR_ERR_BOX_TOO_SMALL = 0, 1, 2, 3, 4
AMR_ERR_NOT_CONVERGED, AMR_ERR_NONFINITE, AMR_ERR_CUDA, AMR_ERR_OOM = 5, 6, 7, 8
DIRICHLET, NEUMANN = 0, 1
FP64, MIXED = 0, 1
NG = 2


class HierarchyDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("ratio", C.c_int), ("n0", C.c_int * 3), ("h0", C.c_double),
                ("nlevels", C.c_int), ("nboxes", C.POINTER(C.c_int)), ("boxes", C.POINTER(C.c_int))]


class PatchInfo(C.Structure):
    _fields_ = [("level", C.c_int), ("box", C.c_int), ("lo", C.c_int * 3), ("hi", C.c_int * 3),
                ("offset", C.c_longlong), ("stride_y", C.c_longlong), ("stride_z", C.c_longlong),
                ("nelems", C.c_longlong)]


class IndexMaps(C.Structure):
    _fields_ = [("ncells_interior", C.c_longlong), ("ncells_padded", C.c_longlong),
                ("valid", C.POINTER(C.c_int)), ("component", C.POINTER(C.c_int)),
                ("ghost_code", C.POINTER(C.c_int)), ("ghost_src", C.POINTER(C.c_int)),
                ("ghost_aux", C.POINTER(C.c_int)), ("ncfi", C.c_longlong),
                ("cfi_cell", C.POINTER(C.c_longlong)), ("cfi_start", C.POINTER(C.c_int)),
                ("cfi_pos", C.POINTER(C.c_int)), ("cfi_sub", C.POINTER(C.c_int)),
                ("nreflux", C.c_longlong), ("reflux_cell", C.POINTER(C.c_int)),
                ("reflux_faces", C.POINTER(C.c_int))]


class SolverParams(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double), ("rtol", C.c_double),
                ("atol", C.c_double), ("max_vcycles", C.c_int), ("precision", C.c_int),
                ("zero_initial", C.c_int), ("use_graph", C.c_int), ("fuse_coarse", C.c_int),
                ("temporal_blocking", C.c_int), ("cycles_per_refinement", C.c_int)]


class RegridParams(C.Structure):
    _fields_ = [("efficiency", C.c_double), ("min_width", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("vcycles", C.c_int), ("rhs_norm", C.c_double), ("final_res", C.c_double),
                ("removed_mean", C.c_double), ("res_history", C.c_double * 64)]


_vp = C.c_void_p
_P = C.POINTER
_sigs = {
    "amr_hierarchy_create": [_P(HierarchyDesc), _P(_vp)],
    "amr_hierarchy_destroy": [_vp],
    "amr_field_layout": [_vp, _P(C.c_int), _P(C.c_longlong), _P(PatchInfo)],
    "amr_bc_layout": [_vp, _P(C.c_longlong)],
    "amr_get_index_maps": [_vp, _P(IndexMaps)],
    "amr_operator_create": [_vp, C.c_double, C.c_double, _P(C.c_int), _P(_vp)],
    "amr_operator_destroy": [_vp],
    "amr_fill_ghosts": [_vp, _vp, _vp, _vp],
    "amr_apply": [_vp, _vp, _vp, _vp, _vp],
    "amr_residual": [_vp, _vp, _vp, _vp, _vp, _P(C.c_double), _vp],
    "amr_smooth": [_vp, C.c_int, C.c_int, C.c_double, _vp, _vp, _vp],
    "amr_vcycle": [_vp, _P(SolverParams), _vp, _vp, _vp, _vp],
    "amr_solve": [_vp, _P(SolverParams), _vp, _vp, _vp, _P(SolveStats), _vp],
    "amr_solve_host": [_vp, _P(SolverParams), _vp, _vp, _vp, _P(SolveStats), _vp],
    "amr_batch_solve": [_P(_vp), C.c_int, _P(SolverParams), _P(_vp), _P(_vp), _P(SolveStats), _P(C.c_int), _vp],
    "amr_batch_solve_host": [_P(_vp), C.c_int, _P(SolverParams), _P(_vp), _P(_vp), _P(SolveStats), _P(C.c_int), _vp],
    "amr_solvability_fix": [_vp, _vp, _vp, _P(C.c_double), _vp],
    "amr_mean_zero": [_vp, _vp, _P(C.c_double), _vp],
    "amr_mean_zero_noalloc": [_vp, _vp, _P(C.c_double), _vp],
    "amr_gradient": [_vp, _P(C.c_int), _vp, _P(_vp), _vp, _vp],
    "amr_divergence": [_vp, _P(C.c_int), _P(_vp), _vp, _P(_vp), _vp],
    "amr_project": [_vp, _P(SolverParams), _P(C.c_int), _P(_vp), _P(_vp), _P(_vp), _vp, _P(SolveStats), _vp],
    "amr_apply_transpose": [_vp, _vp, _vp, _vp],
    "amr_solve_transpose": [_vp, _P(SolverParams), _vp, _vp, _P(SolveStats), _vp],
    "amr_gradient_transpose": [_vp, _P(C.c_int), _P(_vp), _vp, _vp],
    "amr_divergence_transpose": [_vp, _P(C.c_int), _vp, _P(_vp), _vp],
    "amr_project_transpose": [_vp, _P(SolverParams), _P(C.c_int), _P(_vp), _P(_vp), _vp, _P(SolveStats), _vp],
    "amr_cic_ghosts": [_vp, C.c_int, _P(_vp), C.c_double, C.c_double, _vp, _vp, _vp],
    "amr_cic_faces": [_vp, C.c_int, _P(C.c_int), _P(C.c_int), _P(C.c_int), _P(C.c_int), _P(C.c_int)],
    "amr_cic_face_averages": [_vp, C.c_int, _P(_vp), _vp, _vp, _vp, _vp],
    "amr_cic_component_box": [_vp, C.c_int, C.c_int, _P(C.c_int), _P(C.c_int), _P(C.c_int)],
    "amr_migrate": [_vp, _vp, _vp, _vp, _vp],
    "amr_migrate_plan": [_vp, _vp, C.c_int, _P(C.c_int), _P(C.c_int), _P(C.c_longlong), _P(C.c_int), _P(C.c_int),
                         _P(C.c_longlong), _P(C.c_longlong), _P(C.c_longlong), _P(C.c_longlong)],
    "amr_regrid": [C.c_int, C.c_int, _P(C.c_int), C.c_int, _P(C.c_int), _P(_P(C.c_int)), _P(RegridParams),
                   _P(C.c_int), _P(C.c_int), _P(C.c_int), C.c_int],
    "amr_cic_interface_bc": [_vp, C.c_int, C.c_int, _vp, _vp, _vp],
    "amr_default_params": [_P(SolverParams)],
    "amr_last_error": [],
    "amr_kernel_launches": [],
    "amr_profile_enable": [C.c_int],
    "amr_set_tile_rows": [C.c_int],
    "amr_set_fx_residual": [C.c_int],
    "amr_set_bulk_sweep": [C.c_int],
    "amr_check_kernel_flags": [],
    "amr_set_stacked_batches": [C.c_int],
    "amr_profile_read": [C.c_int, _P(C.c_longlong), _P(C.c_double), _P(C.c_double)],
    "amr_profile_read_range": [C.c_int, C.c_double, C.c_double, _P(C.c_longlong), _P(C.c_double), _P(C.c_double)],
}
for _n, _a in _sigs.items():
    _f = getattr(_lib, _n)
    _f.argtypes = _a
    _f.restype = C.c_int
_lib.amr_hierarchy_destroy.restype = None
_lib.amr_operator_destroy.restype = None
_lib.amr_default_params.restype = None
_lib.amr_last_error.restype = C.c_char_p
_lib.amr_kernel_launches.restype = C.c_longlong


def kernel_launches():
    return int(_lib.amr_kernel_launches())


KC_JACOBI, KC_RESID, KC_RESTRICT, KC_PROLONG, KC_DOWN, KC_UP, KC_COARSE, KC_RESID64 = 0, 1, 2, 3, 4, 5, 6, 7


def set_tile_rows(rows):
    """0: autotuned tile shape per grid; 1, 2, 4: cells per thread along y forced in the tiled
    level-operator kernels (3-D: 2 or 4)."""
    _check(_lib.amr_set_tile_rows(int(rows)), "amr_set_tile_rows")


def set_fx_residual(on):
    """1 (default): the 3-D FP64 residual forms its stencil sums exactly in 64-bit fixed point
    (falling back to the plain FP64 kernel when a value leaves the frame); 0: plain FP64."""
    _check(_lib.amr_set_fx_residual(int(on)), "amr_set_fx_residual")


def set_bulk_sweep(on):
    """3-D single-patch levels with x extents a multiple of 64 and y extents a multiple of 16:
    1 (default) the autotuner picks the bulk-copy (TMA) or the z-chunked level operator per
    grid; 2 always the bulk-copy kernel; 0 never."""
    _check(_lib.amr_set_bulk_sweep(int(on)), "amr_set_bulk_sweep")


def set_stacked_batches(on):
    """1: 3-D batches of one geometry and one operator are solved as one stacked problem (one
    launch per phase over all problems); 0 (default): one captured solve per problem,
    launched concurrently."""
    _check(_lib.amr_set_stacked_batches(int(on)), "amr_set_stacked_batches")


def check_kernel_flags():
    """Raises AmrError if a bounded pipeline wait of the 3-D kernel ran out since the last check."""
    _check(_lib.amr_check_kernel_flags(), "amr_check_kernel_flags")


def profile_enable(on):
    _check(_lib.amr_profile_enable(1 if on else 0), "amr_profile_enable")


def profile_read(kernel_class):
    n = C.c_longlong()
    ms = C.c_double()
    by = C.c_double()
    _check(_lib.amr_profile_read(kernel_class, C.byref(n), C.byref(ms), C.byref(by)), "amr_profile_read")
    return {"launches": n.value, "ms": ms.value, "bytes": by.value}


def profile_read_range(kernel_class, min_cells, max_cells):
    """Sums over the recorded launches of one class on grids of min_cells..max_cells cells."""
    n = C.c_longlong()
    ms = C.c_double()
    by = C.c_double()
    _check(_lib.amr_profile_read_range(kernel_class, float(min_cells), float(max_cells), C.byref(n), C.byref(ms),
                                       C.byref(by)), "amr_profile_read_range")
    return {"launches": n.value, "ms": ms.value, "bytes": by.value}

EXPORTED = tuple(_sigs)


class AmrError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.amr_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def _check(st, where, ok=(AMR_OK,)):
    if st not in ok:
        raise AmrError(st, where)
    return st


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return _vp(t.data_ptr())
    return _vp(int(t))


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return _vp(stream.cuda_stream)
    return _vp(int(stream))


def default_params(**kw):
    p = SolverParams()
    _lib.amr_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def stats_dict(s):
    n = min(s.vcycles + 1, 64)
    return {"vcycles": s.vcycles, "rhs_norm": s.rhs_norm, "final_res": s.final_res,
            "removed_mean": s.removed_mean, "res_history": list(s.res_history[:n])}


class Hierarchy:
    """amr_hierarchy: boxes per level as [(lo, hi), ...] with inclusive tuples."""

    def __init__(self, dim, n0, boxes, h0=None, ratio=2):
        self.dim = dim
        self.n0 = tuple(n0)
        self.boxes = [[(tuple(lo), tuple(hi)) for lo, hi in bl] for bl in boxes]
        self.nlevels = len(boxes)
        self.h0 = h0 if h0 is not None else 1.0 / n0[0]
        nb = (C.c_int * self.nlevels)(*[len(b) for b in boxes])
        flat = []
        for bl in boxes:
            for lo, hi in bl:
                flat += list(lo) + list(hi)
        fb = (C.c_int * len(flat))(*flat)
        d = HierarchyDesc(dim, ratio, (C.c_int * 3)(*(list(n0) + [1] * (3 - dim))), self.h0,
                          self.nlevels, nb, fb)
        self._h = _vp()
        _check(_lib.amr_hierarchy_create(C.byref(d), C.byref(self._h)), "amr_hierarchy_create")
        npatch = C.c_int()
        ne = C.c_longlong()
        _check(_lib.amr_field_layout(self._h, C.byref(npatch), C.byref(ne), None), "amr_field_layout")
        arr = (PatchInfo * npatch.value)()
        _check(_lib.amr_field_layout(self._h, None, None, arr), "amr_field_layout")
        self.nelems = ne.value
        self.patches = [{"level": p.level, "box": p.box, "lo": tuple(p.lo[:dim]), "hi": tuple(p.hi[:dim]),
                         "offset": p.offset, "sy": p.stride_y, "sz": p.stride_z, "nelems": p.nelems}
                        for p in arr]
        offs = (C.c_longlong * (self.nlevels * 2 * dim + 1))()
        _check(_lib.amr_bc_layout(self._h, offs), "amr_bc_layout")
        self.bc_offsets = list(offs)
        self.ratio = ratio

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.amr_hierarchy_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- index maps
    def index_maps(self):
        m = IndexMaps()
        _check(_lib.amr_get_index_maps(self._h, C.byref(m)), "amr_get_index_maps")

        def arr(ptr, n, dt):
            if n == 0:
                return np.zeros(0, dt)
            return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt).copy()

        D = self.dim
        return {
            "valid": arr(m.valid, m.ncells_interior, np.int32),
            "component": arr(m.component, sum(len(b) for b in self.boxes), np.int32),
            "ghost_code": arr(m.ghost_code, m.ncells_padded, np.int32),
            "ghost_src": arr(m.ghost_src, m.ncells_padded, np.int32),
            "ghost_aux": arr(m.ghost_aux, m.ncells_padded, np.int32),
            "cfi_cell": arr(m.cfi_cell, m.ncfi, np.int64),
            "cfi_start": arr(m.cfi_start, m.ncfi * D, np.int32).reshape(-1, D),
            "cfi_pos": arr(m.cfi_pos, m.ncfi * D, np.int32).reshape(-1, D),
            "cfi_sub": arr(m.cfi_sub, m.ncfi * D, np.int32).reshape(-1, D),
            "reflux_cell": arr(m.reflux_cell, m.nreflux * 3, np.int32).reshape(-1, 3),
            "reflux_faces": arr(m.reflux_faces, m.nreflux, np.int32),
        }

    # ---------------------------------------------------------------- marshalling
    def _view(self, arr, p):
        """Padded [z][y][x] view of patch p inside a flat composite array."""
        D = self.dim
        n = [p["hi"][d] - p["lo"][d] + 1 for d in range(D)]
        seg = arr[p["offset"]:p["offset"] + p["nelems"]]
        if D == 2:
            return seg.reshape(n[1] + 2 * NG, p["sy"])
        return seg.reshape(n[2] + 2 * NG, n[1] + 2 * NG, p["sy"])

    def interior(self, arr, p):
        D = self.dim
        n = [p["hi"][d] - p["lo"][d] + 1 for d in range(D)]
        v = self._view(arr, p)
        if D == 2:
            return v[NG:NG + n[1], NG:NG + n[0]]
        return v[NG:NG + n[2], NG:NG + n[1], NG:NG + n[0]]

    def pack(self, per_box, fill=0.0, dtype=np.float64):
        """per_box[l][k]: array with axis d = dimension d over box k of level l."""
        out = np.full(self.nelems, fill, dtype=dtype)
        i = 0
        for l, bl in enumerate(self.boxes):
            for k in range(len(bl)):
                p = self.patches[i]
                self.interior(out, p)[...] = np.asarray(per_box[l][k]).transpose()
                i += 1
        return out

    def unpack(self, flat):
        """Composite flat numpy array -> per_box[l][k] arrays (axis d = dimension d)."""
        flat = np.asarray(flat)
        out = []
        i = 0
        for l, bl in enumerate(self.boxes):
            lev = []
            for k in range(len(bl)):
                lev.append(self.interior(flat, self.patches[i]).transpose().copy())
                i += 1
            out.append(lev)
        return out

    def pack_bc(self, data):
        """data[l]: dict face -> array over the domain face at level l (axis order of the
        remaining dimensions), or None.  Returns the flat bc array of the ABI layout."""
        D = self.dim
        out = np.zeros(self.bc_offsets[-1])
        for l in range(self.nlevels):
            if data is None or data[l] is None:
                continue
            for f in range(2 * D):
                if f in data[l] and data[l][f] is not None:
                    a = self.bc_offsets[l * 2 * D + f]
                    b = self.bc_offsets[l * 2 * D + f + 1]
                    out[a:b] = np.asarray(data[l][f], dtype=np.float64).transpose().ravel()
        return out


class Operator:
    """amr_operator: alpha*I + beta*L^comp with boundary types bc_types (2*dim ints)."""

    def __init__(self, hier, alpha, beta, bc_types):
        self.h = hier
        self.alpha, self.beta = alpha, beta
        self.bc_types = list(bc_types)
        bt = (C.c_int * len(bc_types))(*bc_types)
        self._op = _vp()
        _check(_lib.amr_operator_create(hier.handle, alpha, beta, bt, C.byref(self._op)), "amr_operator_create")

    def close(self):
        if self._op:
            _lib.amr_operator_destroy(self._op)
            self._op = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fill_ghosts(self, phi, bc=None, stream=None):
        _check(_lib.amr_fill_ghosts(self._op, _ptr(phi), _ptr(bc), _stream(stream)), "amr_fill_ghosts")

    def apply(self, phi, out, bc=None, stream=None):
        _check(_lib.amr_apply(self._op, _ptr(phi), _ptr(out), _ptr(bc), _stream(stream)), "amr_apply")

    def residual(self, phi, f, res, bc=None, stream=None):
        nrm = C.c_double()
        _check(_lib.amr_residual(self._op, _ptr(phi), _ptr(f), _ptr(res), _ptr(bc), C.byref(nrm),
                                 _stream(stream)), "amr_residual")
        return nrm.value

    def smooth(self, level, nsweeps, omega, x, b, stream=None):
        _check(_lib.amr_smooth(self._op, level, nsweeps, omega, _ptr(x), _ptr(b), _stream(stream)), "amr_smooth")

    def vcycle(self, phi, f, bc=None, params=None, stream=None):
        p = params or default_params()
        _check(_lib.amr_vcycle(self._op, C.byref(p), _ptr(phi), _ptr(f), _ptr(bc), _stream(stream)), "amr_vcycle")

    def solve(self, phi, f, bc=None, params=None, stream=None, allow_not_converged=False):
        p = params or default_params()
        s = SolveStats()
        ok = (AMR_OK, AMR_ERR_NOT_CONVERGED) if allow_not_converged else (AMR_OK,)
        st = _lib.amr_solve(self._op, C.byref(p), _ptr(phi), _ptr(f), _ptr(bc), C.byref(s), _stream(stream))
        _check(st, "amr_solve", ok)
        d = stats_dict(s)
        d["status"] = st
        return d

    def solve_host(self, phi_host, f_host, bc_host=None, params=None, stream=None):
        """phi_host / f_host: numpy float64 arrays (HOST memory) in the composite layout."""
        p = params or default_params()
        s = SolveStats()
        bcp = None if bc_host is None else _vp(bc_host.ctypes.data)
        _check(_lib.amr_solve_host(self._op, C.byref(p), _vp(phi_host.ctypes.data), _vp(f_host.ctypes.data), bcp,
                                   C.byref(s), _stream(stream)), "amr_solve_host")
        return stats_dict(s)

    def solvability_fix(self, f, bc=None, stream=None):
        m = C.c_double()
        _check(_lib.amr_solvability_fix(self._op, _ptr(f), _ptr(bc), C.byref(m), _stream(stream)),
               "amr_solvability_fix")
        return m.value

    def apply_transpose(self, y, out, stream=None):
        _check(_lib.amr_apply_transpose(self._op, _ptr(y), _ptr(out), _stream(stream)), "amr_apply_transpose")

    def solve_transpose(self, lam, g, params=None, stream=None):
        p = params or default_params()
        s = SolveStats()
        _check(_lib.amr_solve_transpose(self._op, C.byref(p), _ptr(lam), _ptr(g), C.byref(s), _stream(stream)),
               "amr_solve_transpose")
        return stats_dict(s)


def batch_solve(ops, phis, fs, params=None, stream=None):
    """amr_batch_solve: returns (list of stats dicts, list of statuses)."""
    n = len(ops)
    p = params or default_params()
    oa = (_vp * n)(*[op._op.value for op in ops])
    st = (SolveStats * n)()
    sc = (C.c_int * n)()
    rc = _lib.amr_batch_solve(oa, n, C.byref(p), _ptr_array(phis), _ptr_array(fs), st, sc, _stream(stream))
    _check(rc, "amr_batch_solve", (AMR_OK, AMR_ERR_NOT_CONVERGED))
    return [stats_dict(st[k]) for k in range(n)], list(sc)


def batch_solve_host(ops, phis_host, fs_host, params=None, stream=None):
    """amr_batch_solve_host: numpy float64 HOST arrays in the composite layout (pinned or
    pageable); returns (list of stats dicts, list of statuses)."""
    n = len(ops)
    p = params or default_params()
    oa = (_vp * n)(*[op._op.value for op in ops])
    st = (SolveStats * n)()
    sc = (C.c_int * n)()
    ph = (_vp * n)(*[a.ctypes.data for a in phis_host])
    fh = (_vp * n)(*[a.ctypes.data for a in fs_host])
    rc = _lib.amr_batch_solve_host(oa, n, C.byref(p), ph, fh, st, sc, _stream(stream))
    _check(rc, "amr_batch_solve_host", (AMR_OK, AMR_ERR_NOT_CONVERGED))
    return [stats_dict(st[k]) for k in range(n)], list(sc)


def _ptr_array(ts):
    return (_vp * len(ts))(*[None if t is None else t.data_ptr() for t in ts])


def mean_zero(hier, phi, stream=None):
    m = C.c_double()
    _check(_lib.amr_mean_zero(hier.handle, _ptr(phi), C.byref(m), _stream(stream)), "amr_mean_zero")
    return m.value


def mean_zero_noalloc(hier, phi, stream=None):
    """amr_mean_zero_noalloc: the same result as mean_zero for callers that must not allocate
    device memory during the call (scratch is a fixed array inside the library)."""
    m = C.c_double()
    _check(_lib.amr_mean_zero_noalloc(hier.handle, _ptr(phi), C.byref(m), _stream(stream)), "amr_mean_zero_noalloc")
    return m.value


def gradient(hier, bc_types, phi, grads, bc=None, stream=None):
    bt = (C.c_int * len(bc_types))(*bc_types)
    _check(_lib.amr_gradient(hier.handle, bt, _ptr(phi), _ptr_array(grads), _ptr(bc), _stream(stream)),
           "amr_gradient")


def divergence(hier, bc_types, u, out, bc=None, stream=None):
    bt = (C.c_int * len(bc_types))(*bc_types)
    bcp = None if bc is None else _ptr_array(bc)
    _check(_lib.amr_divergence(hier.handle, bt, _ptr_array(u), _ptr(out), bcp, _stream(stream)), "amr_divergence")


def gradient_transpose(hier, bc_types, y, out, stream=None):
    """amr_gradient_transpose: out = (G^comp)^T y (y: dim fields)."""
    bt = (C.c_int * len(bc_types))(*bc_types)
    _check(_lib.amr_gradient_transpose(hier.handle, bt, _ptr_array(y), _ptr(out), _stream(stream)),
           "amr_gradient_transpose")


def divergence_transpose(hier, bc_types, y, out, stream=None):
    """amr_divergence_transpose: out[d] = component d of (D^comp)^T y."""
    bt = (C.c_int * len(bc_types))(*bc_types)
    _check(_lib.amr_divergence_transpose(hier.handle, bt, _ptr(y), _ptr_array(out), _stream(stream)),
           "amr_divergence_transpose")


def project_transpose(ppe, vel_bc_types, v, out, lam, params=None, stream=None):
    """amr_project_transpose: out = P^T v; lam receives the adjoint potential."""
    p = params or default_params()
    s = SolveStats()
    bt = (C.c_int * len(vel_bc_types))(*vel_bc_types)
    _check(_lib.amr_project_transpose(ppe._op, C.byref(p), bt, _ptr_array(v), _ptr_array(out), _ptr(lam),
                                      C.byref(s), _stream(stream)), "amr_project_transpose")
    return stats_dict(s)


def project(ppe, vel_bc_types, w, u, phi, w_bc=None, params=None, stream=None):
    p = params or default_params()
    s = SolveStats()
    bt = (C.c_int * len(vel_bc_types))(*vel_bc_types)
    wb = None if w_bc is None else _ptr_array(w_bc)
    _check(_lib.amr_project(ppe._op, C.byref(p), bt, _ptr_array(w), wb, _ptr_array(u), _ptr(phi), C.byref(s),
                            _stream(stream)), "amr_project")
    return stats_dict(s)


def cic_ghosts(hier, level, coarse, k, eta, value, rate=None, stream=None):
    """amr_cic_ghosts: the CF ghosts of `level` at t* from the four coarse time levels
    ``coarse`` (columns of I^(4) in order) into ``value`` and, when given, d/dt into ``rate``."""
    if len(coarse) != 4:
        raise ValueError("cic_ghosts needs four coarse time levels")
    _check(_lib.amr_cic_ghosts(hier.handle, int(level), _ptr_array(coarse), float(k), float(eta), _ptr(value),
                               _ptr(rate), _stream(stream)), "amr_cic_ghosts")


def cic_faces(hier, level):
    """amr_cic_faces: the interface faces of `level` as numpy arrays: cell (n, dim) global index
    of the interior cell, face (n,) = 2 d + side, component (n,); and the component count."""
    nf, nc = C.c_int(), C.c_int()
    _check(_lib.amr_cic_faces(hier.handle, int(level), C.byref(nf), C.byref(nc), None, None, None), "amr_cic_faces")
    n, D = nf.value, hier.dim
    cell = (C.c_int * max(1, n * D))()
    face = (C.c_int * max(1, n))()
    comp = (C.c_int * max(1, n))()
    _check(_lib.amr_cic_faces(hier.handle, int(level), None, None, cell, face, comp), "amr_cic_faces")
    return {"cell": np.ctypeslib.as_array(cell)[:n * D].reshape(n, D).copy(),
            "face": np.ctypeslib.as_array(face)[:n].copy(),
            "component": np.ctypeslib.as_array(comp)[:n].copy(), "ncomponents": nc.value}


def cic_face_averages(hier, level, w, faces, phys=None, delta=None, stream=None):
    """amr_cic_face_averages: corrected normal face averages of the velocity ``w`` (list of dim
    device fields) on the interface faces of `level` into ``faces``; ``phys`` / ``delta``
    (device, one double per component) optional."""
    if len(w) != hier.dim:
        raise ValueError("cic_face_averages needs one field per dimension")
    _check(_lib.amr_cic_face_averages(hier.handle, int(level), _ptr_array(w), _ptr(phys), _ptr(faces), _ptr(delta),
                                      _stream(stream)), "amr_cic_face_averages")


def cic_component_box(hier, level, component):
    """amr_cic_component_box: (lo, hi, interface flags per face 2d+side) of a single-box
    component of `level`."""
    D = hier.dim
    lo, hi, fl = (C.c_int * D)(), (C.c_int * D)(), (C.c_int * (2 * D))()
    _check(_lib.amr_cic_component_box(hier.handle, int(level), int(component), lo, hi, fl), "amr_cic_component_box")
    return tuple(lo), tuple(hi), list(fl)


def cic_interface_bc(hier, level, component, x, bc, stream=None):
    """amr_cic_interface_bc: interface face averages of ``x`` into the boundary data ``bc`` of
    the component's one-level box problem."""
    _check(_lib.amr_cic_interface_bc(hier.handle, int(level), int(component), _ptr(x), _ptr(bc), _stream(stream)),
           "amr_cic_interface_bc")


def regrid(dim, n0, nlevels, tags, efficiency, min_width, ratio=2):
    """amr_regrid: new boxes per level ([[(lo, hi)], ...], level 0 the domain) from ``tags``
    (per level 0..nlevels-2: an (n, dim) integer array of tagged cells)."""
    n0a = (C.c_int * 3)(*(list(n0) + [1] * (3 - dim)))
    arrs = [np.ascontiguousarray(np.asarray(t, dtype=np.int32).reshape(-1, dim)) for t in tags]
    if len(arrs) != nlevels - 1:
        raise ValueError("regrid needs the tags of levels 0 .. nlevels-2")
    nt = (C.c_int * max(1, len(arrs)))(*[len(a) for a in arrs])
    ptrs = (_P(C.c_int) * max(1, len(arrs)))(*[a.ctypes.data_as(_P(C.c_int)) for a in arrs])
    p = RegridParams(float(efficiency), int(min_width))
    nl = C.c_int()
    nb = (C.c_int * nlevels)()
    _check(_lib.amr_regrid(dim, ratio, n0a, nlevels, nt, ptrs, C.byref(p), C.byref(nl), nb, None, 0), "amr_regrid")
    total = sum(nb[l] for l in range(nl.value))
    out = (C.c_int * (2 * dim * total))()
    _check(_lib.amr_regrid(dim, ratio, n0a, nlevels, nt, ptrs, C.byref(p), C.byref(nl), nb, out, total),
           "amr_regrid")
    flat = list(out)
    levels, q = [], 0
    for l in range(nl.value):
        bl = []
        for _ in range(nb[l]):
            bl.append((tuple(flat[q:q + dim]), tuple(flat[q + dim:q + 2 * dim])))
            q += 2 * dim
        levels.append(bl)
    return levels


def migrate(old_hier, old_x, new_hier, new_x, stream=None):
    """amr_migrate: old_x (composite field of old_hier) onto new_x (of new_hier)."""
    _check(_lib.amr_migrate(old_hier.handle, _ptr(old_x), new_hier.handle, _ptr(new_x), _stream(stream)),
           "amr_migrate")


def migrate_plan(old_hier, new_hier, level):
    """amr_migrate_plan of one new level as numpy arrays."""
    D = new_hier.dim
    nb, nc, ns = C.c_int(), C.c_longlong(), C.c_longlong()
    _check(_lib.amr_migrate_plan(old_hier.handle, new_hier.handle, int(level), C.byref(nb), None, C.byref(nc), None,
                                 None, None, None, C.byref(ns), None), "amr_migrate_plan")
    blocks = (C.c_int * max(1, nb.value * (2 + 2 * D)))()
    cells = (C.c_int * max(1, nc.value * D))()
    starts = (C.c_int * max(1, nc.value * D))()
    dst = (C.c_longlong * max(1, nc.value))()
    src = (C.c_longlong * max(1, nc.value))()
    side = (C.c_longlong * max(1, ns.value))()
    _check(_lib.amr_migrate_plan(old_hier.handle, new_hier.handle, int(level), None, blocks, None, cells, starts, dst,
                                 src, None, side), "amr_migrate_plan")
    n, m = nb.value, nc.value
    return {"blocks": np.ctypeslib.as_array(blocks)[:n * (2 + 2 * D)].reshape(n, 2 + 2 * D).copy(),
            "cells": np.ctypeslib.as_array(cells)[:m * D].reshape(m, D).copy(),
            "starts": np.ctypeslib.as_array(starts)[:m * D].reshape(m, D).copy(),
            "dst": np.ctypeslib.as_array(dst)[:m].copy(), "src": np.ctypeslib.as_array(src)[:m].copy(),
            "side": np.ctypeslib.as_array(side)[:ns.value].copy()}
