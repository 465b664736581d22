"""AMR hierarchy of Sec. 5.1 (oracle; test infrastructure).

* Eq. (grids): level l has r^l * n0 cells per dimension, h^l = h^0 / r^l, C_r(i) = floor(i/r).
* Eq. (AMRHier): level 0 is the whole domain; level l > 0 is a set of pairwise disjoint
  boxes [lo, hi] (inclusive multi-indices in level-l index space).
* Eq. (pBlock): proper refinement, every box of level l > 0 is a union of whole children of
  coarse cells (lo and hi+1 divisible by r).
* Proper nesting (paragraph after Eq. pBlock): the paper asks for at least one cell of
  separation.  The fifth-order CF interpolation reads a 5-cell coarse window around the
  parent of a fine ghost cell, which reaches 3 coarse cells beyond C_r(box); the oracle
  therefore requires C_r(box) grown by 3 cells (clipped to the domain) to be covered by
  level l-1.  On level 1 this always holds because level 0 is the domain.
* Eq. (validRegion): the invalid region of level l is C_r of level l+1; valid = rest.
* Sec. 5.1, Fig. 1(b): connected components of the l-th subdomain; two boxes are adjacent
  when they share a face patch of positive measure.  Label = smallest box index.
* Fig. 1(c): ghost cells of a patch are filled by copying (same level), by AMRCFI, or by the
  physical formulas; per-patch ghost maps are produced for index-map parity.

Error codes (same numbering as the library's status enum):
  0 OK, 1 invalid argument, 2 nesting violated, 3 refinement violated, 4 box too small.
Checks run in this order and the first failure is reported: global parameters; then for
every level l >= 1 and every box in order: bounds, size (>= 4 cells per dimension),
alignment; then pairwise disjointness per level; then nesting for l >= 2; finally the
size of the coarsest multigrid grid of level 0.
"""
import itertools

import numpy as np

from .stencil import NG

OK, ERR_INVALID_ARG, ERR_NESTING, ERR_REFINEMENT, ERR_BOX_TOO_SMALL = 0, 1, 2, 3, 4
NESTING_MARGIN = 3
MIN_BOX = 4
MAX_BOTTOM_CELLS = 1024

# ghost-map codes (interface format shared with the library's index maps)
G_INTERIOR, G_PHYS, G_COPY, G_CFI, G_UNUSED = 0, 1, 2, 3, 4


class HierarchyError(Exception):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


def mg_grids(n0):
    """Per-dimension cell counts of the level-0 multigrid grids: halve while every
    dimension is even and the halved grid keeps at least 4 cells per dimension."""
    grids = [tuple(n0)]
    while all(n % 2 == 0 and n // 2 >= MIN_BOX for n in grids[-1]):
        grids.append(tuple(n // 2 for n in grids[-1]))
    return grids


def validate(dim, ratio, n0, boxes, bc, min_n0=5):
    """Return (code, message) for a hierarchy description (see module docstring).
    ``min_n0`` is 5 for AMR hierarchies (the CF window needs 5 coarse cells) and 4 for the
    single-box multigrid grids of level 0."""
    if dim not in (2, 3):
        return ERR_INVALID_ARG, "dim must be 2 or 3"
    if ratio not in (2, 4):
        return ERR_INVALID_ARG, "ratio must be 2 or 4"
    if len(n0) != dim or any(n < min_n0 for n in n0):
        return ERR_INVALID_ARG, f"n0 must have >= {min_n0} cells per dimension"
    if len(bc) != 2 * dim or any(b not in (0, 1) for b in bc):
        return ERR_INVALID_ARG, "bad bc"
    if len(boxes) < 1 or len(boxes[0]) != 1:
        return ERR_INVALID_ARG, "level 0 must be exactly one box"
    lo0, hi0 = boxes[0][0]
    if tuple(lo0) != (0,) * dim or tuple(hi0) != tuple(n - 1 for n in n0):
        return ERR_INVALID_ARG, "level 0 box must be the domain"
    for l in range(1, len(boxes)):
        if len(boxes[l]) < 1:
            return ERR_INVALID_ARG, "empty level"
        ndom = [n * ratio ** l for n in n0]
        for k, (lo, hi) in enumerate(boxes[l]):
            if any(lo[d] > hi[d] or lo[d] < 0 or hi[d] >= ndom[d] for d in range(dim)):
                return ERR_INVALID_ARG, f"box {k} of level {l} out of bounds"
            if any(hi[d] - lo[d] + 1 < MIN_BOX for d in range(dim)):
                return ERR_BOX_TOO_SMALL, f"box {k} of level {l} smaller than {MIN_BOX}"
            if any(lo[d] % ratio or (hi[d] + 1) % ratio for d in range(dim)):
                return ERR_REFINEMENT, f"box {k} of level {l} not properly refined"
    for l in range(1, len(boxes)):
        for (i, a), (j, b) in itertools.combinations(enumerate(boxes[l]), 2):
            if all(max(a[0][d], b[0][d]) <= min(a[1][d], b[1][d]) for d in range(dim)):
                return ERR_INVALID_ARG, f"boxes {i} and {j} of level {l} overlap"
    for l in range(2, len(boxes)):
        nc = [n * ratio ** (l - 1) for n in n0]
        cov = set()
        for lo, hi in boxes[l - 1]:
            for c in itertools.product(*[range(lo[d], hi[d] + 1) for d in range(dim)]):
                cov.add(c)
        for k, (lo, hi) in enumerate(boxes[l]):
            glo = [max(lo[d] // ratio - NESTING_MARGIN, 0) for d in range(dim)]
            ghi = [min(hi[d] // ratio + NESTING_MARGIN, nc[d] - 1) for d in range(dim)]
            for c in itertools.product(*[range(glo[d], ghi[d] + 1) for d in range(dim)]):
                if c not in cov:
                    return ERR_NESTING, f"box {k} of level {l} not properly nested"
    if int(np.prod(mg_grids(n0)[-1])) > MAX_BOTTOM_CELLS:
        return ERR_INVALID_ARG, "coarsest multigrid grid too large for the dense bottom solve"
    return OK, "ok"


class Level:
    """Geometry of one AMR level as seen by the oracle."""

    def __init__(self, l, dim, ratio, n0, h0, boxes):
        self.l = l
        self.D = dim
        self.ndom = tuple(n * ratio ** l for n in n0)
        self.h = h0 / ratio ** l
        self.boxes = [(tuple(lo), tuple(hi)) for lo, hi in boxes]
        blo = [min(b[0][d] for b in self.boxes) for d in range(dim)]
        bhi = [max(b[1][d] for b in self.boxes) for d in range(dim)]
        self.origin = tuple(v - NG for v in blo)
        self.shape = tuple(bhi[d] - blo[d] + 1 + 2 * NG for d in range(dim))
        self.covered = np.zeros(self.shape, bool)
        self.patch = np.full(self.shape, -1, np.int64)
        for k, (lo, hi) in enumerate(self.boxes):
            s = self.box_slice(lo, hi)
            self.covered[s] = True
            self.patch[s] = k
        self.valid = self.covered.copy()  # refined by Hierarchy
        self._classify_ghosts()

    def box_slice(self, lo, hi):
        return tuple(slice(lo[d] - self.origin[d], hi[d] + 1 - self.origin[d]) for d in range(self.D))

    def global_index(self, arr_idx):
        return tuple(arr_idx[d] + self.origin[d] for d in range(self.D))

    def inside_domain(self):
        """bool array: cell inside the physical domain."""
        m = np.ones(self.shape, bool)
        for d in range(self.D):
            g = np.arange(self.shape[d]) + self.origin[d]
            ok = (g >= 0) & (g < self.ndom[d])
            sh = [1] * self.D
            sh[d] = -1
            m &= ok.reshape(sh)
        return m

    def _classify_ghosts(self):
        """CF ghost cells of the level array: inside the domain, not covered, and within
        two cells of a covered cell along some axis (Fig. 1(c) bullets)."""
        reach = np.zeros(self.shape, bool)
        for d in range(self.D):
            for k in (1, 2):
                for s in (1, -1):
                    reach |= np.roll(self.covered, s * k, axis=d) & _no_wrap(self.shape, d, s * k)
        self.cf_ghost = reach & ~self.covered & self.inside_domain()


def _no_wrap(shape, d, k):
    m = np.ones(shape, bool)
    idx = [slice(None)] * len(shape)
    idx[d] = slice(0, k) if k > 0 else slice(shape[d] + k, shape[d])
    m[tuple(idx)] = False
    return m


class Hierarchy:
    """AMR hierarchy (Eq. AMRHier) with derived masks, component labels and index maps."""

    def __init__(self, dim, n0, boxes, bc, ratio=2, lo=None, hi=None, mg_grid=False):
        code, msg = validate(dim, ratio, tuple(n0), boxes, bc, min_n0=4 if mg_grid else 5)
        if code != OK:
            raise HierarchyError(code, msg)
        self.D = dim
        self.ratio = ratio
        self.n0 = tuple(n0)
        self.bc = list(bc)
        lo = lo if lo is not None else (0.0,) * dim
        hi = hi if hi is not None else (1.0,) * dim
        self.lo, self.hi = tuple(lo), tuple(hi)
        self.h0 = (hi[0] - lo[0]) / n0[0]
        self.levels = [Level(l, dim, ratio, self.n0, self.h0, boxes[l]) for l in range(len(boxes))]
        self.lmax = len(self.levels) - 1
        for l in range(self.lmax):
            self._mark_invalid(l)

    def _mark_invalid(self, l):
        """Eq. (validRegion): cells of level l under C_r(level l+1) are invalid."""
        lev, fine = self.levels[l], self.levels[l + 1]
        r = self.ratio
        for lo, hi in fine.boxes:
            clo = tuple(v // r for v in lo)
            chi = tuple(v // r for v in hi)
            lev.valid[lev.box_slice(clo, chi)] = False
        lev.invalid = lev.covered & ~lev.valid

    # ------------------------------------------------------------------ components
    def components(self, l):
        """Connected-component label of every box of level l (Sec. 5.1): union-find over
        face adjacency; label = smallest box index in the component."""
        boxes = self.levels[l].boxes
        parent = list(range(len(boxes)))

        def find(i):
            while parent[i] != i:
                i = parent[i]
            return i

        for i, j in itertools.combinations(range(len(boxes)), 2):
            if _face_adjacent(boxes[i], boxes[j], self.D):
                a, b = find(i), find(j)
                parent[max(a, b)] = min(a, b)
        return [find(i) for i in range(len(boxes))]

    # ------------------------------------------------------------------ index maps
    def ghost_map(self, l, k):
        """Per-patch ghost map of box k on level l over its padded extents (n+4 per dim).
        Returns (code, src_patch, src_cell) int arrays with axis d = dimension d:
        code in {G_INTERIOR, G_PHYS, G_COPY, G_CFI, G_UNUSED}; for G_PHYS src_patch holds
        the face id 2d+side and src_cell the ghost layer (1 or 2); for G_COPY the source
        box and the source cell's interior linear index (x fastest); else -1."""
        lev = self.levels[l]
        lo, hi = lev.boxes[k]
        D = self.D
        ext = tuple(hi[d] - lo[d] + 1 + 2 * NG for d in range(D))
        code = np.full(ext, G_UNUSED, np.int32)
        src_p = np.full(ext, -1, np.int32)
        src_c = np.full(ext, -1, np.int32)
        for a in np.ndindex(*ext):
            g = tuple(lo[d] - NG + a[d] for d in range(D))
            out = [d for d in range(D) if g[d] < lo[d] or g[d] > hi[d]]
            if not out:
                code[a] = G_INTERIOR
                continue
            if len(out) > 1:
                continue
            d = out[0]
            if g[d] < 0 or g[d] >= lev.ndom[d]:
                side = 0 if g[d] < 0 else 1
                code[a] = G_PHYS
                src_p[a] = 2 * d + side
                src_c[a] = (-g[d]) if side == 0 else (g[d] - lev.ndom[d] + 1)
                continue
            q = -1
            for j, (qlo, qhi) in enumerate(lev.boxes):
                if j != k and all(qlo[e] <= g[e] <= qhi[e] for e in range(D)):
                    q = j
                    break
            if q >= 0:
                qlo, qhi = lev.boxes[q]
                code[a] = G_COPY
                src_p[a] = q
                lin, stride = 0, 1
                for e in range(D):
                    lin += (g[e] - qlo[e]) * stride
                    stride *= qhi[e] - qlo[e] + 1
                src_c[a] = lin
            else:
                code[a] = G_CFI
        return code, src_p, src_c


def _face_adjacent(a, b, D):
    for d in range(D):
        touch = a[1][d] + 1 == b[0][d] or b[1][d] + 1 == a[0][d]
        if touch and all(max(a[0][e], b[0][e]) <= min(a[1][e], b[1][e]) for e in range(D) if e != d):
            return True
    return False


def index_maps(H):
    """Index maps in the library's canonical format (see the C header's amr_index_maps):
    valid per interior cell (patch order, x fastest), component per box, ghost maps per
    padded cell, AMRCFI ghost list, coarse cells with CF faces (COH-3)."""
    from .cfi import window_start
    D, r = H.D, H.ratio
    valid, comp, code, src, aux = [], [], [], [], []
    cfi_cell, cfi_start, cfi_pos, cfi_sub = [], [], [], []
    rcell, rfaces = [], []
    base = 0
    for l, lev in enumerate(H.levels):
        comp += H.components(l)
        for k, (lo, hi) in enumerate(lev.boxes):
            sub = lev.valid[lev.box_slice(lo, hi)]
            valid += [int(v) for v in sub.transpose().ravel()]  # x fastest
            c, s, a = H.ghost_map(l, k)
            c_x = c.transpose().ravel()
            code += [int(v) for v in c_x]
            src += [int(v) for v in s.transpose().ravel()]
            aux += [int(v) for v in a.transpose().ravel()]
            ext = c.shape
            for idx in np.nonzero(c_x == G_CFI)[0]:
                # padded index -> coordinates (x fastest)
                a_ = []
                rem = int(idx)
                for d in range(D):
                    a_.append(rem % ext[d])
                    rem //= ext[d]
                g = [lo[d] - NG + a_[d] for d in range(D)]
                crs = H.levels[l - 1]
                par = [g[d] // r for d in range(D)]
                st = [window_start(par[d], crs.ndom[d]) for d in range(D)]
                cfi_cell.append(base + int(idx))
                cfi_start.append(st)
                cfi_pos.append([par[d] - st[d] for d in range(D)])
                cfi_sub.append([g[d] - r * par[d] for d in range(D)])
            base += c.size
    for l in range(H.lmax):
        lev = H.levels[l]
        faces = {}
        for d in range(D):
            for s in (1, -1):
                nb = np.zeros(lev.shape, bool)
                src_, dst_ = [slice(None)] * D, [slice(None)] * D
                if s == 1:
                    dst_[d], src_[d] = slice(0, -1), slice(1, None)
                else:
                    dst_[d], src_[d] = slice(1, None), slice(0, -1)
                nb[tuple(dst_)] = lev.invalid[tuple(src_)]
                for cell in np.argwhere(lev.valid & nb):
                    key = tuple(int(v) for v in cell)
                    faces[key] = faces.get(key, 0) | (1 << (2 * d + (1 if s == 1 else 0)))
        for k, (lo, hi) in enumerate(lev.boxes):
            n = [hi[d] - lo[d] + 1 for d in range(D)]
            ents = []
            for key, f in faces.items():
                g = [key[d] + lev.origin[d] for d in range(D)]
                if all(lo[d] <= g[d] <= hi[d] for d in range(D)):
                    lin, stride = 0, 1
                    for d in range(D):
                        lin += (g[d] - lo[d]) * stride
                        stride *= n[d]
                    ents.append((lin, f))
            for lin, f in sorted(ents):
                rcell.append([l, k, lin])
                rfaces.append(f)
    return {
        "valid": np.asarray(valid, np.int32),
        "component": np.asarray(comp, np.int32),
        "ghost_code": np.asarray(code, np.int32),
        "ghost_src": np.asarray(src, np.int32),
        "ghost_aux": np.asarray(aux, np.int32),
        "cfi_cell": np.asarray(cfi_cell, np.int64),
        "cfi_start": np.asarray(cfi_start, np.int32).reshape(-1, D),
        "cfi_pos": np.asarray(cfi_pos, np.int32).reshape(-1, D),
        "cfi_sub": np.asarray(cfi_sub, np.int32).reshape(-1, D),
        "reflux_cell": np.asarray(rcell, np.int32).reshape(-1, 3),
        "reflux_faces": np.asarray(rfaces, np.int32),
    }
