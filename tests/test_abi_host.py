"""Host-side checks of the C-ABI library (no GPU): it loads, exports every function the
header declares, validates hierarchies with the same status codes as the oracle, and
produces index maps bit-identical to the oracle's (valid regions, components, ghost maps,
AMRCFI stencils, coarse-fine reflux faces)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def amr():
    from paper_2506_02663_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    from paper_2506_02663_gb300 import amr as m
    return m


def test_exports_every_declared_symbol(amr):
    hdr = open(os.path.join(ROOT, "include", "amr4.h")).read()
    declared = set(re.findall(r"^\s*(?:amr_status|void|const char\*|long long)\s+(amr_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 20
    import ctypes
    lib = ctypes.CDLL(amr.LIB)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared <= set(amr.EXPORTED)


CASES = [
    (2, (16, 16), [[((0, 0), (15, 15))], [((8, 8), (23, 23))]]),
    (2, (16, 16), [[((0, 0), (15, 15))], [((0, 12), (11, 31))]]),
    (2, (16, 16), [[((0, 0), (15, 15))], [((4, 4), (15, 19)), ((16, 4), (27, 19))], [((16, 16), (39, 27))]]),
    (2, (12, 20), [[((0, 0), (11, 19))], [((0, 0), (7, 7)), ((8, 0), (15, 7)), ((4, 8), (11, 15))]]),
    (3, (8, 8, 8), [[((0, 0, 0), (7, 7, 7))], [((4, 0, 6), (11, 7, 15))]]),
]


@pytest.mark.parametrize("dim,n0,boxes", CASES)
def test_index_maps_match_oracle(amr, dim, n0, boxes):
    from oracle.hierarchy import Hierarchy, index_maps
    H = Hierarchy(dim, n0, boxes, bc=[0] * (2 * dim))
    ref = index_maps(H)
    h = amr.Hierarchy(dim, n0, boxes)
    got = h.index_maps()
    for key in ref:
        assert got[key].shape == ref[key].shape, key
        assert np.array_equal(got[key], ref[key]), key


BAD = [
    [[((0, 0), (15, 15))], [((8, 8), (9, 23))]],
    [[((0, 0), (15, 15))], [((7, 8), (22, 23))]],
    [[((0, 0), (15, 15))], [((8, 8), (40, 23))]],
    [[((0, 0), (15, 15))], [((8, 8), (23, 23)), ((20, 20), (27, 27))]],
    [[((0, 0), (15, 15))], [((8, 8), (23, 23))], [((16, 16), (31, 31))]],
    [[((0, 0), (15, 15))], [((8, 8), (23, 23))], [((20, 22), (27, 25))]],
    [[((0, 0), (14, 15))]],
    [[((0, 0), (15, 15))], [((8, 8), (9, 23)), ((1, 1), (6, 6))]],
]


@pytest.mark.parametrize("boxes", BAD)
def test_validation_codes_match_oracle(amr, boxes):
    from oracle.hierarchy import validate
    code, _ = validate(2, 2, (16, 16), boxes, [0] * 4)
    assert code != 0
    with pytest.raises(amr.AmrError) as ei:
        amr.Hierarchy(2, (16, 16), boxes)
    assert ei.value.status == code


def test_layout_alignment_and_bc_layout(amr):
    h = amr.Hierarchy(2, (16, 16), CASES[2][2])
    for p in h.patches:
        assert p["offset"] % 32 == 0 and p["sy"] % 4 == 0
    offs = h.bc_offsets
    # level l face arrays have 16 * 2^l entries each, 4 faces per level
    assert offs[-1] == 4 * (16 + 32 + 64)
    rng = np.random.default_rng(0)
    per = [[rng.standard_normal(tuple(b[1][d] - b[0][d] + 1 for d in range(2))) for b in bl] for bl in CASES[2][2]]
    flat = h.pack(per)
    back = h.unpack(flat)
    for l in range(len(per)):
        for k in range(len(per[l])):
            assert np.array_equal(back[l][k], per[l][k])


def test_set_tile_rows_validates(amr):
    """The tile-shape control accepts 0 (autotuned), 1, 2 and 4 and rejects the rest on the
    host, without touching a GPU."""
    with pytest.raises(Exception):
        amr.set_tile_rows(3)
    amr.set_tile_rows(0)


def test_set_fx_residual_validates(amr):
    """The fixed-point residual switch accepts 0 and 1 and rejects the rest on the host."""
    with pytest.raises(Exception):
        amr.set_fx_residual(2)
    amr.set_fx_residual(0)
    amr.set_fx_residual(1)
