"""Host-side checks of the interface-face lists behind the interface-condition calls (no GPU):
amr_cic_faces lists exactly the oracle's coarse-fine interface faces of each refined level
(interior cell, normal and side) with the oracle's connected-component numbering, grouped by
component, and rejects level 0."""
import os

import numpy as np
import pytest

CASES = {
    "two_level": (2, (16, 16), [[((0, 0), (15, 15))], [((8, 8), (23, 23))]]),
    "boundary_box": (2, (16, 16), [[((0, 0), (15, 15))], [((0, 12), (11, 31))]]),
    "three_level_multibox": (2, (16, 16), [[((0, 0), (15, 15))], [((4, 4), (15, 19)), ((16, 4), (27, 19))],
                                           [((16, 16), (39, 27))]]),
    # level 1: two disjoint components (boxes 0 and 2 touch, box 1 stands alone)
    "two_components": (2, (32, 32), [[((0, 0), (31, 31))],
                                     [((8, 8), (19, 19)), ((40, 36), (55, 51)), ((20, 8), (27, 15))]]),
    "full_domain_level": (2, (16, 16), [[((0, 0), (15, 15))], [((0, 0), (31, 31))]]),
    "three_d": (3, (8, 8, 8), [[((0, 0, 0), (7, 7, 7))], [((4, 0, 6), (11, 7, 15))]]),
    "three_d_two_components": (3, (12, 12, 12), [[((0, 0, 0), (11, 11, 11))],
                                                 [((2, 2, 2), (7, 7, 7)), ((14, 14, 12), (21, 21, 19))]]),
}


@pytest.fixture(scope="module")
def amr():
    from paper_2506_02663_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    from paper_2506_02663_gb300 import amr as m
    return m


@pytest.mark.parametrize("name", list(CASES))
def test_interface_faces_match_oracle(amr, name):
    from oracle import cic
    from oracle.hierarchy import Hierarchy
    dim, n0, boxes = CASES[name]
    H = Hierarchy(dim, n0, boxes, bc=[0] * (2 * dim))
    h = amr.Hierarchy(dim, n0, boxes)
    for l in range(1, len(boxes)):
        got = amr.cic_faces(h, l)
        lev = H.levels[l]
        ref = cic.interface_faces(H, l)
        want = sorted((tuple(int(c[e] + lev.origin[e]) for e in range(dim)), 2 * d + (1 if s > 0 else 0), comp)
                      for c, d, s, comp in ref)
        have = sorted((tuple(int(v) for v in got["cell"][i]), int(got["face"][i]), int(got["component"][i]))
                      for i in range(len(got["face"])))
        assert have == want
        assert got["ncomponents"] == len(set(H.components(l)))
        # grouped by component, ascending
        assert np.all(np.diff(got["component"]) >= 0)
        if name == "two_components" and l == 1:
            assert got["ncomponents"] == 2 and set(got["component"]) == {0, 1}
        if name == "full_domain_level":
            assert len(got["face"]) == 0


def test_interface_faces_reject_level_zero(amr):
    dim, n0, boxes = CASES["two_level"]
    h = amr.Hierarchy(dim, n0, boxes)
    with pytest.raises(amr.AmrError):
        amr.cic_faces(h, 0)
    with pytest.raises(amr.AmrError):
        amr.cic_faces(h, 2)


@pytest.mark.parametrize("name", list(CASES))
def test_component_boxes_match_oracle(amr, name):
    """amr_cic_component_box gives the oracle's box and interface flags for every single-box
    component and rejects components of several boxes."""
    from oracle import cic
    from oracle.hierarchy import Hierarchy
    dim, n0, boxes = CASES[name]
    H = Hierarchy(dim, n0, boxes, bc=[0] * (2 * dim))
    h = amr.Hierarchy(dim, n0, boxes)
    for l in range(1, len(boxes)):
        nc = amr.cic_faces(h, l)["ncomponents"]
        for c in range(nc):
            try:
                want = cic.component_box(H, l, c)
            except ValueError:
                with pytest.raises(amr.AmrError):
                    amr.cic_component_box(h, l, c)
                continue
            lo, hi, fl = amr.cic_component_box(h, l, c)
            assert (lo, hi, fl) == (tuple(want[0]), tuple(want[1]), want[2])
        with pytest.raises(amr.AmrError):
            amr.cic_component_box(h, l, nc)
