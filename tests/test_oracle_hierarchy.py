"""Hierarchy pins (Sec. 5.1): validation codes, valid/invalid regions, connected
components and per-patch ghost maps on hand-checked small cases (no GPU)."""
import numpy as np
import pytest

from oracle import hierarchy as hy

D0 = [((0, 0), (15, 15))]


@pytest.mark.parametrize("boxes,code", [
    ([D0, [((8, 8), (23, 23))]], hy.OK),
    ([D0, [((8, 8), (9, 23))]], hy.ERR_BOX_TOO_SMALL),          # 2 cells wide
    ([D0, [((7, 8), (22, 23))]], hy.ERR_REFINEMENT),            # lo not divisible by r
    ([D0, [((8, 8), (22, 23))]], hy.ERR_REFINEMENT),            # hi+1 not divisible by r
    ([D0, [((8, 8), (40, 23))]], hy.ERR_INVALID_ARG),           # outside the domain
    ([D0, [((8, 8), (23, 23)), ((20, 20), (27, 27))]], hy.ERR_INVALID_ARG),  # overlap
    ([D0, [((8, 8), (23, 23))], [((16, 16), (31, 31))]], hy.ERR_NESTING),    # margin < 3
    ([D0, [((8, 8), (23, 23))], [((22, 22), (25, 25))]], hy.OK),             # margin 3
    ([D0, [((8, 8), (23, 23))], [((20, 22), (27, 25))]], hy.ERR_NESTING),    # margin 2 in x
    ([[((0, 0), (14, 15))]], hy.ERR_INVALID_ARG),               # level 0 not the domain
])
def test_validation_codes(boxes, code):
    got, _ = hy.validate(2, 2, (16, 16), boxes, [0] * 4)
    assert got == code


def test_validation_order_and_globals():
    assert hy.validate(4, 2, (16, 16), [D0], [0] * 4)[0] == hy.ERR_INVALID_ARG
    assert hy.validate(2, 3, (16, 16), [D0], [0] * 4)[0] == hy.ERR_INVALID_ARG
    assert hy.validate(2, 2, (4, 4), [[((0, 0), (3, 3))]], [0] * 4)[0] == hy.ERR_INVALID_ARG
    # a too-small box is reported before a misaligned later box
    got, _ = hy.validate(2, 2, (16, 16), [D0, [((8, 8), (9, 23)), ((1, 1), (6, 6))]], [0] * 4)
    assert got == hy.ERR_BOX_TOO_SMALL
    # coarsest multigrid grid too large (prime size never coarsens)
    assert hy.validate(2, 2, (67, 67), [[((0, 0), (66, 66))]], [0] * 4)[0] == hy.ERR_INVALID_ARG


def test_valid_region_counts():
    H = hy.Hierarchy(2, (16, 16), [D0, [((8, 8), (23, 23))], [((22, 22), (25, 25))]], [0] * 4)
    assert H.levels[0].valid.sum() == 256 - 64
    assert H.levels[1].valid.sum() == 256 - 4
    assert H.levels[2].valid.sum() == 16
    assert H.levels[1].invalid.sum() == 4


def test_components():
    boxes = [D0, [((4, 4), (7, 7)), ((8, 4), (11, 7)), ((20, 20), (23, 23)), ((8, 8), (11, 11)),
                  ((24, 24), (27, 27))]]
    H = hy.Hierarchy(2, (16, 16), boxes, [0] * 4)
    # boxes 0-1 share a face, 1-3 share a face; 2 and 4 touch only at a corner
    assert H.components(1) == [0, 0, 2, 0, 4]
    assert H.components(0) == [0]


def test_ghost_map_two_boxes():
    H = hy.Hierarchy(2, (16, 16), [D0, [((0, 8), (7, 15)), ((8, 8), (15, 15))]], [0] * 4)
    code, sp, sc = H.ghost_map(1, 0)
    assert code.shape == (12, 12)
    # x-low side of box 0 is the physical boundary (global x = -1, -2)
    assert (code[0:2, 2:10] == hy.G_PHYS).all()
    assert sp[1, 5] == 0 and sc[1, 5] == 1 and sc[0, 5] == 2
    # x-high side is box 1 (copy); source cell of global (8, 8+j) is x=0, y=j in box 1
    assert (code[10:12, 2:10] == hy.G_COPY).all()
    assert sp[10, 2] == 1 and sc[10, 2] == 0 and sc[11, 3] == 1 + 8
    # y sides are CF interfaces
    assert (code[2:10, 0:2] == hy.G_CFI).all() and (code[2:10, 10:12] == hy.G_CFI).all()
    # corners unused, interior interior
    assert (code[0:2, 0:2] == hy.G_UNUSED).all()
    assert (code[2:10, 2:10] == hy.G_INTERIOR).all()


def test_mg_grids():
    assert hy.mg_grids((256, 256))[-1] == (4, 4)
    assert hy.mg_grids((96, 96))[-1] == (6, 6)
    assert len(hy.mg_grids((64, 64))) == 5
