"""The allocation-free mean-zero entry point, for callers that must not allocate device
memory during the call (device memory held by another allocator's pool, or a
latency-critical loop where cudaMalloc's implicit synchronisation is not acceptable),
against the regular entry point through the C ABI.  Both launch the same kernels with the
same launch shapes, so the results must agree bitwise; the oracle's mean-zero confirms the
value.  Collected last so that a run stopping at the first failure has run every other
test before it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import solve as so  # noqa: E402
from oracle.hierarchy import Hierarchy as OH  # noqa: E402

from _gpu_helpers import from_packed, max_abs, max_diff, to_packed  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    # 2-D, three levels, ragged base
    "2d_three_level": (2, (40, 24), [[((0, 0), (39, 23))], [((0, 8), (27, 39))], [((8, 24), (39, 55))]]),
    # 3-D, two levels (the z-chunked layout's tile multiples on the base)
    "3d_two_level": (3, (32, 32, 16), [[((0, 0, 0), (31, 31, 15))], [((8, 16, 4), (39, 47, 19))]]),
}


def _amr():
    from paper_2506_02663_gb300 import amr
    return amr


def _field(H, rng, shift):
    U = so.Unknowns(H)
    return U.scatter(rng.standard_normal(U.n) + shift)


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_mean_zero_matches_regular_entry_point_twice(name):
    amr = _amr()
    dim, n0, boxes = CASES[name]
    hi = tuple(n0[d] / n0[0] for d in range(dim))
    H = OH(dim, n0, boxes, bc=[1] * (2 * dim), hi=hi)
    gh = amr.Hierarchy(dim, n0, boxes, h0=1.0 / n0[0])
    op = amr.Operator(gh, 0.0, 1.0, [1] * (2 * dim))  # gives the hierarchy its device copy
    rng = np.random.default_rng(31)
    for call in range(2):  # two calls in a row share the fixed scratch array
        F = _field(H, rng, 3.0 * (call + 1))
        host = to_packed(gh, H, F)
        a = torch.from_numpy(host.copy()).cuda()
        b = torch.from_numpy(host.copy()).cuda()
        ma = amr.mean_zero(gh, a)
        mb = amr.mean_zero_noalloc(gh, b)
        assert ma == mb, (call, ma, mb)
        assert torch.equal(a, b), call
        ref, mref = so.mean_zero(H, F)
        assert abs(mb - mref) <= 1e-14 * abs(mref), (call, mb, mref)
        got = from_packed(gh, H, b.cpu().numpy())
        assert max_diff(H, got, ref, "covered") <= 1e-14 * max_abs(H, F), call
    op.close()
    gh.close()


def test_noalloc_mean_zero_needs_the_device_copy():
    amr = _amr()
    gh = amr.Hierarchy(2, (16, 16), [[((0, 0), (15, 15))]])  # no device call on it yet
    x = torch.ones(gh.nelems, dtype=torch.float64, device="cuda")
    with pytest.raises(amr.AmrError) as ei:
        amr.mean_zero_noalloc(gh, x)
    assert ei.value.status == amr.AMR_ERR_INVALID_ARG
    assert bool(torch.all(x == 1.0))
    gh.close()


def _deep_hierarchy():
    """2-D, 21 levels: levels 4..20 each one centred box of 368^2 cells, so that each needs
    512 reduction blocks and the hierarchy 8,910 in all (more than the 8192 the fixed
    scratch holds).  Every level nests in the one below with the margin of 3 coarse cells."""
    n0 = 32
    half = [None, 30, 52, 96] + [184] * 17
    boxes = [[((0, 0), (n0 - 1, n0 - 1))]]
    for l in range(1, 21):
        c = (n0 << l) // 2
        boxes.append([((c - half[l], c - half[l]), (c + half[l] - 1, c + half[l] - 1))])
    return n0, boxes


def test_noalloc_mean_zero_rejects_hierarchies_beyond_the_fixed_scratch():
    amr = _amr()
    n0, boxes = _deep_hierarchy()
    gh = amr.Hierarchy(2, (n0, n0), boxes)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    x = torch.randn(gh.nelems, dtype=torch.float64, device="cuda", generator=g)
    keep = x.clone()
    # the regular entry point has the same limit; it also gives the hierarchy its device copy
    with pytest.raises(amr.AmrError) as ei:
        amr.mean_zero(gh, x)
    assert ei.value.status == amr.AMR_ERR_INVALID_ARG
    assert torch.equal(x, keep)  # rejected before any launch
    with pytest.raises(amr.AmrError) as ei:
        amr.mean_zero_noalloc(gh, x)
    assert ei.value.status == amr.AMR_ERR_INVALID_ARG
    assert "8910" in str(ei.value)
    assert torch.equal(x, keep)
    gh.close()
