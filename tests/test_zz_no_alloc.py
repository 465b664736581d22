"""The allocation-free mean-zero entry point (for callers that must not allocate device
memory during the call) against the regular one, through the C ABI.  Collected last so
that a run stopping at the first failure has run every other test before it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BOXES = [[((0, 0), (39, 23))], [((0, 8), (27, 39))], [((8, 24), (39, 55))]]


def test_noalloc_mean_zero_matches_regular_entry_point_twice():
    from paper_2506_02663_gb300 import amr
    gh = amr.Hierarchy(2, (40, 24), BOXES, h0=1.0 / 40)
    op = amr.Operator(gh, 0.0, 1.0, [1, 1, 1, 1])  # gives the hierarchy its device copy
    rng = np.random.default_rng(31)
    for call in range(2):  # two calls in a row share the fixed scratch array
        per = [[rng.standard_normal(tuple(hi[d] - lo[d] + 1 for d in range(2))) + 3.0 * (call + 1)
                for lo, hi in bl] for bl in BOXES]
        host = gh.pack(per)
        a = torch.from_numpy(host.copy()).cuda()
        b = torch.from_numpy(host.copy()).cuda()
        ma = amr.mean_zero(gh, a)
        mb = amr.mean_zero_noalloc(gh, b)
        assert abs(ma - mb) <= 1e-14 * abs(ma)
        ua, ub = gh.unpack(a.cpu().numpy()), gh.unpack(b.cpu().numpy())
        scale = max(float(np.max(np.abs(x))) for lev in ua for x in lev)
        for la, lb in zip(ua, ub):
            for xa, xb in zip(la, lb):
                assert np.max(np.abs(xa - xb)) <= 1e-13 * scale
    op.close()
    gh.close()
