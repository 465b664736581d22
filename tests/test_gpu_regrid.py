"""GPU parity of the data migration after regridding (Sec. 5.4, last paragraph) through the C
ABI against the oracle's migration (oracle/regrid.py): random old fields and quartic cell
averages (which the migration reproduces exactly on the new hierarchy), within 1e-13 of the
field's scale (two chained 5^D-term AMRCFI sums in different orders on the two sides)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import regrid as orr, solve as so  # noqa: E402
from oracle.hierarchy import Hierarchy as OH  # noqa: E402

from _gpu_helpers import from_packed, to_packed  # noqa: E402
from test_migrate_host import PAIRS, _quartic_field  # noqa: E402

pytestmark = pytest.mark.gpu


def _amr():
    from paper_2506_02663_gb300 import amr
    return amr


@pytest.mark.parametrize("name", list(PAIRS))
@pytest.mark.parametrize("kind", ["random", "quartic"])
def test_migration_matches_oracle(name, kind):
    amr = _amr()
    dim, n0, bo, bn = PAIRS[name]
    hi = tuple(n0[d] / n0[0] for d in range(dim))
    Ho, Hn = OH(dim, n0, bo, bc=[0] * (2 * dim), hi=hi), OH(dim, n0, bn, bc=[0] * (2 * dim), hi=hi)
    go = amr.Hierarchy(dim, n0, bo, h0=1.0 / n0[0])
    gn = amr.Hierarchy(dim, n0, bn, h0=1.0 / n0[0])
    if kind == "random":
        U = so.Unknowns(Ho)
        Fo = U.scatter(np.random.default_rng(3).standard_normal(U.n), fill_invalid=True)
    else:
        Fo = _quartic_field(Ho)
    xo = torch.from_numpy(to_packed(go, Ho, Fo)).cuda()
    xn = torch.full((gn.nelems,), np.nan, dtype=torch.float64, device="cuda")
    amr.migrate(go, xo, gn, xn)
    torch.cuda.synchronize()
    got = from_packed(gn, Hn, xn.cpu().numpy())
    ref = orr.migrate(Ho, Fo, Hn)
    scale = max(float(np.max(np.abs(F[lev.covered]))) for F, lev in zip(ref, Hn.levels))
    for l, lev in enumerate(Hn.levels):
        assert np.max(np.abs(got[l][lev.covered] - ref[l][lev.covered])) <= 1e-13 * scale, l
    if kind == "quartic":
        exact = _quartic_field(Hn)
        for l, lev in enumerate(Hn.levels):
            assert np.max(np.abs(got[l][lev.covered] - exact[l][lev.covered])) <= 1e-12


def test_migration_rejects_mismatched_hierarchies():
    amr = _amr()
    go = amr.Hierarchy(2, (16, 16), [[((0, 0), (15, 15))]])
    gn = amr.Hierarchy(2, (24, 24), [[((0, 0), (23, 23))]])
    xo = torch.zeros(go.nelems, dtype=torch.float64, device="cuda")
    xn = torch.zeros(gn.nelems, dtype=torch.float64, device="cuda")
    with pytest.raises(amr.AmrError):
        amr.migrate(go, xo, gn, xn)
