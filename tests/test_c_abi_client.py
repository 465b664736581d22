"""The C ABI from plain C (no GPU): tests/c_abi_client.c is compiled with the system C
compiler against include/amr4.h, linked with the library, and its output (field layout,
interface faces, regridded boxes) must equal the Python binding's results."""
import os
import shutil
import subprocess

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


def test_c_client_matches_binding(amr, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = amr.LIB
    exe = tmp_path / "client"
    cmd = [cc, "-std=c99", "-O1", "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_client.c"),
           "-o", str(exe), lib, f"-Wl,-rpath,{os.path.dirname(lib)}", "-lstdc++", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stderr
    lines = run.stdout.strip().splitlines()

    boxes = [[((0, 0), (31, 31))], [((8, 8), (23, 27)), ((40, 36), (55, 51))]]
    h = amr.Hierarchy(2, (32, 32), boxes)
    assert lines[0] == f"layout {len(h.patches)} {h.nelems}"
    for p, line in zip(h.patches, lines[1:1 + len(h.patches)]):
        assert line == f"patch {p['level']} {p['box']} {p['offset']} {p['sy']} {p['nelems']}"
    info = amr.cic_faces(h, 1)
    s = int(np.sum(info["cell"][:, 0] * 7 + info["cell"][:, 1] * 13 + info["face"] * 3 + info["component"]))
    assert lines[1 + len(h.patches)] == f"faces {len(info['face'])} {info['ncomponents']} {s}"
    x, y = np.meshgrid(np.arange(4, 14), np.arange(10, 16), indexing="xy")
    tags = np.stack([x.ravel(), y.ravel()], axis=1)
    new = amr.regrid(2, (32, 32), 2, [tags], 0.8, 2)
    flat = [v for level in new for lo, hi in level for v in (*lo, *hi)]
    assert lines[-1] == "regrid " + " ".join(str(v) for v in [len(new)] + flat)
