"""The step kernel's own indexing, checked on the GPU (compute-sanitizer is not available here).

The LBM_BOUNDS_CHECK build tests every shared- and global-memory index of the step kernel before
use: the pull columns in the row slots, the density ring, the wall-list data, the field outputs and
the population stores, ghost copies included. An index outside its buffer sets bit 4 of the
context's error word, skips the access, and is reported by the next synchronising call. The
lattices below exercise the kernel's edges: partial windows, periodic wrap, walls, open inlet and
outflow columns, sliding walls, both block widths, 16-bit storage and the fields pass. No index may
trip, and every state must equal the normal build's bit for bit.
"""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUNNER = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2505_22256_gb300 import lbm, scenarios as S
lbm.load_library(sys.argv[2])


def pillar():  # an 8x8 periodic box around a single solid node
    solid = np.zeros((8, 8), np.uint8)
    solid[3, 3] = 1
    r = np.where(solid == 1, 0.0, 0.6)
    return S.Scenario("pillar8", solid, r, r * 0.5, bc_x="periodic", bc_y="periodic", lam=0.5)


cases = {
    "ragged131x77": (lambda: S.cylinder_droplet(77, nx=131, R=12, r=15, lam=1.4), "f32", 128),
    "ragged131x77_w64": (lambda: S.cylinder_droplet(77, nx=131, R=12, r=15, lam=1.4), "f32", 64),
    "porous_open": (lambda: S.porous_disks(nx=192, ny=96, rmin=5, rmax=11, keep_out=(12, 12), seed=9, porosity=0.7),
                    "f32", 128),
    "couette_sliding": (lambda: S.couette_channel(nx=40, ny=48, U=0.01), "f32", 64),
    "pillar8_f16": (lambda: pillar(), "f16", 128),
    "throat_f16": (lambda: S.throat_channel(256, 96, R=34, r=22, g=1e-5), "f16", 128),
}
out = {}
for name, (make, storage, width) in cases.items():
    lat = lbm.Lattice(make(), storage)
    lbm.lbm_set_launch(lat.ctx, width, 16)
    lat.step(29)
    rA, rB, ux, uy = lat.fields()          # the fields pass
    d = lat.diagnostics()                  # synchronises and reports the device error word
    f = lat.populations()
    lat.close()
    out[name] = {"f": f.tolist(), "rA": rA.tolist(), "umax": d["umax"]}
json.dump(out, open(sys.argv[3], "w"))
"""


def _run(lib, path):
    r = subprocess.run([sys.executable, "-c", RUNNER, ROOT, lib, path], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.load(open(path))


def test_checked_build_finds_no_index_outside_its_buffer():
    from paper_2505_22256_gb300 import build

    normal = build.build()
    checked = build.build(out_dir=os.path.join(os.path.dirname(build.LIB), "checked"),
                          defines={"LBM_BOUNDS_CHECK": 1})
    with tempfile.TemporaryDirectory() as d:
        a = _run(normal, os.path.join(d, "normal.json"))
        b = _run(checked, os.path.join(d, "checked.json"))
    assert a.keys() == b.keys()
    for name in a:
        np.testing.assert_array_equal(np.array(b[name]["f"]), np.array(a[name]["f"]), err_msg=name)
        np.testing.assert_array_equal(np.array(b[name]["rA"]), np.array(a[name]["rA"]), err_msg=name)
        assert b[name]["umax"] == a[name]["umax"], name
