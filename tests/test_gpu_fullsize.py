"""Full-size parity in the benchmark's launch configuration.

At the workload sizes the oracle cannot follow hundreds of steps, so each test advances the GPU
state, downloads it, takes one more GPU step and compares every node with the oracle's step from
the same downloaded state; global invariants (per-component mass) are checked over the whole run."""
import numpy as np
import pytest

import oracle
from paper_2505_22256_gb300 import lbm, scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2505_22256_gb300 import build

    build.build()
    oracle.build()
    lbm.load_library()


def _compare_step(sc, before, after, tol):
    cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
    o = oracle.run(cfg, sc.solid, before, 1)
    scale = np.abs(o).max(axis=(2, 3), keepdims=True)
    err = float(np.max(np.abs(after - o) / scale))
    assert err <= tol, err
    return err


def test_sweep_1024_seven_cases_one_step_parity_and_mass():
    """The benchmark workload: seven 1024x1024 cylinder cases, FP32, default launch shape."""
    cases = S.lambda_sweep_cylinder(1024)
    lat = lbm.Lattice(cases, "f32")
    m0 = [lat.diagnostics(i) for i in range(len(cases))]
    lat.step(60)
    sample = (0, 3, 6)
    before = {i: lat.populations(i) for i in sample}
    lat.step(1)
    for i in sample:
        _compare_step(cases[i], before[i], lat.populations(i), 2e-6)
    for i in range(len(cases)):
        m1 = lat.diagnostics(i)
        for k in ("mass_A", "mass_B"):
            assert abs(m1[k] / m0[i][k] - 1) < 1e-5, (i, k)
    lat.close()


@pytest.mark.parametrize("workload", ["sweep", "couette"])
def test_autotuned_launch_shape_one_step_parity(workload):
    """The launch shape bench.py times is the one lbm_autotune(ctx, 4) picks on the live state (block
    width, wall-list form, row chunks); one more step in that shape matches the oracle's step from
    the same state, and mass is kept over the tuning steps."""
    cases = S.lambda_sweep_cylinder(1024) if workload == "sweep" else \
        [S.couette_channel(seed=7 + 100 * j) for j in range(512)]
    lat = lbm.Lattice(cases, "f32")
    m0 = lat.diagnostics(0)
    lbm.lbm_autotune(lat.ctx, 4)
    info = lat.info()
    assert info["block_threads"] in (64, 128) and info["wall_inline"] in (0, 1)
    lat.step(7)
    sample = (0, len(cases) // 2, len(cases) - 1)
    before = {i: lat.populations(i) for i in sample}
    lat.step(1)
    for i in sample:
        _compare_step(cases[i], before[i], lat.populations(i), 2e-6)
    m1 = lat.diagnostics(0)
    for k in ("mass_A", "mass_B"):
        assert abs(m1[k] / m0[k] - 1) < 1e-5, k
    lat.close()


def test_porous_4096x2048_open_boundaries_one_step_parity():
    sc = S.porous_disks()
    fl = sc.solid == 0
    lat = lbm.Lattice(sc, "f32")
    node = lat.wall_list()[0]
    # the synthetic medium has the stated porosity and wall-adjacent share
    assert abs(fl.mean() - 0.6) < 0.01
    assert len(node) >= 0.05 * fl.sum()
    lat.step(40)
    before = lat.populations()
    lat.step(1)
    _compare_step(sc, before, lat.populations(), 2e-6)
    lat.close()


def test_throat_2048x512_one_step_parity_f32_and_f16():
    sc = S.throat_channel()
    for storage, tol in (("f32", 2e-6), ("f16", 2e-3)):
        lat = lbm.Lattice(sc, storage)
        lat.step(30)
        before = lat.populations()
        lat.step(1)
        _compare_step(sc, before, lat.populations(), tol)
        lat.close()


def test_uneven_ensemble_and_cocurrent_channel():
    """256 uneven contact-angle cases plus the 4096x256 co-current channel in one context:
    sampled cases step exactly like the oracle from the same state."""
    cases = S.ensemble_cases(256) + [S.cocurrent_channel()]
    lat = lbm.Lattice(cases, "f32")
    info = lat.info()
    assert info["ncases"] == 257
    lat.step(20)
    sample = (0, 1, 100, 255, 256)
    before = {i: lat.populations(i) for i in sample}
    lat.step(1)
    for i in sample:
        _compare_step(cases[i], before[i], lat.populations(i), 2e-6)
    lat.close()
