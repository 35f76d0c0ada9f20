"""The scheme comparison (Sec. 3.2) through the library, checked against the FP64 oracle on the
paper's 300x350 geometry: after 200 steps every record the study reports for a case equals the
same quantity computed from the oracle's state."""
import numpy as np
import pytest

import oracle
from paper_2505_22256_gb300 import lbm, scenarios as S
from paper_2505_22256_gb300 import study_schemes as st

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2505_22256_gb300 import build

    build.build()
    oracle.build()
    lbm.load_library()


def test_study_records_match_the_oracle():
    cases = S.scheme_study((30, 150))
    rows = st.run(cases, steps=200, check=100, storage="f64")
    assert [r["scheme"] for r in rows] == ["improved", "improved", "original", "original"]
    for sc, r in zip(cases, rows):
        cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
        f = oracle.run(cfg, sc.solid, oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0), 200)
        rA, rB, ux, uy = oracle.fields(cfg, sc.solid, f)
        d = oracle.diagnostics(cfg, sc.solid, f)
        th, _, _ = oracle.contact_angle(cfg, sc.solid, f, sc.surface)
        layer, share = st.wall_layer(sc.solid, rA, rB)
        assert r["theta"] == pytest.approx(th, abs=1e-6), sc.name
        assert r["umax"] == pytest.approx(d["umax"], rel=1e-8), sc.name
        far = ~st.near_solid(sc.solid)
        assert r["umax_off_wall"] == pytest.approx(float(np.max(np.hypot(ux, uy)[far])), rel=1e-8)
        assert r["umax_off_wall"] <= r["umax"] * (1 + 1e-12)
        assert r["rho_min"] == pytest.approx(min(d["rhoA_min"], d["rhoB_min"]), rel=1e-10)
        assert r["rho_max"] == pytest.approx(max(d["rhoA_max"], d["rhoB_max"]), rel=1e-10)
        assert r["wall_layer_rhoA"] == pytest.approx(layer, rel=1e-9)
        assert r["attached"] == (share > 0) and r["attached"]
        assert not r["unstable"]
        assert np.isfinite(r["du_last"]) and np.isfinite(r["dtheta_last"])
    table = st.table(rows)
    assert table.count("\n") == 1 + len(rows)


def test_cocurrent_records_match_the_oracle():
    """Two intervals of 500 steps of the Sec. 3.1 channels (Poiseuille and Couette, one angle):
    the profile errors and extrema the study reports equal those of the oracle's state."""
    from paper_2505_22256_gb300 import study_cocurrent as cc

    cs = cc.cases((45,))
    rows = cc.run(cs, max_steps=1000, storage="f64", interval=500)
    for sc, r in zip(cs, rows):
        cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
        f = oracle.run(cfg, sc.solid, oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0), 1000)
        rA, rB, ux, _ = oracle.fields(cfg, sc.solid, f)
        u = ux.mean(axis=1)
        rho = (rA + rB).mean(axis=1)
        assert r["steps"] == 1000 and r["converged_at"] is None  # far from steady after 1,000 steps
        assert r["eps_analytic"] == pytest.approx(cc.rel_l2(u, cc.analytic_profile(sc)), rel=1e-8), sc.name
        assert r["eps_balance"] == pytest.approx(cc.rel_l2(u, cc.balance_profile(sc, rho)), rel=1e-8), sc.name
        assert r["u_peak"] == pytest.approx(float(np.max(np.abs(u))), rel=1e-9)
        assert r["rho_min"] == pytest.approx(float(rho.min()), rel=1e-12)
        assert not r["unstable"]
    assert cc.table(rows).count("\n") == 1 + len(rows)


def test_obstacle_records_match_the_oracle():
    """The square-obstacle case under both schemes, 150 and 300 steps: region counts, areas and
    wall-layer medians equal those of the oracle's state."""
    from paper_2505_22256_gb300 import study_obstacle as so

    cs = so.cases()
    rows = so.run(cs, (150, 300), storage="f64")
    assert len(rows) == 4
    for sc in cs:
        cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
        f = oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
        for t0, t in ((0, 150), (150, 300)):
            f = oracle.run(cfg, sc.solid, f, t - t0)
            rA, rB, _, _ = oracle.fields(cfg, sc.solid, f)
            want = so.snapshot(sc, rA, rB)
            got = [r for r in rows if r["case"] == sc.name and r["step"] == t][0]
            for k in ("regions", "wall_regions", "obstacle_regions", "largest_area", "total_area"):
                assert got[k] == want[k], (sc.name, t, k)
            for k in ("obstacle_layer_rhoA", "wall_layer_rhoA"):
                assert got[k] == pytest.approx(want[k], rel=1e-9), (sc.name, t, k)
            assert got["umax"] == pytest.approx(oracle.diagnostics(cfg, sc.solid, f)["umax"], rel=1e-8)
    assert so.table(rows).count("\n") == 1 + len(rows)


def test_sphere3d_records_match_the_oracle():
    """The 3-D sphere case scaled to 24 x 24 x 34, two intervals of 100 steps: the angle after each
    interval and the diagnostics equal those of the oracle's state."""
    from oracle import d3
    from paper_2505_22256_gb300 import study_sphere3d as s3

    d3.build()
    rows = s3.run((0.38, 2.1), steps=200, interval=100, storage="f64", n=24)
    for lam, r in zip((0.38, 2.1), rows):
        sc = s3.case(lam, 24)
        p = sc.params()
        nz, ny, nx = sc.solid.shape
        cfg = d3.Config3(nx, ny, nz, scheme=p["scheme"], tau=p["tau"], G=p["G"], lam=p["lam"], Gw2=p["Gw2"],
                         delta=p["delta"], g=p["g"], second_layer=p["second_layer"])
        f = d3.init3(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
        for k in range(2):
            f = d3.run3(cfg, sc.solid, f, 100)
            th, _, _ = d3.contact_angle_sphere(cfg, sc.solid, f, sc.sphere)
            assert r["history"][k] == pytest.approx(th, abs=1e-6), (lam, k)
        od = d3.diagnostics3(cfg, sc.solid, f)
        for key in ("umax", "rhoA_min", "rhoA_max", "rhoB_min", "rhoB_max"):
            assert r[key] == pytest.approx(od[key], rel=1e-9), (lam, key)
        assert r["theta"] == r["history"][-1] and not r["unstable"]
    assert s3.table(rows).count("\n") == 1 + len(rows)


def test_sweep_records_match_the_oracle():
    """The steady-state sweep driver on the scaled cylinder case (96 x 96, two angles, 200 FP64
    steps): the angles after each interval, max |u| and the mass drift equal the oracle's."""
    from paper_2505_22256_gb300 import study_sweep as sw

    rows = sw.run(steps=200, check=100, storage="f64", n=96, angles=(30, 150))
    cases = S.lambda_sweep_cylinder(n=96, seed=2, angles=(30, 150))
    for sc, r in zip(cases, rows):
        cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
        f0 = oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
        m0 = f0.reshape(2, -1).sum(axis=1)
        f = f0
        for k in range(2):
            f = oracle.run(cfg, sc.solid, f, 100)
            th, _, _ = oracle.contact_angle(cfg, sc.solid, f, sc.surface)
            assert r["theta_history"][k][1] == pytest.approx(th, abs=1e-6), (sc.name, k)
        d = oracle.diagnostics(cfg, sc.solid, f)
        assert r["umax"] == pytest.approx(d["umax"], rel=1e-8)
        m1 = f.reshape(2, -1).sum(axis=1)
        assert r["mass_drift_A"] == pytest.approx(m1[0] / m0[0] - 1, abs=1e-12)
        assert r["mass_drift_B"] == pytest.approx(m1[1] / m0[1] - 1, abs=1e-12)
        assert r["dtheta_last"] == pytest.approx(abs(r["theta_history"][1][1] - r["theta_history"][0][1]))
    assert sw.table(rows).count("\n") == 1 + len(cases)


def test_displacement_records_match_the_oracle():
    """The porous displacement driver on a 256 x 128 medium, two intervals of 150 FP64 steps: mass,
    saturation and front equal those of the oracle's state."""
    from paper_2505_22256_gb300 import study_displacement as sd

    sc = sd.case(256, 128)
    rows = sd.run(sc, steps=300, check=150, storage="f64")
    cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
    f = oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
    for k, r in enumerate(rows):
        f = oracle.run(cfg, sc.solid, f, 150)
        rA, rB, _, _ = oracle.fields(cfg, sc.solid, f)
        d = oracle.diagnostics(cfg, sc.solid, f)
        want = sd.snapshot(sc, rA, rB)
        assert r["step"] == 150 * (k + 1)
        assert r["mass_A"] == pytest.approx(d["mass_A"], rel=1e-10)
        assert r["mass_B"] == pytest.approx(d["mass_B"], rel=1e-10)
        assert r["saturation_A"] == want["saturation_A"] and r["front_x"] == want["front_x"]
        assert r["inflow_A_per_step"] == pytest.approx(1.0 * 0.005 * int((sc.solid[:, 0] == 0).sum()))
        assert not r["unstable"]
    assert sd.table(rows).count("\n") == 3 + len(rows)
