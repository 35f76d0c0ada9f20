"""Host side of the scheme comparison (Sec. 3.2): the paper-geometry case list and the wall-layer
statistics the study computes from the library's fields.  No GPU."""
import numpy as np
import pytest

from paper_2505_22256_gb300 import scenarios as S
from paper_2505_22256_gb300 import study_schemes as st


def test_first_layer_of_a_single_solid_node_is_its_eight_neighbours():
    solid = np.zeros((8, 8), np.uint8)
    solid[3, 5] = 1
    m = st.first_layer(solid)
    want = {(3 + dy, 5 + dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)} - {(3, 5)}
    assert {tuple(p) for p in np.argwhere(m)} == want


def test_first_layer_wraps_periodically_and_surrounds_a_block():
    solid = np.zeros((8, 8), np.uint8)
    solid[0, 0] = 1
    got = {tuple(p) for p in np.argwhere(st.first_layer(solid))}
    assert got == {(0, 1), (1, 0), (1, 1), (0, 7), (7, 0), (7, 7), (1, 7), (7, 1)}
    solid = np.zeros((9, 9), np.uint8)
    solid[3:6, 3:6] = 1
    assert st.first_layer(solid).sum() == 5 * 5 - 3 * 3  # the ring around a 3x3 block


def test_near_solid_is_a_periodic_square_neighbourhood():
    solid = np.zeros((12, 12), np.uint8)
    solid[0, 0] = 1
    m = st.near_solid(solid, 3)
    assert m.sum() == 7 * 7
    assert m[3, 3] and m[-3, -3] and not m[4, 0] and not m[0, 4]


def test_wall_layer_median_ignores_the_few_contact_line_nodes():
    solid = np.zeros((10, 10), np.uint8)
    solid[4:6, :] = 1  # a solid band: first layer = rows 3 and 6, 20 nodes
    rA = np.full((10, 10), 0.03)
    rB = np.full((10, 10), 1.0)
    rA[3, :3] = 1.0  # A covers three first-layer nodes
    rB[3, :3] = 0.03
    rA[3, 3] = 0.4  # a contact-line node on the B side
    med, share = st.wall_layer(solid, rA, rB)
    assert med == pytest.approx(0.03)
    assert share == pytest.approx(3 / 20)
    rA[6, :] = 0.2  # a film of A along the other side of the band
    med, _ = st.wall_layer(solid, rA, rB)
    assert med == pytest.approx(0.2)


def test_scheme_study_cases_follow_the_paper_geometry():
    cases = S.scheme_study((30, 90, 150))
    assert [c.scheme for c in cases] == ["improved"] * 3 + ["original"] * 3
    for a, b in zip(cases[:3], cases[3:]):  # same geometry, initial state and lambda under both schemes
        assert np.array_equal(a.solid, b.solid) and np.array_equal(a.rhoA0, b.rhoA0)
        assert a.lam == b.lam and a.extra["target_theta"] == b.extra["target_theta"]
    lams = [c.lam for c in cases[:3]]
    assert lams == sorted(lams) and lams[1] == pytest.approx(S.lambda_for_angle(90))
    c = cases[0]
    assert (c.ny, c.nx) == (350, 300) and c.bc_x == c.bc_y == "periodic"
    assert c.solid.sum() == pytest.approx(np.pi * 70 ** 2, rel=0.01)
    inside = (c.rhoA0 > 0.5) & (c.solid == 0)
    ys, xs = np.nonzero(inside)
    # a disk of radius 50 about (150, 230), 0.6 r above the cylinder top, minus the cylinder
    assert np.all((xs - 150.0) ** 2 + (ys - 230.0) ** 2 <= 50.0 ** 2)
    assert xs.mean() == pytest.approx(150, abs=1e-9) and ys.max() == 280
    assert np.all((xs - 150.0) ** 2 + (ys - 130.0) ** 2 > 70.0 ** 2)
    assert c.solid[ys.min() - 1, 150] == 1  # the lowest row of A sits on the cylinder


# ---------------------------------------------------------------------------------------------
# co-current flow (Sec. 3.1)
# ---------------------------------------------------------------------------------------------
def test_cocurrent_cases_follow_the_paper_layout():
    from paper_2505_22256_gb300 import study_cocurrent as cc

    cs = cc.cases((45, 90, 135))
    assert [c.extra["flow"] for c in cs] == ["poiseuille"] * 3 + ["couette"] * 3
    for c in cs:
        assert (c.ny, c.nx) == (100, 50) and c.bc_x == "periodic" and c.bc_y == "wall"
        assert c.tau == (1.01, 1.01)
        a = c.rhoA0[:, 0] > 0.5  # A in the central half: rows 25 .. 74
        assert a.sum() == 50 and a[25] and a[74] and not a[24] and not a[75]
    assert cs[0].g == (1e-6, 0.0) and cs[0].u_wall == (0.0, 0.0)
    assert cs[3].g == (0.0, 0.0) and cs[3].u_wall == (-0.005, 0.005)


def test_momentum_balance_profile_reduces_to_the_analytic_one_for_uniform_density():
    """With a uniform density the balance is the single-fluid problem: the Couette line is reproduced
    exactly and the Poiseuille parabola to the O(1/H^2) of the mirrored ghost row."""
    from paper_2505_22256_gb300 import study_cocurrent as cc

    p, c = cc.cases((90,))
    rho = np.full(100, 1.03)
    uc = cc.balance_profile(c, rho)
    np.testing.assert_allclose(uc, cc.analytic_profile(c), rtol=0, atol=1e-15)
    up = cc.balance_profile(p, rho)
    ua = cc.analytic_profile(p)
    assert cc.rel_l2(up, ua) < 3 / 100 ** 2
    # g s (H - s) / (2 nu) at the two central nodes, s = 49.5 and 50.5 (the peak g H^2 / (8 nu) lies between)
    assert ua.max() == pytest.approx(1e-6 * 49.5 * 50.5 / (2 * 0.17), rel=1e-12)
    # a density dip at the two interfaces steepens the Couette profile there, and the shear stress
    # rho nu du/dy stays the same on every face
    rho2 = rho.copy()
    rho2[[24, 25, 74, 75]] = 0.7
    u2 = cc.balance_profile(c, rho2)
    rf = 0.5 * (rho2[1:] + rho2[:-1])
    stress = rf * np.diff(u2)
    np.testing.assert_allclose(stress, stress[0], rtol=1e-10)
    assert cc.rel_l2(u2, cc.analytic_profile(c)) > 1e-3


# ---------------------------------------------------------------------------------------------
# droplet past a square obstacle (Sec. 3.3)
# ---------------------------------------------------------------------------------------------
def test_obstacle_snapshot_counts_regions_by_what_they_touch():
    from paper_2505_22256_gb300 import study_obstacle as so

    sc = so.cases()[0]
    assert (sc.ny, sc.nx) == (150, 350) and sc.bc_x == "open" and sc.inlet_profile == "poiseuille"
    assert sc.solid.sum() == 25 * 25 and sc.solid[75, 122] == 1 and sc.solid[75, 135] == 0
    rA = np.full(sc.solid.shape, 0.03)
    rB = np.full(sc.solid.shape, 1.0)
    rA[sc.solid == 1] = rB[sc.solid == 1] = 0.0
    for sl in (np.s_[70:80, 40:50],     # a free droplet
               np.s_[0:3, 200:210],     # one on the lower channel wall
               np.s_[149, 300],         # a single node on the upper wall
               np.s_[61:63, 115:130]):  # a film on the obstacle's lower face (the square spans rows 63..87)
        rA[sl], rB[sl] = 1.0, 0.03
    # an A-enriched but B-dominated layer over the top and both side faces: 77 of the 89 B-side
    # first-layer nodes of the square (a ring of 104, 15 of them under the film)
    rA[63:89, 109] = rA[63:89, 135] = 0.3
    rA[88, 109:136] = 0.3
    d = so.snapshot(sc, rA, rB)
    assert d["regions"] == 4 and d["wall_regions"] == 2 and d["obstacle_regions"] == 1
    assert d["largest_area"] == 100 and d["total_area"] == 100 + 30 + 1 + 30
    assert d["wall_layer_rhoA"] == pytest.approx(0.03)
    ol = st.first_layer(sc.solid)
    b_side = ol & ~((rA > rB) & (sc.solid == 0))
    assert d["obstacle_layer_rhoA"] == pytest.approx(float(np.median(rA[b_side])))
    assert d["obstacle_layer_rhoA"] == pytest.approx(0.3)


def test_study_tables_render_missing_and_unsteady_values():
    from paper_2505_22256_gb300 import study_cocurrent as cc
    from paper_2505_22256_gb300 import study_sphere3d as s3

    rows = [{"scheme": "original", "target_theta": 150.0, "lambda": 2.17, "theta": None, "dtheta_last": float("nan"),
             "du_last": float("nan"), "umax": 0.37, "umax_off_wall": 0.2, "rho_min": 0.02, "rho_max": 1.1,
             "wall_layer_rhoA": float("nan"), "attached": False, "unstable": True}]
    t = st.table(rows)
    assert t.count("\n") == 2 and "| — |" in t and "no (unstable)" in t
    crow = [{"flow": "couette", "target_theta": 90.0, "lambda": 0.9951, "converged_at": None, "steps": 400000,
             "eps_analytic": 0.0955, "eps_balance": 0.0959, "u_peak": 5.4e-3, "u_peak_analytic": 4.95e-3,
             "rho_min": 0.66}]
    ct = cc.table(crow)
    assert "not within 400000" in ct and "9.55 %" in ct
    srow = [{"lambda": 0.38, "paper_theta": 45.0, "theta": 75.2, "dtheta_last": float("nan"), "umax": 0.012,
             "rhoA_min": 0.02, "rhoA_max": 1.05, "rhoB_min": 0.02, "rhoB_max": 1.02, "unstable": False}]
    assert "| 0.38 | 45 | 75.2 | — |" in s3.table(srow)
