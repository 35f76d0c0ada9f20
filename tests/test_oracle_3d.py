"""Pins of the 3-D oracle (Sec. 3.5): stencil isotropy, brute-force stencil sums, conservation,
rest state, symmetry, the lambda = 1 identity, the Laplace law and the sphere fit."""
import itertools

import numpy as np
import pytest

from oracle import d3

CS2 = 1.0 / 3.0


def test_stencil_has_92_offsets_and_the_shell_counts():
    offs = d3.stencil_offsets()
    assert len(offs) == 92
    counts = {q: sum(1 for e in offs if sum(t * t for t in e) == q) for q in d3.SHELLS3}
    assert counts == {1: 6, 2: 12, 3: 8, 4: 6, 5: 24, 6: 24, 8: 12}


def test_weights_are_positive_and_isotropic_in_every_direction():
    """Isotropy of the moment tensors up to 8th order means that sum_e w (e.n)^k is the same for
    every unit vector n (k = 2, 4, 6, 8), equal to M(k,0,0); odd moments vanish.  Checked for
    random directions -- a different form of the conditions the weights were solved from."""
    w = d3.e8_weights_3d()
    assert all(v > 0 for v in w.values())
    offs = np.array(d3.stencil_offsets(), dtype=np.float64)
    wt = np.array([float(w[int(round(np.dot(e, e)))]) for e in offs])
    rng = np.random.default_rng(0)
    for k, expect in ((2, 1.0), (4, 12 / 7), (6, 32 / 7), (8, 16.0)):
        for _ in range(8):
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            assert np.sum(wt * (offs @ n) ** k) == pytest.approx(expect, rel=1e-12), k
    for k in (1, 3, 5, 7):
        n = rng.normal(size=3)
        assert abs(np.sum(wt * (offs @ n) ** k)) < 1e-12


def test_d3q19_moments_and_guo_moments():
    e = np.array(d3.E19, dtype=np.float64)
    rho, u, F = 0.9, np.array([0.02, -0.01, 0.015]), np.array([1e-3, 2e-3, -5e-4])
    fe = d3.feq3(rho, *u)
    assert fe.sum() == pytest.approx(rho, rel=1e-14)
    np.testing.assert_allclose(fe @ e, rho * u, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose((e.T * fe) @ e, rho * CS2 * np.eye(3) + rho * np.outer(u, u), rtol=1e-12, atol=1e-15)
    Fi = d3.guo3(*u, *F)
    assert abs(Fi.sum()) < 1e-16
    np.testing.assert_allclose(Fi @ e, F, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose((e.T * Fi) @ e, np.outer(u, F) + np.outer(F, u), rtol=1e-12, atol=1e-18)


def _brute_forces(cfg, solid, rA, rB, x, y, z):
    """Direct triple loop over the stencil with an independently written second-layer rule."""
    w = {q: float(v) for q, v in d3.e8_weights_3d().items()}
    nz, ny, nx = solid.shape

    def site(px, py, pz):
        return pz % nz, py % ny, px % nx

    gA, gB, a = np.zeros(3), np.zeros(3), np.zeros(3)
    for e in itertools.product(range(-2, 3), repeat=3):
        q = sum(t * t for t in e)
        if q not in w:
            continue
        s = site(x + e[0], y + e[1], z + e[2])
        replaced = max(abs(t) for t in e) == 2 and solid[s]
        if replaced:
            s = site(x + int(np.sign(e[0])), y + int(np.sign(e[1])), z + int(np.sign(e[2])))
        pa, pb, sw = (0.0, 0.0, 1.0) if solid[s] else (rA[s], rB[s], 0.0)
        if replaced and cfg.second_layer == "psi":  # psi copied, the solid site keeps its switch
            sw = 1.0
        gA += w[q] * pa * np.array(e)
        gB += w[q] * pb * np.array(e)
        a += w[q] * sw * np.array(e)
    if cfg.adhesion_stencil == "d3q19":  # Eq. 9 as printed: D3Q19 weights over the first neighbours
        a = np.zeros(3)
        for e in itertools.product(range(-1, 2), repeat=3):
            q = sum(t * t for t in e)
            if q in (1, 2) and solid[site(x + e[0], y + e[1], z + e[2])]:
                a += (1.0 / 18.0 if q == 1 else 1.0 / 36.0) * np.array(e)
    ra, rb = rA[z, y, x], rB[z, y, x]
    re = (ra - rb) / (ra + rb)
    lam, dl = cfg.lam, cfg.delta
    if re > dl:
        h = lam
    elif re > 0:
        h = 2 * lam / (1 + lam) + 2 * (lam * lam - lam) / (dl * (1 + lam)) * re + (lam - lam * lam) / (dl * dl * (1 + lam)) * re * re
    elif re > -dl:
        h = 2 * lam / (1 + lam) + 2 * (lam - 1) / (dl * (1 + lam)) * re + (lam - 1) / (dl * dl * (1 + lam)) * re * re
    else:
        h = 1.0
    FA = -cfg.G * ra * gB - cfg.Gw2 * h * ra * a
    FB = -cfg.G * rb * gA - cfg.Gw2 * rb * a
    return FA, FB


@pytest.mark.parametrize("second_layer,adhesion_stencil", [("psi_and_solid", "e8"), ("psi", "e8"),
                                                            ("psi_and_solid", "d3q19"), ("psi", "d3q19")])
def test_forces_match_brute_force_next_to_a_solid_block(second_layer, adhesion_stencil):
    n = 9
    solid = np.zeros((n, n, n), np.uint8)
    solid[3:6, 2:5, 4:7] = 1
    solid[7, 7, 1] = 1
    rng = np.random.default_rng(5)
    rA = np.where(solid, 0.0, 0.2 + 0.8 * rng.random((n, n, n)))
    rB = np.where(solid, 0.0, 0.2 + 0.8 * rng.random((n, n, n)))
    cfg = d3.Config3(n, n, n, G=1.1, lam=0.6, Gw2=0.35, second_layer=second_layer,
                     adhesion_stencil=adhesion_stencil)
    f = d3.init3(cfg, solid, rA, rB)
    FA, FB, _ = d3.forces3(cfg, solid, f)
    for (z, y, x) in [(2, 3, 5), (6, 3, 5), (4, 1, 5), (4, 5, 3), (0, 0, 0), (7, 6, 2), (4, 8, 8)]:
        assert not solid[z, y, x]
        ba, bb = _brute_forces(cfg, solid, rA, rB, x, y, z)
        np.testing.assert_allclose(FA[:, z, y, x], ba, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(FB[:, z, y, x], bb, rtol=1e-12, atol=1e-14)


def _sphere_case(n=20, R=4.0, r=4.5, lam=0.7, noise=True, seed=3):
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
    c = (n - 1) / 2.0
    solid = ((x - c) ** 2 + (y - c) ** 2 + (z - 0.35 * n) ** 2 <= R * R).astype(np.uint8)
    inside = (x - c) ** 2 + (y - c) ** 2 + (z - (0.35 * n + R + 0.6 * r)) ** 2 <= r * r
    rng = np.random.default_rng(seed)
    amp = 1e-4 if noise else 0.0
    rA = np.where(inside, 1.0, 0.03) + amp * (rng.random((n, n, n)) - 0.5)
    rB = np.where(inside, 0.03, 1.0) + amp * (rng.random((n, n, n)) - 0.5)
    rA[solid == 1] = 0.0
    rB[solid == 1] = 0.0
    return solid, rA, rB


def test_mass_is_conserved_per_component_around_a_sphere():
    solid, rA, rB = _sphere_case()
    n = solid.shape[0]
    cfg = d3.Config3(n, n, n, G=1.205, lam=0.7, Gw2=0.3)
    f = d3.run3(cfg, solid, d3.init3(cfg, solid, rA, rB), 150)
    d = d3.diagnostics3(cfg, solid, f)
    assert d["mass_A"] == pytest.approx(rA.sum(), rel=1e-12)
    assert d["mass_B"] == pytest.approx(rB.sum(), rel=1e-12)


def test_uniform_state_stays_at_rest_and_momentum_is_conserved():
    n = 8
    solid = np.zeros((n, n, n), np.uint8)
    cfg = d3.Config3(n, n, n, G=1.205, lam=1.0, Gw2=0.3)
    f0 = d3.init3(cfg, solid, np.full((n, n, n), 1.0), np.full((n, n, n), 0.03))
    f1 = d3.run3(cfg, solid, f0, 20)
    np.testing.assert_allclose(f1, f0, rtol=1e-14, atol=1e-17)
    rng = np.random.default_rng(2)
    rA = 0.5 + 0.3 * rng.random((n, n, n))
    f = d3.init3(cfg, solid, rA, 1.0 - rA)
    FA, FB, _ = d3.forces3(cfg, solid, f)
    assert np.max(np.abs((FA + FB).sum(axis=(1, 2, 3)))) < 1e-12
    f = d3.run3(cfg, solid, f, 30)
    d = d3.diagnostics3(cfg, solid, f)
    assert max(abs(d["mom_x"]), abs(d["mom_y"]), abs(d["mom_z"])) < 1e-11


@pytest.mark.parametrize("adhesion_stencil", ["e8", "d3q19"])
def test_lambda_one_makes_improved_equal_original(adhesion_stencil):
    solid, rA, rB = _sphere_case(n=14, R=3.0, r=3.5)
    n = solid.shape[0]
    out = []
    for scheme in ("improved", "original"):
        cfg = d3.Config3(n, n, n, scheme=scheme, G=1.205, lam=1.0, Gw2=0.3, adhesion_stencil=adhesion_stencil)
        out.append(d3.run3(cfg, solid, d3.init3(cfg, solid, rA, rB), 40))
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("adhesion_stencil", ["e8", "d3q19"])
def test_mirror_symmetry_of_a_symmetric_droplet_on_a_sphere(adhesion_stencil):
    solid, rA, rB = _sphere_case(n=16, R=3.5, r=3.5, noise=False)
    n = solid.shape[0]
    cfg = d3.Config3(n, n, n, G=1.205, lam=0.5, Gw2=0.3, adhesion_stencil=adhesion_stencil)
    f = d3.run3(cfg, solid, d3.init3(cfg, solid, rA, rB), 60)
    ra, rb, ux, uy, uz = d3.fields3(cfg, solid, f)
    for a in (ra, rb, uy, uz):  # x -> n-1-x mirror (the geometry is symmetric about x = (n-1)/2)
        assert np.max(np.abs(a - a[:, :, ::-1])) <= 1e-12
    assert np.max(np.abs(ux + ux[:, :, ::-1])) <= 1e-12


def test_sphere_fit_recovers_exact_spheres_and_the_contact_angle_formula():
    rng = np.random.default_rng(7)
    c, r = np.array([3.2, -1.5, 7.7]), 5.5
    v = rng.normal(size=(400, 3))
    pts = c + r * v / np.linalg.norm(v, axis=1)[:, None]
    cx, cy, cz, rr, rms = d3.fit_sphere(pts)
    np.testing.assert_allclose([cx, cy, cz, rr], [*c, r], rtol=1e-12, atol=1e-12)
    assert rms < 1e-12
    # two spheres meeting at a known angle: the formula returns it
    for theta in (30.0, 90.0, 140.0):
        R, rd = 10.0, 6.0
        d = np.sqrt(R * R + rd * rd - 2 * R * rd * np.cos(np.radians(theta)))
        cth = (R * R + rd * rd - d * d) / (2 * rd * R)
        assert np.degrees(np.arccos(cth)) == pytest.approx(theta, abs=1e-10)


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_contact_angle_of_a_constructed_droplet_on_a_sphere(theta):
    """A smooth droplet whose rho^e = 0 surface is the sphere |p - c| = r, meeting the solid sphere
    (effective radius R + 1/2) at the angle theta: the measurement returns theta."""
    n, R, r = 40, 8.0, 9.0
    Re = R + 0.5
    sc = np.array([19.5, 19.5, 12.0])
    d = np.sqrt(Re * Re + r * r - 2 * Re * r * np.cos(np.radians(theta)))
    cc = sc + np.array([0.0, 0.0, d])
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
    solid = ((x - sc[0]) ** 2 + (y - sc[1]) ** 2 + (z - sc[2]) ** 2 <= R * R).astype(np.uint8)
    dist = np.sqrt((x - cc[0]) ** 2 + (y - cc[1]) ** 2 + (z - cc[2]) ** 2)
    rA = 0.515 + 0.485 * np.tanh((r - dist) / 2.0)
    rB = 1.03 - rA
    rA[solid == 1] = 0.0
    rB[solid == 1] = 0.0
    cfg = d3.Config3(n, n, n, G=1.205, lam=1.0, Gw2=0.3)
    f = d3.init3(cfg, solid, rA, rB)
    th, rms, npts = d3.contact_angle_sphere(cfg, solid, f, {"c": tuple(sc), "R": Re})
    assert npts > 200
    assert th == pytest.approx(theta, abs=0.5)
    assert rms < 0.05


@pytest.mark.slow
def test_laplace_law_3d():
    """Free droplets in a periodic box: the pressure jump p = c_s^2 (rho_A + rho_B) + G rho_A rho_B
    grows linearly with the mean curvature 1/R of the fitted sphere, through the origin."""
    n = 32  # a 24^3 box leaves too little outer phase: the periodic images shift the jumps
    inv_r, dp = [], []
    for R in (6.0, 8.0, 10.0):
        z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
        inside = (x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2 <= R * R
        rA = np.where(inside, 1.0, 0.03)
        rB = np.where(inside, 0.03, 1.0)
        solid = np.zeros((n, n, n), np.uint8)
        cfg = d3.Config3(n, n, n, G=1.205)
        f = d3.run3(cfg, solid, d3.init3(cfg, solid, rA, rB), 1500)
        ra, rb, _, _, _ = d3.fields3(cfg, solid, f)
        p = CS2 * (ra + rb) + cfg.G * ra * rb
        h = n // 2
        pin = p[h - 1:h + 1, h - 1:h + 1, h - 1:h + 1].mean()
        pout = p[:2, :2, :2].mean()
        pts = d3.interface_points3(solid, ra, rb)
        _, _, _, r, _ = d3.fit_sphere(pts)
        inv_r.append(1.0 / r)
        dp.append(pin - pout)
    slope, icpt = np.polyfit(inv_r, dp, 1)
    pred = slope * np.array(inv_r) + icpt
    r2 = 1 - np.sum((np.array(dp) - pred) ** 2) / np.sum((np.array(dp) - np.mean(dp)) ** 2)
    assert slope > 0 and r2 > 0.99, (inv_r, dp)
    assert abs(icpt) < 0.15 * slope * min(inv_r), (slope, icpt)


def test_d3q19_adhesion_by_hand_next_to_a_flat_wall():
    """Eq. 9 as printed in 3-D, next to a solid plane z = 0 (uniform densities, no cohesion): the
    first layer sees e_z = -1 on one axis and four diagonal velocities, a_z = -(1/18 + 4/36) = -1/6,
    so F_k = G_w,k rho_k / 6 along +z; the second layer feels nothing; the two second-layer readings
    give one state."""
    n = 8
    solid = np.zeros((n, n, n), np.uint8)
    solid[0] = 1
    rA = np.where(solid, 0.0, 0.8)
    rB = np.where(solid, 0.0, 0.1)
    cfg = d3.Config3(n, n, n, scheme="original", G=0.0, lam=0.5, Gw2=0.3, adhesion_stencil="d3q19", nthreads=1)
    FA, FB, _ = d3.forces3(cfg, solid, d3.init3(cfg, solid, rA, rB))
    np.testing.assert_allclose(FA[2, 1], 0.5 * 0.3 * 0.8 / 6.0, rtol=1e-14)
    np.testing.assert_allclose(FB[2, 1], 0.3 * 0.1 / 6.0, rtol=1e-14)
    np.testing.assert_allclose(FA[2, n - 1], -0.5 * 0.3 * 0.8 / 6.0, rtol=1e-14)  # periodic: the plane again
    assert np.all(FA[:2] == 0.0) and np.all(FA[2, 2:n - 1] == 0.0)
    solid, rA, rB = _sphere_case(n=14, R=3.0, r=3.5)
    out = []
    for layer in ("psi_and_solid", "psi"):
        cfg = d3.Config3(14, 14, 14, G=1.205, lam=1.6, Gw2=0.3, second_layer=layer, adhesion_stencil="d3q19")
        out.append(d3.run3(cfg, solid, d3.init3(cfg, solid, rA, rB), 30))
    np.testing.assert_array_equal(out[0], out[1])
