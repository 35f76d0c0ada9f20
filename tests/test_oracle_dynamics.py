"""Pins for the oracle's time step against invariants, closed forms and textbook limits:
moments of Eq. 6 and Eq. 7, a quiescent uniform state, per-component mass, total momentum, the
BGK shear-wave decay, Poiseuille flow between halfway bounce-back walls (Eq. 13 within the
paper's 1.84 % bound), the Laplace law and mirror symmetry."""
import numpy as np
import pytest

import oracle
from paper_2505_22256_gb300 import scenarios as S

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
CS2 = 1.0 / 3.0


# ---------------------------------------------------------------------------------------------
# Eq. 6 and Eq. 7: velocity moments
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.03, 0.05, -0.02), (1.3, -0.11, 0.07)])
def test_equilibrium_moments(rho, ux, uy):
    fe = oracle.feq(rho, ux, uy)
    assert fe.sum() == pytest.approx(rho, rel=1e-14)
    assert (fe * CX).sum() == pytest.approx(rho * ux, abs=1e-15)
    assert (fe * CY).sum() == pytest.approx(rho * uy, abs=1e-15)
    u = (ux, uy)
    for a, ca in enumerate((CX, CY)):
        for b, cb in enumerate((CX, CY)):
            want = rho * CS2 * (a == b) + rho * u[a] * u[b]
            assert (fe * ca * cb).sum() == pytest.approx(want, rel=1e-13, abs=1e-16)


@pytest.mark.parametrize("ux,uy,Fx,Fy", [(0.0, 0.0, 1e-3, 0.0), (0.04, -0.03, -2e-3, 5e-4),
                                          (-0.1, 0.2, 0.3, -0.1)])
def test_guo_forcing_moments(ux, uy, Fx, Fy):
    """Guo's term carries no mass, momentum F and second moment u F + F u."""
    Fi = oracle.guo(ux, uy, Fx, Fy)
    assert Fi.sum() == pytest.approx(0.0, abs=1e-16)
    assert (Fi * CX).sum() == pytest.approx(Fx, rel=1e-13, abs=1e-17)
    assert (Fi * CY).sum() == pytest.approx(Fy, rel=1e-13, abs=1e-17)
    u, F = (ux, uy), (Fx, Fy)
    for a, ca in enumerate((CX, CY)):
        for b, cb in enumerate((CX, CY)):
            assert (Fi * ca * cb).sum() == pytest.approx(u[a] * F[b] + F[a] * u[b], rel=1e-12, abs=1e-17)


def test_guo_expanded_form():
    """(uF + Fu):(e e - c_s^2 I) = 2 (e.u)(e.F) - 2 c_s^2 u.F, so Eq. 7 equals
    w_i [ (e_i - u).F / c_s^2 + (e_i.u)(e_i.F) / c_s^4 ]."""
    W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    ux, uy, Fx, Fy = 0.07, -0.04, 0.011, 0.023
    eu = CX * ux + CY * uy
    eF = CX * Fx + CY * Fy
    alt = W * ((eF - (ux * Fx + uy * Fy)) / CS2 + eu * eF / CS2 ** 2)
    np.testing.assert_allclose(oracle.guo(ux, uy, Fx, Fy), alt, rtol=1e-13, atol=1e-18)


# ---------------------------------------------------------------------------------------------
# P6: quiescent uniform state
# ---------------------------------------------------------------------------------------------
def test_uniform_state_stays_at_rest():
    n = 24
    solid = np.zeros((n, n), np.uint8)
    cfg = oracle.Config(nx=n, ny=n, bc_x="periodic", bc_y="periodic", G=S.G_DEFAULT, lam=0.5)
    f0 = oracle.init(cfg, solid, np.full((n, n), S.RHO_M), np.full((n, n), S.RHO_D))
    f = oracle.run(cfg, solid, f0, 50)
    rA, rB, ux, uy = oracle.fields(cfg, solid, f)
    assert np.all(ux == 0.0) and np.all(uy == 0.0)
    np.testing.assert_allclose(f, f0, rtol=1e-14, atol=0)


# ---------------------------------------------------------------------------------------------
# P4: mass conservation; P5: momentum conservation
# ---------------------------------------------------------------------------------------------
def test_mass_conserved_per_component_with_walls():
    sc = S.cylinder_droplet(48, lam=0.6)
    cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
    f = oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
    m0 = f.reshape(2, -1).sum(axis=1)
    f = oracle.run(cfg, sc.solid, f, 2000)
    m1 = f.reshape(2, -1).sum(axis=1)
    assert np.all(np.abs(m1 / m0 - 1) <= 1e-12), m1 / m0 - 1
    assert np.all(np.isfinite(f))


def test_total_force_vanishes_and_momentum_is_conserved_when_periodic():
    sc = S.free_droplet(40, R=9)
    cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
    f = oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
    f = oracle.run(cfg, sc.solid, f, 30)
    FA, FB = oracle.forces(cfg, sc.solid, f)
    tot = (FA + FB).reshape(2, -1).sum(axis=1)
    assert np.all(np.abs(tot) < 1e-13), tot
    mom0 = np.array([(f * CX[None, :, None, None]).sum(), (f * CY[None, :, None, None]).sum()])
    f2 = oracle.run(cfg, sc.solid, f, 200)
    mom1 = np.array([(f2 * CX[None, :, None, None]).sum(), (f2 * CY[None, :, None, None]).sum()])
    assert np.all(np.abs(mom1 - mom0) < 1e-12), (mom0, mom1)


# ---------------------------------------------------------------------------------------------
# P7: BGK shear-wave decay, nu = (tau - 1/2) c_s^2
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("tau", [0.8, 1.0, 1.4])
def test_shear_wave_decay(tau):
    nx, ny, U, t = 4, 128, 1e-4, 1600
    k = 2 * np.pi / ny
    solid = np.zeros((ny, nx), np.uint8)
    cfg = oracle.Config(nx=nx, ny=ny, bc_x="periodic", bc_y="periodic", G=0.0, tau=(tau, tau))
    f = np.zeros((2, 9, ny, nx))
    for y in range(ny):
        ux = U * np.sin(k * y)
        for comp, rho in enumerate((0.7, 0.3)):
            f[comp, :, y, :] = oracle.feq(rho, ux, 0.0)[:, None]
    f = oracle.run(cfg, solid, f, t)
    _, _, ux, _ = oracle.fields(cfg, solid, f)
    amp = 2.0 / ny * np.sum(ux[:, 0] * np.sin(k * np.arange(ny)))
    nu = (tau - 0.5) * CS2
    assert amp / U == pytest.approx(np.exp(-nu * k * k * t), rel=2e-3)


# ---------------------------------------------------------------------------------------------
# P8: Poiseuille flow with body force between halfway bounce-back walls (Eq. 13, Sec. 3.1)
# ---------------------------------------------------------------------------------------------
def _channel_profile(cfg, solid, rA0, rB0, steps):
    f = oracle.init(cfg, solid, rA0, rB0)
    f = oracle.run(cfg, solid, f, steps)
    _, _, ux, _ = oracle.fields(cfg, solid, f)
    return ux[:, 0]


def test_poiseuille_single_fluid_matches_parabola():
    """Walls at half a link beyond rows 1 and ny-2: u(y) = g/(2 nu) (L^2 - y^2), L = (ny-2)/2."""
    nx, ny, g, tau = 4, 34, 1e-6, 1.0
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    cfg = oracle.Config(nx=nx, ny=ny, bc_x="periodic", bc_y="wall", G=0.0, g=(g, 0.0), tau=(tau, tau))
    ux = _channel_profile(cfg, solid, np.full((ny, nx), 0.6), np.full((ny, nx), 0.4), 12000)
    nu = (tau - 0.5) * CS2
    L = (ny - 2) / 2.0
    y = np.arange(ny) - (ny - 1) / 2.0
    ua = g / (2 * nu) * (L * L - y * y)
    fl = slice(1, ny - 1)
    assert np.max(np.abs(ux[fl] - ua[fl])) / ua.max() < 0.01


def _momentum_balance_profile(rho, g, nu):
    """Steady parallel flow of a fluid of density rho(y) and kinematic viscosity nu driven by the
    acceleration g: d/dy(nu rho du/dy) = -rho g, u = 0 half a link outside the first and last
    fluid rows.  Finite-volume form with face densities (rho_j + rho_j+1)/2."""
    n = len(rho)
    A = np.zeros((n, n))
    b = -np.asarray(rho) * g
    for j in range(n):
        for k in (j - 1, j + 1):
            m = nu * (0.5 * (rho[j] + rho[k]) if 0 <= k < n else 2.0 * rho[j])
            A[j, j] -= m
            if 0 <= k < n:
                A[j, k] += m
    return np.linalg.solve(A, b)


def test_cocurrent_two_layer_flow_obeys_momentum_balance():
    """Sec. 3.1 layout: fluid 1 in |y| <= a, fluid 2 outside, equal viscosity and main density,
    body force g on both, no wall adhesion.  The interface is diffuse, so Eq. 13's sharp-interface
    parabola is not exact; the steady x-momentum balance with the simulated mixture density is."""
    nx, ny, g, a = 4, 52, 1e-6, 12.5
    y = np.arange(ny) - (ny - 1) / 2.0
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    inner = np.abs(y) <= a
    rA0 = np.where(inner, S.RHO_M, S.RHO_D)[:, None] * np.ones((1, nx))
    rB0 = np.where(inner, S.RHO_D, S.RHO_M)[:, None] * np.ones((1, nx))
    rA0[solid == 1] = 0
    rB0[solid == 1] = 0
    cfg = oracle.Config(nx=nx, ny=ny, bc_x="periodic", bc_y="wall", G=S.G_DEFAULT, lam=1.0, Gw2=0.0,
                        g=(g, 0.0), tau=(1.0, 1.0))
    f = oracle.init(cfg, solid, rA0, rB0)
    f = oracle.run(cfg, solid, f, 30000)
    rA, rB, ux, _ = oracle.fields(cfg, solid, f)
    ub = _momentum_balance_profile((rA + rB)[1:-1, 0], g, 0.5 * CS2)
    err = np.max(np.abs(ux[1:-1, 0] - ub)) / ub.max()
    assert err < 0.015, err
    # the two layers really are separated: main / dissolved densities in each layer
    assert rA[ny // 2, 0] > 0.9 and rB[ny // 2, 0] < 0.1 and rB[3, 0] > 0.9


# ---------------------------------------------------------------------------------------------
# P9: Laplace law, p = c_s^2 (rho_A + rho_B) + G rho_A rho_B for weights with sum w e_x^2 = 1
# ---------------------------------------------------------------------------------------------
@pytest.mark.slow
def test_laplace_law():
    n = 80
    inv_r, dp = [], []
    for R in (10, 14, 18, 22):
        sc = S.free_droplet(n, R=R, amp=0.0)
        cfg = oracle.Config(nx=n, ny=n, **sc.params())
        f = oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
        f = oracle.run(cfg, sc.solid, f, 3000)
        rA, rB, _, _ = oracle.fields(cfg, sc.solid, f)
        p = CS2 * (rA + rB) + cfg.G * rA * rB
        pin = p[n // 2 - 2:n // 2 + 2, n // 2 - 2:n // 2 + 2].mean()
        pout = p[:3, :3].mean()
        pts = oracle.interface_points(cfg, sc.solid, rA, rB)
        _, _, r, _ = oracle.fit_circle(pts)
        inv_r.append(1.0 / r)
        dp.append(pin - pout)
    slope, icpt = np.polyfit(inv_r, dp, 1)
    pred = slope * np.array(inv_r) + icpt
    r2 = 1 - np.sum((np.array(dp) - pred) ** 2) / np.sum((np.array(dp) - np.mean(dp)) ** 2)
    assert slope > 0 and r2 > 0.99
    assert abs(icpt) < 0.1 * slope * min(inv_r), (slope, icpt)


# ---------------------------------------------------------------------------------------------
# P10: mirror symmetry of a symmetric flat-wall case
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("adhesion_stencil", ["e8", "d2q9"])
@pytest.mark.parametrize("lam", [0.4, 1.8])
def test_flat_wall_mirror_symmetry(lam, adhesion_stencil):
    sc = S.flat_droplet(nx=40, ny=30, r=9, lam=lam, amp=0.0)
    sc.adhesion_stencil = adhesion_stencil
    cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
    f = oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0)
    f = oracle.run(cfg, sc.solid, f, 400)
    rA, rB, ux, uy = oracle.fields(cfg, sc.solid, f)
    for a in (rA, rB, uy):
        assert np.max(np.abs(a - a[:, ::-1])) <= 1e-12
    assert np.max(np.abs(ux + ux[:, ::-1])) <= 1e-12


@pytest.mark.parametrize("u_wall", [(-0.01, 0.01), (0.0, 0.008)])
def test_couette_between_sliding_walls_is_exactly_linear(u_wall):
    """Sec. 3.1's Couette flow, single phase (G = 0): halfway bounce-back walls half a cell below
    row 0 and above row ny-1 slide at u_wall; the steady profile is the linear Couette solution
    u(s) = u_lo + (u_hi - u_lo) s / H, s = y + 1/2, H = ny, with no wall-normal velocity."""
    nx, ny = 4, 16
    solid = np.zeros((ny, nx), np.uint8)
    cfg = oracle.Config(nx=nx, ny=ny, bc_x="periodic", bc_y="wall", G=0.0, u_wall=u_wall)
    f = oracle.init(cfg, solid, np.ones((ny, nx)), np.full((ny, nx), 1e-3))
    f = oracle.run(cfg, solid, f, 6000)  # slowest mode decays as exp(-nu pi^2 t / H^2)
    _, _, ux, uy = oracle.fields(cfg, solid, f)
    s = np.arange(ny) + 0.5
    exact = u_wall[0] + (u_wall[1] - u_wall[0]) * s / ny
    np.testing.assert_allclose(ux, np.repeat(exact[:, None], nx, axis=1), rtol=0, atol=1e-12)
    assert np.max(np.abs(uy)) < 1e-14


@pytest.mark.parametrize("scheme,second_layer,adhesion_stencil",
                         [("improved", "psi_and_solid", "e8"), ("original", "psi_and_solid", "e8"),
                          ("improved", "psi", "e8"), ("original", "psi", "e8"),
                          ("improved", "psi_and_solid", "d2q9"), ("original", "psi_and_solid", "d2q9")])
def test_exchanging_the_components_at_lambda_one_exchanges_the_state(scheme, second_layer, adhesion_stencil):
    """At lambda = 1 (and equal tau) nothing distinguishes A from B: cohesion uses the other
    component, both adhesion parameters are G_w2 (Eq. 12 gives h = 1), and the collision is the
    same.  A droplet of B started from the swapped densities must therefore reach the swapped
    state, up to the order of the sums over components (1e-13).  A wrong component index, or a
    term applied to one component only, breaks this."""
    sc = S.flat_droplet(40, 28, r=8, lam=1.0, scheme=scheme)
    sc.solid[10:13, 6:9] = 1  # a small block as well, for curved-wall stencil sites
    sc.rhoA0[sc.solid == 1] = 0.0
    sc.rhoB0[sc.solid == 1] = 0.0
    sc.second_layer = second_layer
    sc.adhesion_stencil = adhesion_stencil
    cfg = oracle.Config(nx=sc.nx, ny=sc.ny, **sc.params())
    fA = oracle.run(cfg, sc.solid, oracle.init(cfg, sc.solid, sc.rhoA0, sc.rhoB0), 150)
    fB = oracle.run(cfg, sc.solid, oracle.init(cfg, sc.solid, sc.rhoB0, sc.rhoA0), 150)
    a = oracle.fields(cfg, sc.solid, fA)
    b = oracle.fields(cfg, sc.solid, fB)
    np.testing.assert_allclose(b[0], a[1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b[1], a[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b[2], a[2], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b[3], a[3], rtol=0, atol=1e-13)
    assert np.max(np.abs(a[0] - a[1])) > 0.5  # a genuine two-phase state
