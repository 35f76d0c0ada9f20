"""Seeded synthetic inputs: solid masks and initial component densities.

This module holds none of the method's arithmetic: it only draws geometries shaped like the
paper's test cases (a droplet resting on a cylinder, Sec. 3.2; a droplet in a confined channel,
Sec. 3.3; immiscible displacement, Sec. 3.4; co-current layers, Sec. 3.1) and initial density
fields.  Both the CUDA library's callers and the CPU checker receive these arrays as inputs.

Conventions: arrays are indexed [y, x]; ``solid`` is uint8 (1 = solid node); component A is the
paper's fluid 1 and B its fluid 2.  Initial densities are a sharp step between the main density
rho^m and the dissolved density rho^d (Sec. 2.1), plus independent uniform noise in
[-amp, amp) on each fluid node and component from a counter-based generator (SplitMix64 of
(seed, node, component)), so any node's noise can be regenerated on its own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RHO_M = 1.0
RHO_D = 0.03
NOISE_AMP = 1.0e-4


def mean_field_G(rho_m: float = RHO_M, rho_d: float = RHO_D, cs2: float = 1.0 / 3.0) -> float:
    """Inter-component strength at which the mean-field coexisting densities of the symmetric
    two-component mixture are (rho_m, rho_d), for stencil weights normalised to
    sum_e w e_x^2 = 1: G (rho_m - rho_d) = c_s^2 ln(rho_m / rho_d)."""
    return cs2 * math.log(rho_m / rho_d) / (rho_m - rho_d)


# Default G_AB: 1.205 for 1.0 / 0.03.  (G_AB = 3.5 in this weight normalisation diverges within two
# steps on the 96x96 cylinder case.)
G_DEFAULT = round(mean_field_G(), 3)

# Default adhesion parameter of component B for the synthetic workloads.  With both forces on the
# same normalised stencil, G_w2 = G_AB puts a wall force of about 0.53 lambda per unit density on
# the main phase and cases with lambda >= 1.7 diverge; G_w2 = 0.3 keeps the whole lambda range of
# the sweep (0.22 .. 2.17) stable with theta increasing in lambda.
GW2_DEFAULT = 0.3

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) applied to uint64 counters."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def node_noise(seed: int, ny: int, nx: int, comp: int, amp: float = NOISE_AMP) -> np.ndarray:
    """Uniform noise in [-amp, amp) for every node of an ny x nx grid and one component.
    Counter = seed << 40 | node << 1 | comp, node = y*nx + x; u = top 53 bits / 2^53."""
    node = np.arange(ny * nx, dtype=np.uint64)
    ctr = (np.uint64(seed) << np.uint64(40)) | (node << np.uint64(1)) | np.uint64(comp)
    u = (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (amp * (2.0 * u - 1.0)).reshape(ny, nx)


def lambda_for_angle(theta_deg: float) -> float:
    """Strength coefficient lambda for a target contact angle from the paper's empirical
    correlation theta = -13.76 lambda^2 + 94.62 lambda + 9.47 (Sec. 3.2, Fig. 7): smaller root."""
    a, b, c = -13.76, 94.62, 9.47 - theta_deg
    disc = b * b - 4 * a * c
    if disc < 0:
        raise ValueError("angle outside the correlation's range")
    return (-b + math.sqrt(disc)) / (2 * a)


@dataclass
class Scenario:
    """One lattice case: geometry, initial densities and model parameters."""
    name: str
    solid: np.ndarray          # (ny, nx) uint8
    rhoA0: np.ndarray          # (ny, nx) float64
    rhoB0: np.ndarray          # (ny, nx) float64
    bc_x: str = "periodic"     # periodic | wall | open
    bc_y: str = "wall"         # periodic | wall
    scheme: str = "improved"
    tau: tuple = (1.0, 1.0)
    G: float = G_DEFAULT
    lam: float = 1.0
    Gw2: float | None = GW2_DEFAULT
    delta: float = 0.8
    g: tuple = (0.0, 0.0)
    u_in: float = 0.0
    rho_in: tuple = (RHO_M, RHO_D)
    u_wall: tuple = (0.0, 0.0)         # x-velocity of the lower / upper wall (bc_y = wall)
    inlet_profile: str = "uniform"     # uniform | poiseuille (open x)
    # what a non-fluid second-layer stencil site takes from x + sign(e) (Sec. 2.4, Table 1):
    # psi_and_solid | psi
    second_layer: str = "psi_and_solid"
    # stencil of the adhesion sum of Eq. 9: e8 (the cohesion force's 24-node stencil) | d2q9 (as
    # printed: D2Q9 weights over the eight first-layer neighbours)
    adhesion_stencil: str = "e8"
    # outflow at x = nx-1 of an open x: copy (from column nx-2) | pressure (Zou-He density
    # condition holding rho_out per component)
    outlet: str = "copy"
    rho_out: tuple = (RHO_D, RHO_M)
    surface: dict | None = None  # for the contact angle: {"kind": "flat"|"circle", ...}
    # 16-bit storage keeps f_i - w_i rho0 per component; the dissolved-phase density serves both
    # phases best (ignored by FP32 / FP64 storage)
    rho0_store: tuple = (RHO_D, RHO_D)
    extra: dict = field(default_factory=dict)

    @property
    def ny(self) -> int:
        return self.solid.shape[0]

    @property
    def nx(self) -> int:
        return self.solid.shape[1]

    def params(self) -> dict:
        return dict(bc_x=self.bc_x, bc_y=self.bc_y, scheme=self.scheme, tau=tuple(self.tau),
                    G=self.G, lam=self.lam, Gw2=self.Gw2, delta=self.delta, g=tuple(self.g),
                    u_in=self.u_in, rho_in=tuple(self.rho_in), u_wall=tuple(self.u_wall),
                    inlet_profile=self.inlet_profile, second_layer=self.second_layer,
                    adhesion_stencil=self.adhesion_stencil, outlet=self.outlet, rho_out=tuple(self.rho_out))


def _grid(ny, nx):
    y, x = np.mgrid[0:ny, 0:nx]
    return y.astype(np.float64), x.astype(np.float64)


def _phase_fields(inside_A: np.ndarray, solid: np.ndarray, seed: int, amp: float = NOISE_AMP,
                  rho_m: float = RHO_M, rho_d: float = RHO_D):
    ny, nx = solid.shape
    rA = np.where(inside_A, rho_m, rho_d) + node_noise(seed, ny, nx, 0, amp)
    rB = np.where(inside_A, rho_d, rho_m) + node_noise(seed, ny, nx, 1, amp)
    rA[solid.astype(bool)] = 0.0
    rB[solid.astype(bool)] = 0.0
    return rA, rB


def cylinder_droplet(n: int = 96, R: float | None = None, r: float | None = None, lam: float = 1.0,
                     seed: int = 1, scheme: str = "improved", G: float = G_DEFAULT, tau=(1.0, 1.0),
                     nx: int | None = None, amp: float = NOISE_AMP) -> Scenario:
    """Droplet of A resting on a solid cylinder (Sec. 3.2, Fig. 5) at the 96x96 scale: rows 0 and
    ny-1 solid, x periodic, a cylinder of radius R = n/6 centred on the bottom row, a droplet of
    radius r = 5n/24 centred 0.6 r above the cylinder top (the paper's 300x350 case has the droplet
    centre 0.6 r above the cylinder top as well)."""
    ny = n
    nx = n if nx is None else nx
    R = n / 6.0 if R is None else R
    r = 5.0 * n / 24.0 if r is None else r
    y, x = _grid(ny, nx)
    cx, cy = nx // 2, 0
    solid = ((x - cx) ** 2 + (y - cy) ** 2 <= R * R)
    solid[0, :] = True
    solid[ny - 1, :] = True
    dcy = cy + R + 0.6 * r
    inside = (x - cx) ** 2 + (y - dcy) ** 2 <= r * r
    solid = solid.astype(np.uint8)
    rA, rB = _phase_fields(inside, solid, seed, amp)
    return Scenario(f"cylinder_droplet_{nx}x{ny}", solid, rA, rB, bc_x="periodic", bc_y="wall",
                    scheme=scheme, tau=tuple(tau), G=G, lam=lam,
                    surface={"kind": "circle", "cx": float(cx), "cy": float(cy), "R": R + 0.5})


def cylinder_in_box(nx: int = 300, ny: int = 350, R: float = 70.0, centre=(150.0, 130.0), r: float = 50.0,
                    drop=(150.0, 230.0), lam: float = 1.0, seed: int = 31, scheme: str = "improved",
                    G: float = G_DEFAULT, Gw2: float | None = GW2_DEFAULT, tau=(1.0, 1.0),
                    rho_m: float = RHO_M, rho_d: float = RHO_D, second_layer: str = "psi_and_solid",
                    adhesion_stencil: str = "e8") -> Scenario:
    """The paper's own Sec. 3.2 geometry (Fig. 5): a 300x350 box periodic in x and y, a solid
    cylinder of radius 70 centred at (150, 130), and a droplet of A of radius 50 centred at
    (150, 230), 0.6 r above the cylinder top.  Gw2 None means G_w2 = G."""
    y, x = _grid(ny, nx)
    solid = ((x - centre[0]) ** 2 + (y - centre[1]) ** 2 <= R * R).astype(np.uint8)
    inside = (x - drop[0]) ** 2 + (y - drop[1]) ** 2 <= r * r
    rA, rB = _phase_fields(inside, solid, seed, rho_m=rho_m, rho_d=rho_d)
    return Scenario(f"cylinder_in_box_{nx}x{ny}", solid, rA, rB, bc_x="periodic", bc_y="periodic",
                    scheme=scheme, tau=tuple(tau), G=G, Gw2=Gw2, lam=lam, rho_in=(rho_m, rho_d),
                    second_layer=second_layer, adhesion_stencil=adhesion_stencil,
                    surface={"kind": "circle", "cx": float(centre[0]), "cy": float(centre[1]), "R": R + 0.5})


# The parameters Sec. 3.2 states for its cylinder case: main / dissolved densities 1.02 / 0.05,
# kinematic viscosity 0.17 (tau = 3 nu + 1/2 = 1.01) and G_w2 = G_12.  G_12 takes the mean-field
# value for those densities in this build's weight normalisation (1.036).
PAPER_SEC32 = {"rho_m": 1.02, "rho_d": 0.05, "tau": (1.01, 1.01), "G": round(mean_field_G(1.02, 0.05), 3),
               "Gw2": None}


def flat_droplet(nx: int = 64, ny: int = 48, r: float = 12.0, lam: float = 1.0, seed: int = 11,
                 scheme: str = "improved", G: float = G_DEFAULT, h: float | None = None,
                 amp: float = NOISE_AMP) -> Scenario:
    """Droplet of A on a flat wall: rows 0 and ny-1 solid, x periodic, droplet of radius r centred
    at (nx/2 - 1/2, 0.6 r) -- mirror-symmetric about x = nx/2 - 1/2 when the noise is off."""
    y, x = _grid(ny, nx)
    solid = np.zeros((ny, nx), bool)
    solid[0, :] = True
    solid[ny - 1, :] = True
    h = 0.6 * r if h is None else h
    inside = (x - (nx - 1) / 2.0) ** 2 + (y - h) ** 2 <= r * r
    solid = solid.astype(np.uint8)
    rA, rB = _phase_fields(inside, solid, seed, amp)
    return Scenario(f"flat_droplet_{nx}x{ny}", solid, rA, rB, bc_x="periodic", bc_y="wall",
                    scheme=scheme, G=G, lam=lam,
                    surface={"kind": "flat", "y_w": 0.5, "normal": 1})


def free_droplet(n: int = 64, R: float = 12.0, seed: int = 21, G: float = G_DEFAULT,
                 amp: float = NOISE_AMP) -> Scenario:
    """Free droplet of A in B, fully periodic, no solid (Laplace-law case)."""
    y, x = _grid(n, n)
    inside = (x - n / 2.0) ** 2 + (y - n / 2.0) ** 2 <= R * R
    solid = np.zeros((n, n), np.uint8)
    rA, rB = _phase_fields(inside, solid, seed, amp)
    return Scenario(f"free_droplet_{n}_R{R:g}", solid, rA, rB, bc_x="periodic", bc_y="periodic", G=G)


def throat_channel(nx: int = 2048, ny: int = 512, R: float = 180.0, r: float = 120.0, seed: int = 3,
                   g: float = 1e-6, lam: float | None = None, G: float = G_DEFAULT) -> Scenario:
    """Droplet through a confined geometry (Sec. 3.3 shape): rows 0, ny-1 solid, x periodic, two
    opposing half-disks of radius R centred at (nx/2, 0) and (nx/2, ny-1), a droplet of radius r at
    (nx*400/2048, ny/2) in B, body force g along x."""
    y, x = _grid(ny, nx)
    solid = ((x - nx / 2) ** 2 + y ** 2 <= R * R) | ((x - nx / 2) ** 2 + (y - (ny - 1)) ** 2 <= R * R)
    solid[0, :] = True
    solid[ny - 1, :] = True
    inside = (x - nx * 400.0 / 2048.0) ** 2 + (y - ny / 2.0) ** 2 <= r * r
    solid = solid.astype(np.uint8)
    rA, rB = _phase_fields(inside, solid, seed)
    lam = lambda_for_angle(90.0) if lam is None else lam
    return Scenario(f"throat_channel_{nx}x{ny}", solid, rA, rB, bc_x="periodic", bc_y="wall",
                    g=(g, 0.0), lam=lam, G=G)


def porous_disks(nx: int = 4096, ny: int = 2048, porosity: float = 0.6, rmin: float = 12.0,
                 rmax: float = 40.0, seed: int = 4, keep_out: tuple = (64, 64), u_in: float = 0.005,
                 G: float = G_DEFAULT, lam: float | None = None, max_tries: int = 2_000_000) -> Scenario:
    """Immiscible displacement in a synthetic porous medium (Sec. 3.4 shape): rows 0, ny-1 solid;
    random non-overlapping disks with radii uniform in [rmin, rmax] placed by rejection sampling
    until the porosity drops to ``porosity``, kept out of the first and last ``keep_out`` columns;
    filled with B; A enters through a velocity inlet at x = 0 (u_in), outflow at x = nx-1."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((ny, nx), bool)
    solid[0, :] = True
    solid[ny - 1, :] = True
    target_solid = (1.0 - porosity) * nx * ny
    cell = int(2 * rmax) + 2
    buckets: dict = {}
    disks = []
    area = float(solid.sum())
    tries = 0
    while area < target_solid and tries < max_tries:
        tries += 1
        rad = rng.uniform(rmin, rmax)
        cx = rng.uniform(keep_out[0] + rad, nx - keep_out[1] - rad)
        cy = rng.uniform(1 + rad, ny - 1 - rad)
        bx, by = int(cx // cell), int(cy // cell)
        ok = True
        for jx in range(bx - 1, bx + 2):
            for jy in range(by - 1, by + 2):
                for (ox, oy, orad) in buckets.get((jx, jy), ()):
                    if (cx - ox) ** 2 + (cy - oy) ** 2 < (rad + orad + 1.0) ** 2:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        buckets.setdefault((bx, by), []).append((cx, cy, rad))
        disks.append((cx, cy, rad))
        x0, x1 = int(max(0, cx - rad - 1)), int(min(nx, cx + rad + 2))
        y0, y1 = int(max(0, cy - rad - 1)), int(min(ny, cy + rad + 2))
        yy, xx = np.mgrid[y0:y1, x0:x1]
        m = (xx - cx) ** 2 + (yy - cy) ** 2 <= rad * rad
        area += float((m & ~solid[y0:y1, x0:x1]).sum())
        solid[y0:y1, x0:x1] |= m
    solid = solid.astype(np.uint8)
    inside = np.zeros((ny, nx), bool)
    rA, rB = _phase_fields(inside, solid, seed)
    lam = lambda_for_angle(45.0) if lam is None else lam
    return Scenario(f"porous_disks_{nx}x{ny}", solid, rA, rB, bc_x="open", bc_y="wall",
                    tau=(0.8, 1.0), u_in=u_in, rho_in=(RHO_M, RHO_D), lam=lam, G=G,
                    extra={"n_disks": len(disks)})


def cocurrent_channel(nx: int = 4096, ny: int = 256, frac_A: float = 0.4, g: float = 1e-6,
                      lam: float | None = None, seed: int = 5, G: float = G_DEFAULT,
                      amp: float = NOISE_AMP) -> Scenario:
    """Co-current stratified flow (Sec. 3.1 shape): rows 0, ny-1 solid, x periodic, A in the bottom
    ``frac_A`` of the channel, B above, body force g along x."""
    y, x = _grid(ny, nx)
    solid = np.zeros((ny, nx), bool)
    solid[0, :] = True
    solid[ny - 1, :] = True
    inside = y < frac_A * ny
    solid = solid.astype(np.uint8)
    rA, rB = _phase_fields(inside, solid, seed, amp)
    lam = lambda_for_angle(120.0) if lam is None else lam
    return Scenario(f"cocurrent_{nx}x{ny}", solid, rA, rB, bc_x="periodic", bc_y="wall",
                    g=(g, 0.0), lam=lam, G=G)


NU_SEC3 = 0.17                   # kinematic viscosity of both fluids in Secs. 3.1 and 3.3
TAU_SEC3 = 3.0 * NU_SEC3 + 0.5    # nu = c_s^2 (tau - 1/2)


def couette_channel(nx: int = 50, ny: int = 100, U: float = 0.005, lam: float | None = None,
                    seed: int = 7, G: float = G_DEFAULT, scheme: str = "improved",
                    amp: float = NOISE_AMP, Gw2: float | None = GW2_DEFAULT, rho_m: float = RHO_M,
                    rho_d: float = RHO_D) -> Scenario:
    """Two-layer Couette flow (Sec. 3.1, Fig. 3b): x periodic, walls half a cell below row 0 and
    above row ny-1 sliding at -U (lower) and +U (upper); A in the central half of the channel
    (|y - H/2| <= H/4), B next to both walls; nu = 0.17 for both fluids."""
    y, x = _grid(ny, nx)
    solid = np.zeros((ny, nx), np.uint8)
    s = y + 0.5
    inside = np.abs(s - ny / 2.0) <= ny / 4.0
    rA, rB = _phase_fields(inside, solid, seed, amp, rho_m=rho_m, rho_d=rho_d)
    lam = lambda_for_angle(90.0) if lam is None else lam
    return Scenario(f"couette_{nx}x{ny}", solid, rA, rB, bc_x="periodic", bc_y="wall", scheme=scheme,
                    tau=(TAU_SEC3, TAU_SEC3), G=G, Gw2=Gw2, lam=lam, u_wall=(-U, U), rho_in=(rho_m, rho_d))


def poiseuille_channel(nx: int = 50, ny: int = 100, g: float = 1e-6, lam: float | None = None,
                       seed: int = 17, G: float = G_DEFAULT, scheme: str = "improved",
                       amp: float = NOISE_AMP, Gw2: float | None = GW2_DEFAULT, rho_m: float = RHO_M,
                       rho_d: float = RHO_D) -> Scenario:
    """Two-layer Poiseuille flow (Sec. 3.1, Fig. 3a): the Couette channel's layers between walls
    at rest, driven by the body acceleration g along x on both components."""
    sc = couette_channel(nx, ny, 0.0, lam, seed, G, scheme, amp, Gw2, rho_m, rho_d)
    sc.name = f"poiseuille_{nx}x{ny}"
    sc.u_wall = (0.0, 0.0)
    sc.g = (g, 0.0)
    return sc


def square_obstacle_channel(nx: int = 350, ny: int = 150, side: int = 25, center=(122, 75), r: float = 25.0,
                            drop=(55, 75), Re: float = 7.5, theta: float = 30.2, seed: int = 8,
                            G: float = G_DEFAULT, scheme: str = "improved", amp: float = NOISE_AMP,
                            Gw2: float | None = GW2_DEFAULT) -> Scenario:
    """Droplet driven past a square obstacle in a microchannel (Sec. 3.3, Fig. 12): walls half a
    cell below row 0 and above row ny-1; a square of the given side centred at ``center``; a
    droplet of A (radius r) at ``drop``, B elsewhere; a velocity inlet at x = 0 with the Poiseuille
    profile of peak U_m (fluid B enters), outflow at x = nx-1; nu = 0.17; lambda for the static
    angle ``theta`` on the square.  U_m from Re = U_m (2 r) / nu."""
    y, x = _grid(ny, nx)
    h = side / 2.0
    solid = ((np.abs(x - center[0]) < h) & (np.abs(y - center[1]) < h)).astype(np.uint8)
    inside = (x - drop[0]) ** 2 + (y - drop[1]) ** 2 <= r * r
    rA, rB = _phase_fields(inside, solid, seed, amp)
    Um = Re * NU_SEC3 / (2.0 * r)
    return Scenario(f"square_obstacle_{nx}x{ny}", solid, rA, rB, bc_x="open", bc_y="wall", scheme=scheme,
                    tau=(TAU_SEC3, TAU_SEC3), G=G, Gw2=Gw2, lam=lambda_for_angle(theta), u_in=Um,
                    rho_in=(RHO_D, RHO_M), inlet_profile="poiseuille")


def ensemble_cases(ncases: int = 256, nmin: int = 64, nmax: int = 512, seed: int = 5,
                   lam_range=(0.22, 2.17), G: float = G_DEFAULT) -> list:
    """Uneven contact-angle ensemble: square cases of side n ~ U{nmin..nmax}, half flat wall and
    half cylinder (R = n/6, droplet r = n/5 centred 0.6 r above the solid top), lambda uniform in
    ``lam_range``."""
    rng = np.random.default_rng(seed)
    cases = []
    for c in range(ncases):
        n = int(rng.integers(nmin, nmax + 1))
        lam = float(rng.uniform(*lam_range))
        if c % 2 == 0:
            sc = flat_droplet(nx=n, ny=n, r=n / 5.0, lam=lam, seed=seed * 1000 + c, G=G)
        else:
            sc = cylinder_droplet(n=n, R=n / 6.0, r=n / 5.0, lam=lam, seed=seed * 1000 + c, G=G)
        sc.name = f"case{c:03d}_{sc.name}"
        cases.append(sc)
    return cases


def lambda_sweep_cylinder(n: int = 1024, seed: int = 2, angles=(30, 50, 70, 90, 110, 130, 150),
                          G: float = G_DEFAULT, scheme: str = "improved") -> list:
    """The 1024x1024 cylinder contact-angle sweep: one case per target angle, lambda from the
    paper's correlation (Sec. 3.2), cylinder radius 160 and droplet radius 200 at n = 1024."""
    out = []
    for k, th in enumerate(angles):
        sc = cylinder_droplet(n=n, R=160.0 * n / 1024.0, r=200.0 * n / 1024.0,
                              lam=lambda_for_angle(th), seed=seed * 100 + k, G=G, scheme=scheme)
        sc.name = f"sweep_theta{th}_{sc.name}"
        out.append(sc)
    return out


def scheme_comparison(n: int = 1024, seed: int = 2, angles=(30, 50, 70, 90, 110, 130, 150),
                      G: float = G_DEFAULT) -> list:
    """The cylinder sweep under both solid-fluid schemes (Secs. 2.3, 3.2): the improved scheme's
    cases, then the original scheme's on the same geometries and initial states (G_w1 = lambda
    G_w2 everywhere), for the comparison of spurious currents and density extrema."""
    out = []
    for scheme in ("improved", "original"):
        for sc in lambda_sweep_cylinder(n, seed, angles, G, scheme=scheme):
            sc.name = f"{scheme}_{sc.name}"
            out.append(sc)
    return out


def scheme_study(angles=(30, 50, 70, 90, 110, 130, 150), seed: int = 31, paper_params: bool = False,
                 Gw2: float | None = -1.0, second_layer: str = "psi_and_solid", adhesion_stencil: str = "e8") -> list:
    """The comparison of Sec. 3.2 (Figs. 6, 10, 11) on the paper's 300x350 geometry: one case per
    target angle (lambda from the correlation) under the improved scheme, then the same geometries
    and initial states under the original scheme (G_w1 = lambda G_w2 everywhere).  paper_params
    takes the densities, viscosity and G_w2 = G_12 of Sec. 3.2 (PAPER_SEC32) in place of this
    build's defaults; Gw2 >= 0 (or None: G_w2 = G) overrides G_w2."""
    extra = dict(PAPER_SEC32) if paper_params else {}
    if Gw2 is None or Gw2 >= 0:
        extra["Gw2"] = Gw2
    extra["second_layer"] = second_layer
    extra["adhesion_stencil"] = adhesion_stencil
    out = []
    for scheme in ("improved", "original"):
        for k, th in enumerate(angles):
            sc = cylinder_in_box(lam=lambda_for_angle(th), seed=seed * 100 + k, scheme=scheme, **extra)
            sc.name = f"{scheme}_theta{th}_{sc.name}"
            sc.extra["target_theta"] = float(th)
            out.append(sc)
    return out


# ------------------------------------------------------------------------------------------------
# 3-D (Sec. 3.5): a droplet on a solid sphere, periodic in x, y and z
# ------------------------------------------------------------------------------------------------
@dataclass
class Scenario3:
    """One 3-D lattice case: mask and initial densities [nz][ny][nx], parameters, the sphere."""
    name: str
    solid: np.ndarray
    rhoA0: np.ndarray
    rhoB0: np.ndarray
    tau: tuple = (TAU_SEC3, TAU_SEC3)
    G: float = G_DEFAULT
    lam: float = 1.0
    Gw2: float | None = GW2_DEFAULT
    delta: float = 0.8
    g: tuple = (0.0, 0.0, 0.0)
    scheme: str = "improved"
    sphere: dict | None = None   # {"c": (x, y, z), "R": effective radius} for the contact angle
    second_layer: str = "psi_and_solid"  # or "psi" (Sec. 2.4, Table 1)
    adhesion_stencil: str = "e8"  # or "d3q19": Eq. 9 as printed, first layer, D3Q19 weights
    # 16-bit storage keeps f_i - w_i rho0 per component; the dissolved-phase density serves both
    rho0_store: tuple = (RHO_D, RHO_D)

    @property
    def shape(self):
        return self.solid.shape

    def params(self) -> dict:
        return dict(tau=tuple(self.tau), G=self.G, scheme=self.scheme, lam=self.lam, Gw2=self.Gw2,
                    delta=self.delta, g=tuple(self.g), second_layer=self.second_layer,
                    adhesion_stencil=self.adhesion_stencil, rho0_store=tuple(self.rho0_store))


def sphere_droplet_3d(nx: int = 200, ny: int = 200, nz: int = 280, R: float = 50.0, sphere=(100.0, 100.0, 100.0),
                      r: float = 45.0, drop=(100.0, 100.0, 180.0), lam: float = 1.0, seed: int = 9,
                      G: float = G_DEFAULT, scheme: str = "improved", amp: float = NOISE_AMP) -> Scenario3:
    """Sec. 3.5: a droplet of A (radius r, centre ``drop``) on a solid sphere (radius R, centre
    ``sphere``), B elsewhere, periodic in every direction; the paper's 200x200x280 grid by default
    (lambda = 0.38, 1, 2.1 for theta ~ 45, 90, 146 degrees).  Noise as in 2-D, counter over the
    node index z (ny nx) + y nx + x."""
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    solid = ((x - sphere[0]) ** 2 + (y - sphere[1]) ** 2 + (z - sphere[2]) ** 2 <= R * R).astype(np.uint8)
    inside = (x - drop[0]) ** 2 + (y - drop[1]) ** 2 + (z - drop[2]) ** 2 <= r * r
    rA = np.where(inside, RHO_M, RHO_D) + node_noise(seed, nz * ny, nx, 0, amp).reshape(nz, ny, nx)
    rB = np.where(inside, RHO_D, RHO_M) + node_noise(seed, nz * ny, nx, 1, amp).reshape(nz, ny, nx)
    rA[solid == 1] = 0.0
    rB[solid == 1] = 0.0
    return Scenario3(f"sphere_droplet_{nx}x{ny}x{nz}", solid, rA, rB, G=G, lam=lam, scheme=scheme,
                     sphere={"c": tuple(sphere), "R": R + 0.5})


def sphere_droplet_3d_small(n: int = 40, lam: float = 1.0, seed: int = 9, scheme: str = "improved",
                            amp: float = NOISE_AMP) -> Scenario3:
    """The Sec. 3.5 geometry scaled to an n x n x 1.4n box (R = n/4, r = 0.225 n, centres as in the
    paper scaled by n/200)."""
    k = n / 200.0
    return sphere_droplet_3d(nx=n, ny=n, nz=int(round(1.4 * n)), R=50 * k, sphere=(100 * k, 100 * k, 100 * k),
                             r=45 * k, drop=(100 * k, 100 * k, 180 * k), lam=lam, seed=seed, scheme=scheme, amp=amp)
