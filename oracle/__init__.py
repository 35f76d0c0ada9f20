"""Plain FP64 CPU oracle for the two-component pseudopotential LBM time step of arXiv 2505.22256.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package; the CUDA product path never imports, links or runs it, and the two
share no code.  Everything here is double precision and written for checking by eye against the
paper:

* ``lbm_oracle.c`` -- one time step, node by node, in the paper's order (Eqs. 1-12, Sec. 2.4
  second-layer copy of Table 1, halfway bounce-back of Sec. 3.5, the open boundaries of Sec. 3.3);
* this module -- the derivation of the eighth-order isotropic (E8) weights from their defining
  moment conditions (Sec. 2.4, refs. [20,35,36] of the paper), the global diagnostics used for
  Figs. 10-11 (maximum spurious velocity, density extrema) and mass, and the contact-angle
  measurement of Sec. 3.2 (the paper does not say how it measured angles; the reading used here is
  an algebraic circle fit to the rho^e = 0 contour, refined by one Gauss-Newton step).

Pins: ``tests/test_oracle_*.py`` (closed forms, invariants, brute force and the paper's own
coefficient definitions).  Parity pinned for every function here except where a docstring says
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")

BC_PERIODIC, BC_WALL, BC_OPEN = 0, 1, 2
SCHEME_ORIGINAL, SCHEME_IMPROVED = 0, 1
_BC_NAMES = {"periodic": BC_PERIODIC, "wall": BC_WALL, "open": BC_OPEN}


# ------------------------------------------------------------------------------------------------
# build / load
# ------------------------------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` with gcc into ``oracle/_build/liblbm_oracle.so``.

    ``-ffp-contract=off`` keeps every multiply and add separately rounded, so x86 and Arm hosts give
    the same doubles.  OpenMP parallelises the node loops only (every node is independent); the
    library is rebuilt without it if the compiler lacks it."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _SO, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        cp = ctypes.POINTER(_Cfg)
        lib.oracle_feq.argtypes = [ctypes.c_double] * 3 + [dp]
        lib.oracle_guo.argtypes = [ctypes.c_double] * 4 + [dp]
        lib.oracle_local_G.argtypes = [ctypes.c_double] * 3
        lib.oracle_local_G.restype = ctypes.c_double
        lib.oracle_e8_table.argtypes = [ctypes.POINTER(ctypes.c_int32)] * 2
        lib.oracle_wall_list.argtypes = [cp, u8p, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_uint32), dp, dp]
        lib.oracle_wall_list.restype = ctypes.c_int64
        lib.oracle_init.argtypes = [cp, u8p, dp, dp, dp]
        lib.oracle_collide.argtypes = [cp, u8p, dp, dp]
        lib.oracle_stream.argtypes = [cp, u8p, dp, dp]
        lib.oracle_run.argtypes = [cp, u8p, dp, dp, ctypes.c_int64]
        lib.oracle_fields.argtypes = [cp, u8p, dp, dp, dp, dp, dp]
        lib.oracle_forces.argtypes = [cp, u8p, dp, dp, dp, dp, dp]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


# ------------------------------------------------------------------------------------------------
# E8 weights (Sec. 2.4): derived from the moment conditions, exactly, in rational arithmetic
# ------------------------------------------------------------------------------------------------
SHELLS = (1, 2, 4, 5, 8)


def e8_offsets():
    """The oracle's 24 stencil offsets in the numbering of Fig. 2(a) / Table 1 (1-8 first layer)."""
    ex = (ctypes.c_int32 * 24)()
    ey = (ctypes.c_int32 * 24)()
    _load().oracle_e8_table(ex, ey)
    return [(int(ex[n]), int(ey[n])) for n in range(24)]


def e8_weights() -> dict:
    """Weights w(|e|^2) of the eighth-order isotropic stencil over the 5x5 neighbourhood.

    They are the unique solution of five linear conditions on the lattice moments
    M(a, b) = sum_e w(|e|^2) e_x^a e_y^b: normalisation M(2,0) = 1 and isotropy of the 4th, 6th and
    8th order moment tensors (M(4,0) = 3 M(2,2); M(6,0) = 5 M(4,2); M(8,0) = 7 M(6,2);
    5 M(4,4) = 3 M(6,2)), solved by exact Gaussian elimination over the rationals."""
    offs = [(dx, dy) for dy in range(-2, 3) for dx in range(-2, 3) if (dx, dy) != (0, 0)]

    def mom(q, a, b):
        return sum(Fraction(dx) ** a * Fraction(dy) ** b for dx, dy in offs if dx * dx + dy * dy == q)

    rows = []
    rows.append([mom(q, 2, 0) for q in SHELLS] + [Fraction(1)])
    rows.append([mom(q, 4, 0) - 3 * mom(q, 2, 2) for q in SHELLS] + [Fraction(0)])
    rows.append([mom(q, 6, 0) - 5 * mom(q, 4, 2) for q in SHELLS] + [Fraction(0)])
    rows.append([mom(q, 8, 0) - 7 * mom(q, 6, 2) for q in SHELLS] + [Fraction(0)])
    rows.append([5 * mom(q, 4, 4) - 3 * mom(q, 6, 2) for q in SHELLS] + [Fraction(0)])
    n = len(SHELLS)
    for col in range(n):
        piv = next(r for r in range(col, n) if rows[r][col] != 0)
        rows[col], rows[piv] = rows[piv], rows[col]
        for r in range(n):
            if r != col and rows[r][col] != 0:
                fac = rows[r][col] / rows[col][col]
                rows[r] = [a - fac * b for a, b in zip(rows[r], rows[col])]
    return {q: rows[i][n] / rows[i][i] for i, q in enumerate(SHELLS)}


# ------------------------------------------------------------------------------------------------
# configuration
# ------------------------------------------------------------------------------------------------
class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc_x", ctypes.c_int32),
                ("bc_y", ctypes.c_int32), ("scheme", ctypes.c_int32), ("nthreads", ctypes.c_int32),
                ("tau", ctypes.c_double * 2), ("G", ctypes.c_double), ("lam", ctypes.c_double),
                ("Gw2", ctypes.c_double), ("delta", ctypes.c_double), ("g", ctypes.c_double * 2),
                ("u_in", ctypes.c_double), ("rho_in", ctypes.c_double * 2),
                ("wE8", ctypes.c_double * 5), ("inlet_profile", ctypes.c_int32), ("second_layer", ctypes.c_int32),
                ("u_wall", ctypes.c_double * 2), ("adhesion_stencil", ctypes.c_int32), ("outlet", ctypes.c_int32),
                ("rho_out", ctypes.c_double * 2)]


@dataclass
class Config:
    """Model parameters (names follow the paper; see ``lbm_oracle.c`` for each one's passage)."""
    nx: int
    ny: int
    bc_x: str = "periodic"          # periodic | wall | open
    bc_y: str = "wall"              # periodic | wall
    scheme: str = "improved"        # improved (Eqs. 10-12) | original (Eq. 9)
    tau: tuple = (1.0, 1.0)
    G: float = 3.5
    lam: float = 1.0
    Gw2: float | None = None        # defaults to G (the paper's G_w2 = G_12)
    delta: float = 0.8
    g: tuple = (0.0, 0.0)
    u_in: float = 0.0
    rho_in: tuple = (1.0, 0.03)
    inlet_profile: str = "uniform"  # uniform | poiseuille (peak u_in; Sec. 3.3)
    u_wall: tuple = (0.0, 0.0)      # x-velocity of the lower / upper wall of a walled y (Sec. 3.1)
    # what a replaced second-layer node takes from x + sign(e) (Sec. 2.4, Table 1): "psi_and_solid"
    # or "psi" (the non-fluid site keeps its solid switch in the adhesion sum)
    second_layer: str = "psi_and_solid"
    # stencil of the adhesion sum of Eq. 9: "e8" (the 24-node stencil of the cohesion force, Sec. 2.4)
    # or "d2q9" (as printed: D2Q9 weights w_i over the eight first-layer neighbours)
    adhesion_stencil: str = "e8"
    # outflow at x = nx-1 (Sec. 3.3): "copy" (entering populations from column nx-2) or "pressure"
    # (Zou-He density condition holding rho_out per component)
    outlet: str = "copy"
    rho_out: tuple = (0.03, 1.0)
    nthreads: int = field(default_factory=lambda: int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)))

    def c(self) -> _Cfg:
        w = e8_weights()
        s = _Cfg()
        s.nx, s.ny = self.nx, self.ny
        s.bc_x, s.bc_y = _BC_NAMES[self.bc_x], _BC_NAMES[self.bc_y]
        s.scheme = SCHEME_IMPROVED if self.scheme == "improved" else SCHEME_ORIGINAL
        s.nthreads = max(1, int(self.nthreads))
        s.tau[0], s.tau[1] = self.tau
        s.G, s.lam = self.G, self.lam
        s.Gw2 = self.G if self.Gw2 is None else self.Gw2
        s.delta = self.delta
        s.g[0], s.g[1] = self.g
        s.u_in = self.u_in
        s.rho_in[0], s.rho_in[1] = self.rho_in
        s.inlet_profile = {"uniform": 0, "poiseuille": 1}[self.inlet_profile]
        s.u_wall[0], s.u_wall[1] = self.u_wall
        s.second_layer = {"psi_and_solid": 0, "psi": 1}[self.second_layer]
        s.adhesion_stencil = {"e8": 0, "d2q9": 1}[self.adhesion_stencil]
        s.outlet = {"copy": 0, "pressure": 1}[self.outlet]
        s.rho_out[0], s.rho_out[1] = self.rho_out
        for i, q in enumerate(SHELLS):
            s.wE8[i] = float(w[q])
        return s


def _solid(cfg: Config, solid) -> np.ndarray:
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    assert s.shape == (cfg.ny, cfg.nx)
    return s


# ------------------------------------------------------------------------------------------------
# node-level building blocks (for the pins)
# ------------------------------------------------------------------------------------------------
def feq(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    _load().oracle_feq(rho, ux, uy, _dp(out))
    return out


def guo(ux, uy, Fx, Fy) -> np.ndarray:
    out = np.zeros(9)
    _load().oracle_guo(ux, uy, Fx, Fy, _dp(out))
    return out


def local_G(rho_e, lam, delta=0.8) -> float:
    """G_w1(x) / G_w2 of Eq. 12."""
    return float(_load().oracle_local_G(rho_e, lam, delta))


# ------------------------------------------------------------------------------------------------
# whole-lattice operations
# ------------------------------------------------------------------------------------------------
def init(cfg: Config, solid, rhoA0, rhoB0) -> np.ndarray:
    """f = f^eq(rho_k, 0) at fluid nodes (state shape (2, 9, ny, nx))."""
    s = _solid(cfg, solid)
    f = np.zeros((2, 9, cfg.ny, cfg.nx))
    rA = np.ascontiguousarray(rhoA0, dtype=np.float64)
    rB = np.ascontiguousarray(rhoB0, dtype=np.float64)
    _load().oracle_init(ctypes.byref(cfg.c()), _u8(s), _dp(rA), _dp(rB), _dp(f))
    return f


def collide(cfg: Config, solid, f) -> np.ndarray:
    s = _solid(cfg, solid)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    if _load().oracle_collide(ctypes.byref(cfg.c()), _u8(s), _dp(f), _dp(out)):
        raise MemoryError("oracle_collide")
    return out


def stream(cfg: Config, solid, fstar) -> np.ndarray:
    s = _solid(cfg, solid)
    fstar = np.ascontiguousarray(fstar, dtype=np.float64)
    out = np.empty_like(fstar)
    _load().oracle_stream(ctypes.byref(cfg.c()), _u8(s), _dp(fstar), _dp(out))
    return out


def run(cfg: Config, solid, f, nsteps: int) -> np.ndarray:
    """n time steps (collide then stream), returning the new post-streaming state."""
    s = _solid(cfg, solid)
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    scratch = np.empty_like(f)
    if _load().oracle_run(ctypes.byref(cfg.c()), _u8(s), _dp(f), _dp(scratch), int(nsteps)):
        raise MemoryError("oracle_run")
    return f


def fields(cfg: Config, solid, f):
    """(rho_A, rho_B, u_x, u_y) at the current state; u includes the half-force shift."""
    s = _solid(cfg, solid)
    f = np.ascontiguousarray(f, dtype=np.float64)
    outs = [np.zeros((cfg.ny, cfg.nx)) for _ in range(4)]
    _load().oracle_fields(ctypes.byref(cfg.c()), _u8(s), _dp(f), *[_dp(o) for o in outs])
    return tuple(outs)


def forces(cfg: Config, solid, f):
    """(F_A, F_B) as arrays of shape (2, ny, nx): total force per component (step 5)."""
    s = _solid(cfg, solid)
    f = np.ascontiguousarray(f, dtype=np.float64)
    outs = [np.zeros((cfg.ny, cfg.nx)) for _ in range(4)]
    if _load().oracle_forces(ctypes.byref(cfg.c()), _u8(s), _dp(f), *[_dp(o) for o in outs]):
        raise MemoryError("oracle_forces")
    return np.stack(outs[:2]), np.stack(outs[2:])


def wall_list(cfg: Config, solid):
    """(node, subst, seff, ax, ay): the wall list of step a1, sorted by node index y*nx + x."""
    s = _solid(cfg, solid)
    lib = _load()
    c = cfg.c()
    n = lib.oracle_wall_list(ctypes.byref(c), _u8(s), None, None, None, None, None)
    if n < 0:
        raise MemoryError("oracle_wall_list")
    node = np.zeros(n, np.int32)
    subst = np.zeros(n, np.uint32)
    seff = np.zeros(n, np.uint32)
    ax = np.zeros(n)
    ay = np.zeros(n)
    lib.oracle_wall_list(ctypes.byref(c), _u8(s), node.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         subst.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                         seff.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _dp(ax), _dp(ay))
    return node, subst, seff, ax, ay


# ------------------------------------------------------------------------------------------------
# measurements (Sec. 3.2): diagnostics and contact angle
# ------------------------------------------------------------------------------------------------
def diagnostics(cfg: Config, solid, f) -> dict:
    """Global FP64 diagnostics over fluid nodes: per-component mass, total momentum
    sum (rho_A + rho_B) u, maximum |u| (the spurious-current measure of Fig. 10) and per-component
    density extrema (Fig. 11)."""
    s = _solid(cfg, solid).astype(bool)
    rA, rB, ux, uy = fields(cfg, solid, f)
    fl = ~s
    rho = rA + rB
    return {
        "mass_A": float(np.sum(rA[fl])), "mass_B": float(np.sum(rB[fl])),
        "mom_x": float(np.sum((rho * ux)[fl])), "mom_y": float(np.sum((rho * uy)[fl])),
        "umax": float(np.max(np.hypot(ux, uy)[fl])),
        "rhoA_min": float(rA[fl].min()), "rhoA_max": float(rA[fl].max()),
        "rhoB_min": float(rB[fl].min()), "rhoB_max": float(rB[fl].max()),
    }


def near_solid(cfg: Config, solid, margin: int = 3) -> np.ndarray:
    """Nodes with a non-fluid site (solid, or outside the array along a non-periodic direction)
    in the (2*margin+1)^2 box around them."""
    s = _solid(cfg, solid).astype(bool)
    ny, nx = s.shape
    m = margin
    # embed in a frame of width m: periodic directions wrap, others are non-fluid
    ext = np.pad(s, ((m, m), (m, m)), mode="constant", constant_values=True)
    if cfg.bc_x == "periodic":
        ext[:, :m] = ext[:, nx:nx + m]
        ext[:, nx + m:] = ext[:, m:2 * m]
    if cfg.bc_y == "periodic":
        ext[:m, :] = ext[ny:ny + m, :]
        ext[ny + m:, :] = ext[m:2 * m, :]
    out = np.zeros_like(s)
    for dy in range(-m, m + 1):
        for dx in range(-m, m + 1):
            out |= ext[m + dy:m + dy + ny, m + dx:m + dx + nx]
    return out


def interface_points(cfg: Config, solid, rhoA, rhoB, margin: int = 3) -> np.ndarray:
    """Points where the effective density rho^e = (rho_A - rho_B)/(rho_A + rho_B) (Eq. 10) changes
    sign along a lattice row or column, linearly interpolated between the two nodes.  A crossing is
    kept only when both nodes are fluid and more than ``margin`` cells (Chebyshev) from any
    non-fluid site.  Pairs across a periodic seam are not used.  Horizontal crossings first (row
    by row), then vertical ones."""
    s = _solid(cfg, solid).astype(bool)
    ok = ~s & ~near_solid(cfg, solid, margin)
    phi = np.where(s, 0.0, (rhoA - rhoB) / np.where(s, 1.0, rhoA + rhoB))
    a, b = phi[:, :-1], phi[:, 1:]
    hmask = ok[:, :-1] & ok[:, 1:] & ((a > 0) != (b > 0))
    hy, hx = np.nonzero(hmask)
    hpts = np.stack([hx + a[hy, hx] / (a[hy, hx] - b[hy, hx]), hy.astype(np.float64)], axis=1)
    a, b = phi[:-1, :], phi[1:, :]
    vmask = ok[:-1, :] & ok[1:, :] & ((a > 0) != (b > 0))
    vy, vx = np.nonzero(vmask)
    vpts = np.stack([vx.astype(np.float64), vy + a[vy, vx] / (a[vy, vx] - b[vy, vx])], axis=1)
    return np.concatenate([hpts, vpts]).reshape(-1, 2)


def fit_circle(pts: np.ndarray):
    """Algebraic (Kasa) circle fit in centroid coordinates, followed by one Gauss-Newton step on
    the geometric residuals |p - c| - r.  Returns (cx, cy, r, rms residual after the step)."""
    x, y = pts[:, 0], pts[:, 1]
    xm, ym = x.mean(), y.mean()
    u, v = x - xm, y - ym
    Suu, Suv, Svv = np.sum(u * u), np.sum(u * v), np.sum(v * v)
    rhs = 0.5 * np.array([np.sum(u ** 3) + np.sum(u * v * v), np.sum(v ** 3) + np.sum(v * u * u)])
    uc, vc = np.linalg.solve(np.array([[Suu, Suv], [Suv, Svv]]), rhs)
    r = np.sqrt(uc * uc + vc * vc + (Suu + Svv) / len(x))
    cx, cy = xm + uc, ym + vc
    d = np.hypot(x - cx, y - cy)
    res = d - r
    J = np.stack([-(x - cx) / d, -(y - cy) / d, -np.ones_like(x)], axis=1)
    step = np.linalg.solve(J.T @ J, -J.T @ res)
    cx, cy, r = cx + step[0], cy + step[1], r + step[2]
    rms = float(np.sqrt(np.mean((np.hypot(x - cx, y - cy) - r) ** 2)))
    return float(cx), float(cy), float(r), rms


def contact_angle_from_circle(cx, cy, r, surface: dict) -> float:
    """Contact angle in degrees, measured through the droplet (component A), from the fitted
    droplet circle.  cos(theta) is the dot product of the droplet's outward normal and the solid's
    normal pointing into the fluid at the contact point:
      flat wall y = y_w with fluid on the side ``normal`` (+1 above, -1 below):
          cos(theta) = -normal * (cy - y_w) / r;
      circular solid of centre (sx, sy), radius R (halfway bounce-back: R = disk radius + 0.5):
          cos(theta) = (R^2 + r^2 - d^2) / (2 r R), d = distance between the centres."""
    if surface["kind"] == "flat":
        c = -surface.get("normal", 1) * (cy - surface["y_w"]) / r
    else:
        R = surface["R"]
        d2 = (cx - surface["cx"]) ** 2 + (cy - surface["cy"]) ** 2
        c = (R * R + r * r - d2) / (2.0 * r * R)
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def contact_angle(cfg: Config, solid, f, surface: dict, margin: int = 3):
    """(theta_deg, fit_rms, n_points) of the droplet at the current state."""
    rA, rB, _, _ = fields(cfg, solid, f)
    pts = interface_points(cfg, solid, rA, rB, margin)
    cx, cy, r, rms = fit_circle(pts)
    return contact_angle_from_circle(cx, cy, r, surface), rms, len(pts)
