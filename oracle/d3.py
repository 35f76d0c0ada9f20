"""Plain FP64 CPU oracle for the three-dimensional form of the time step (arXiv 2505.22256,
Sec. 3.5: static contact angles on a spherical surface).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the test-suite, ``__graft_entry__`` and the
CPU-baseline leg of ``bench.py`` use it; the CUDA product path never imports, links or runs it.

* ``lbm_oracle3d.c`` -- the step node by node (D3Q19; the 92-offset eighth-order gradient stencil
  with the second-layer copy x + sign(e); cohesion, adhesion with the local parameter of
  Eqs. 10-12, Guo-forced SRT collision, halfway bounce-back; periodic in x, y and z).  The readings
  the paper leaves open in 3-D are listed at the top of that file.
* this module -- the stencil weights from their moment conditions (exact rational solve), the
  diagnostics, and the contact angle on a sphere: rho^e = 0 crossings along the three lattice
  directions away from the solid, an algebraic sphere fit refined by one Gauss-Newton step, and
  cos(theta) = (R^2 + r^2 - d^2) / (2 r R) between the droplet sphere (r) and the solid sphere (R).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle3d.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle3d.so")

SHELLS3 = (1, 2, 3, 4, 5, 6, 8)
SCHEME_ORIGINAL, SCHEME_IMPROVED = 0, 1

# D3Q19 in the order of lbm_oracle3d.c (kept here for the pins; the C file has its own copy)
E19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0),
       (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1),
       (0, -1, 1)]


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle3d.c`` (gcc, -ffp-contract=off, OpenMP over planes when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _SO, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _SO


def stencil_offsets():
    """The 92 offsets e with |e|_inf <= 2 and |e|^2 in SHELLS3."""
    return [e for e in itertools.product(range(-2, 3), repeat=3) if sum(t * t for t in e) in SHELLS3]


def e8_weights_3d() -> dict:
    """Weights w(|e|^2) of eighth-order isotropy on the 92-offset stencil: the unique solution of
    seven linear conditions on M(a, b, c) = sum_e w e_x^a e_y^b e_z^c -- normalisation M(2,0,0) = 1
    and the isotropic ratios of the 4th, 6th and 8th order moments (M(4,0,0) = 3 M(2,2,0);
    M(6,0,0) = 5 M(4,2,0), M(4,2,0) = 3 M(2,2,2); M(8,0,0) = 7 M(6,2,0), 3 M(6,2,0) = 5 M(4,4,0),
    M(4,4,0) = 3 M(4,2,2)), solved by exact Gaussian elimination over the rationals."""
    offs = [e for e in itertools.product(range(-2, 3), repeat=3) if e != (0, 0, 0)]

    def mom(q, a, b, c):
        return sum(Fraction(x) ** a * Fraction(y) ** b * Fraction(z) ** c for x, y, z in offs
                   if x * x + y * y + z * z == q)

    conds = [(lambda q: mom(q, 2, 0, 0), 1),
             (lambda q: mom(q, 4, 0, 0) - 3 * mom(q, 2, 2, 0), 0),
             (lambda q: mom(q, 6, 0, 0) - 5 * mom(q, 4, 2, 0), 0),
             (lambda q: mom(q, 4, 2, 0) - 3 * mom(q, 2, 2, 2), 0),
             (lambda q: mom(q, 8, 0, 0) - 7 * mom(q, 6, 2, 0), 0),
             (lambda q: 3 * mom(q, 6, 2, 0) - 5 * mom(q, 4, 4, 0), 0),
             (lambda q: mom(q, 4, 4, 0) - 3 * mom(q, 4, 2, 2), 0)]
    rows = [[fn(q) for q in SHELLS3] + [Fraction(r)] for fn, r in conds]
    n = len(SHELLS3)
    for col in range(n):
        piv = next(r for r in range(col, n) if rows[r][col] != 0)
        rows[col], rows[piv] = rows[piv], rows[col]
        for r in range(n):
            if r != col and rows[r][col] != 0:
                fac = rows[r][col] / rows[col][col]
                rows[r] = [a - fac * b for a, b in zip(rows[r], rows[col])]
    return {q: rows[i][n] / rows[i][i] for i, q in enumerate(SHELLS3)}


class _Cfg3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("nthreads", ctypes.c_int32), ("second_layer", ctypes.c_int32),
                ("adhesion_stencil", ctypes.c_int32), ("pad_", ctypes.c_int32), ("tau", ctypes.c_double * 2), ("G", ctypes.c_double), ("lam", ctypes.c_double),
                ("Gw2", ctypes.c_double), ("delta", ctypes.c_double), ("g", ctypes.c_double * 3),
                ("w", ctypes.c_double * 7)]


@dataclass
class Config3:
    """Model parameters of the 3-D step (names as in the 2-D ``oracle.Config``)."""
    nx: int
    ny: int
    nz: int
    scheme: str = "improved"
    tau: tuple = (1.0, 1.0)
    G: float = 1.205
    lam: float = 1.0
    Gw2: float | None = None
    delta: float = 0.8
    g: tuple = (0.0, 0.0, 0.0)
    second_layer: str = "psi_and_solid"  # or "psi" (Sec. 2.4, Table 1: what a replaced site copies)
    # adhesion sum of Eq. 9: "e8" (the 92-offset stencil) or "d3q19" (as printed: D3Q19 weights over
    # the 18 first-layer neighbours)
    adhesion_stencil: str = "e8"
    nthreads: int = field(default_factory=lambda: int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)))

    def c(self) -> _Cfg3:
        w = e8_weights_3d()
        s = _Cfg3()
        s.nx, s.ny, s.nz = self.nx, self.ny, self.nz
        s.scheme = SCHEME_IMPROVED if self.scheme == "improved" else SCHEME_ORIGINAL
        s.nthreads = max(1, int(self.nthreads))
        s.tau[0], s.tau[1] = self.tau
        s.G, s.lam = self.G, self.lam
        s.Gw2 = self.G if self.Gw2 is None else self.Gw2
        s.delta = self.delta
        for d in range(3):
            s.g[d] = self.g[d]
        for i, q in enumerate(SHELLS3):
            s.w[i] = float(w[q])
        s.second_layer = {"psi_and_solid": 0, "psi": 1}[self.second_layer]
        s.adhesion_stencil = {"e8": 0, "d3q19": 1}[self.adhesion_stencil]
        return s


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        cp = ctypes.POINTER(_Cfg3)
        lib.oracle3_feq.argtypes = [ctypes.c_double] * 4 + [dp]
        lib.oracle3_guo.argtypes = [ctypes.c_double] * 6 + [dp]
        for name in ("oracle3_collide", "oracle3_stream", "oracle3_fields", "oracle3_forces"):
            getattr(lib, name).argtypes = [cp, u8p, dp, dp]
            getattr(lib, name).restype = ctypes.c_int
        lib.oracle3_run.argtypes = [cp, u8p, dp, ctypes.c_int]
        lib.oracle3_run.restype = ctypes.c_int
        lib.oracle3_init.argtypes = [cp, u8p, dp, dp, dp]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _solid(cfg: Config3, solid) -> np.ndarray:
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    assert s.shape == (cfg.nz, cfg.ny, cfg.nx)
    return s


def _u8(s):
    return s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def feq3(rho, ux, uy, uz) -> np.ndarray:
    out = np.zeros(19)
    _load().oracle3_feq(rho, ux, uy, uz, _dp(out))
    return out


def guo3(ux, uy, uz, Fx, Fy, Fz) -> np.ndarray:
    out = np.zeros(19)
    _load().oracle3_guo(ux, uy, uz, Fx, Fy, Fz, _dp(out))
    return out


def init3(cfg: Config3, solid, rhoA0, rhoB0) -> np.ndarray:
    s = _solid(cfg, solid)
    a = np.ascontiguousarray(rhoA0, np.float64)
    b = np.ascontiguousarray(rhoB0, np.float64)
    f = np.zeros((2, 19, cfg.nz, cfg.ny, cfg.nx))
    c = cfg.c()
    _load().oracle3_init(ctypes.byref(c), _u8(s), _dp(a), _dp(b), _dp(f))
    return f


def _call(name, cfg, solid, f, out_shape):
    s = _solid(cfg, solid)
    f = np.ascontiguousarray(f, np.float64)
    out = np.zeros(out_shape)
    c = cfg.c()
    if getattr(_load(), name)(ctypes.byref(c), _u8(s), _dp(f), _dp(out)):
        raise MemoryError(name)
    return out


def collide3(cfg: Config3, solid, f) -> np.ndarray:
    return _call("oracle3_collide", cfg, solid, f, f.shape)


def stream3(cfg: Config3, solid, fstar) -> np.ndarray:
    return _call("oracle3_stream", cfg, solid, fstar, fstar.shape)


def run3(cfg: Config3, solid, f, nsteps: int) -> np.ndarray:
    s = _solid(cfg, solid)
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    c = cfg.c()
    if _load().oracle3_run(ctypes.byref(c), _u8(s), _dp(g), int(nsteps)):
        raise MemoryError("oracle3_run")
    return g


def fields3(cfg: Config3, solid, f):
    """(rho_A, rho_B, ux, uy, uz), each [nz][ny][nx]; u is Eq. 5's velocity with the half-force
    shift; zero at solid nodes."""
    out = _call("oracle3_fields", cfg, solid, f, (5, cfg.nz, cfg.ny, cfg.nx))
    return tuple(out[i] for i in range(5))


def forces3(cfg: Config3, solid, f):
    """(F_A [3], F_B [3], u [3]) per node, each [3][nz][ny][nx]."""
    out = _call("oracle3_forces", cfg, solid, f, (9, cfg.nz, cfg.ny, cfg.nx))
    return out[0:3], out[3:6], out[6:9]


def diagnostics3(cfg: Config3, solid, f) -> dict:
    """Global FP64 diagnostics over fluid nodes (as in 2-D): masses, momentum, max |u|, extrema."""
    s = _solid(cfg, solid).astype(bool)
    rA, rB, ux, uy, uz = fields3(cfg, solid, f)
    fl = ~s
    rho = rA + rB
    return {
        "mass_A": float(np.sum(rA[fl])), "mass_B": float(np.sum(rB[fl])),
        "mom_x": float(np.sum((rho * ux)[fl])), "mom_y": float(np.sum((rho * uy)[fl])),
        "mom_z": float(np.sum((rho * uz)[fl])),
        "umax": float(np.max(np.sqrt(ux * ux + uy * uy + uz * uz)[fl])),
        "rhoA_min": float(rA[fl].min()), "rhoA_max": float(rA[fl].max()),
        "rhoB_min": float(rB[fl].min()), "rhoB_max": float(rB[fl].max()),
    }


def near_solid3(solid, margin: int = 3) -> np.ndarray:
    """Nodes with a solid node within ``margin`` cells (Chebyshev), periodic in all directions."""
    s = np.asarray(solid).astype(bool)
    out = np.zeros_like(s)
    for dz in range(-margin, margin + 1):
        for dy in range(-margin, margin + 1):
            for dx in range(-margin, margin + 1):
                out |= np.roll(s, (dz, dy, dx), axis=(0, 1, 2))
    return out


def interface_points3(solid, rhoA, rhoB, margin: int = 3) -> np.ndarray:
    """rho^e = 0 crossings (Eq. 10) along x, then y, then z lines, linearly interpolated; both
    nodes fluid and more than ``margin`` cells from solid; pairs across a periodic seam unused."""
    s = np.asarray(solid).astype(bool)
    ok = ~s & ~near_solid3(solid, margin)
    phi = np.where(s, 0.0, (rhoA - rhoB) / np.where(s, 1.0, rhoA + rhoB))
    pts = []
    for axis in (2, 1, 0):  # x, y, z
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis], hi[axis] = slice(None, -1), slice(1, None)
        a, b = phi[tuple(lo)], phi[tuple(hi)]
        m = ok[tuple(lo)] & ok[tuple(hi)] & ((a > 0) != (b > 0))
        z, y, x = np.nonzero(m)
        t = a[z, y, x] / (a[z, y, x] - b[z, y, x])
        p = np.stack([x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)], axis=1)
        p[:, 2 - axis] += t
        pts.append(p)
    return np.concatenate(pts).reshape(-1, 3)


def fit_sphere(pts: np.ndarray):
    """Algebraic sphere fit in centroid coordinates (|p - c|^2 = r^2 linear in c and
    r^2 - |c|^2), followed by one Gauss-Newton step on |p - c| - r.  Returns (cx, cy, cz, r, rms)."""
    m = pts.mean(axis=0)
    q = pts - m
    A = np.concatenate([2 * q, np.ones((len(q), 1))], axis=1)
    rhs = np.sum(q * q, axis=1)
    sol = np.linalg.solve(A.T @ A, A.T @ rhs)
    c = sol[:3]
    r = np.sqrt(sol[3] + c @ c)
    c = c + m
    d = np.linalg.norm(pts - c, axis=1)
    res = d - r
    J = np.concatenate([-(pts - c) / d[:, None], -np.ones((len(d), 1))], axis=1)
    step = np.linalg.solve(J.T @ J, -J.T @ res)
    c, r = c + step[:3], r + step[3]
    rms = float(np.sqrt(np.mean((np.linalg.norm(pts - c, axis=1) - r) ** 2)))
    return float(c[0]), float(c[1]), float(c[2]), float(r), rms


def contact_angle_sphere(cfg: Config3, solid, f, sphere: dict, margin: int = 3):
    """(theta_deg, fit_rms, n_points): droplet sphere against the solid sphere of centre
    ``sphere["c"]`` and effective radius ``sphere["R"]`` (halfway bounce-back: R + 0.5)."""
    rA, rB, _, _, _ = fields3(cfg, solid, f)
    pts = interface_points3(solid, rA, rB, margin)
    cx, cy, cz, r, rms = fit_sphere(pts)
    R = sphere["R"]
    d2 = sum((a - b) ** 2 for a, b in zip((cx, cy, cz), sphere["c"]))
    cth = (R * R + r * r - d2) / (2.0 * r * R)
    return float(np.degrees(np.arccos(np.clip(cth, -1.0, 1.0)))), rms, len(pts)
