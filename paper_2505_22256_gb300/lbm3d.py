"""ctypes binding of the 3-D C ABI (include/lbm3d.h): argument marshalling only.  The calls run in
the same in-tree CUDA library as the 2-D ones (``lbm.load_library``)."""
from __future__ import annotations

import ctypes
from ctypes import POINTER, c_double, c_int32, c_int64, c_uint8, c_void_p
from dataclasses import dataclass, field

import numpy as np

from . import lbm

SYMBOLS3 = ("lbm3d_create", "lbm3d_destroy", "lbm3d_step", "lbm3d_fields", "lbm3d_get_populations",
            "lbm3d_set_populations", "lbm3d_diagnostics", "lbm3d_contact_angle", "lbm3d_set_densities",
            "lbm3d_set_densities_async", "lbm3d_fields_async", "lbm3d_synchronize")


class lbm3d_grid(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32)]


class lbm3d_params(ctypes.Structure):
    _fields_ = [("tau", c_double * 2), ("G_AB", c_double), ("mode", c_int32), ("second_layer", c_int32),
                ("lambda_", c_double),
                ("G_w2", c_double), ("delta", c_double), ("g", c_double * 3), ("adhesion_stencil", c_int32),
                ("pad_", c_int32), ("rho0_store", c_double * 2)]


ADHESION_STENCIL3 = {"e8": 0, "d3q19": 1}


class lbm3d_diag(ctypes.Structure):
    _fields_ = [("mass_A", c_double), ("mass_B", c_double), ("mom_x", c_double), ("mom_y", c_double),
                ("mom_z", c_double), ("umax", c_double), ("rhoA_min", c_double), ("rhoA_max", c_double),
                ("rhoB_min", c_double), ("rhoB_max", c_double), ("n_fluid", c_int64), ("unstable", c_int32),
                ("pad_", c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


_ready = False


def _lib():
    global _ready
    lib = lbm.load_library()
    if not _ready:
        d = POINTER(c_double)
        lib.lbm3d_create.argtypes = [POINTER(lbm3d_grid), POINTER(c_uint8), POINTER(lbm3d_params), d, d, c_int32,
                                     c_void_p, POINTER(c_void_p)]
        lib.lbm3d_destroy.argtypes = [c_void_p]
        lib.lbm3d_destroy.restype = None
        lib.lbm3d_step.argtypes = [c_void_p, c_int64]
        lib.lbm3d_fields.argtypes = [c_void_p] + [c_void_p] * 5 + [c_int32]
        lib.lbm3d_get_populations.argtypes = [c_void_p, c_void_p]
        lib.lbm3d_set_populations.argtypes = [c_void_p, c_void_p]
        lib.lbm3d_set_densities.argtypes = [c_void_p, c_void_p, c_void_p, c_int32]
        lib.lbm3d_set_densities_async.argtypes = [c_void_p, c_void_p, c_void_p]
        lib.lbm3d_fields_async.argtypes = [c_void_p] + [c_void_p] * 5
        lib.lbm3d_synchronize.argtypes = [c_void_p]
        lib.lbm3d_diagnostics.argtypes = [c_void_p, POINTER(lbm3d_diag)]
        lib.lbm3d_contact_angle.argtypes = [c_void_p, POINTER(c_double), c_double, d, d, POINTER(c_int64)]
        for name in SYMBOLS3:
            if name != "lbm3d_destroy":
                getattr(lib, name).restype = c_int32
        _ready = True
    return lib


def make_params3(tau=(1.0, 1.0), G=1.205, scheme="improved", lam=1.0, Gw2=None, delta=0.8,
                 g=(0.0, 0.0, 0.0), second_layer="psi_and_solid", adhesion_stencil="e8",
                 rho0_store=(0.0, 0.0)) -> lbm3d_params:
    p = lbm3d_params()
    p.tau[0], p.tau[1] = tau
    p.G_AB = G
    p.mode = lbm.LBM_ADS_IMPROVED if scheme == "improved" else lbm.LBM_ADS_ORIGINAL
    p.lambda_ = lam
    p.G_w2 = G if Gw2 is None else Gw2
    p.delta = delta
    for i in range(3):
        p.g[i] = g[i]
    p.second_layer = lbm.SECOND_LAYER[second_layer]
    p.adhesion_stencil = ADHESION_STENCIL3[adhesion_stencil]
    p.rho0_store[0], p.rho0_store[1] = rho0_store
    return p


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Lattice3:
    """One 3-D lattice on the GPU (periodic in x, y, z; solid mask; storage f64, f32, f16 or bf16)."""

    def __init__(self, solid, rhoA0, rhoB0, params, storage: str = "f32", cuda_stream: int | None = None):
        solid = _c(solid, np.uint8)
        self.nz, self.ny, self.nx = solid.shape
        g = lbm3d_grid(self.nx, self.ny, self.nz)
        p = params if isinstance(params, lbm3d_params) else make_params3(**params)
        a, b = _c(rhoA0, np.float64), _c(rhoB0, np.float64)
        ctx = c_void_p()
        st = lbm.STORAGE[storage]
        lbm._check(_lib().lbm3d_create(ctypes.byref(g), solid.ctypes.data_as(POINTER(c_uint8)), ctypes.byref(p),
                                       a.ctypes.data_as(POINTER(c_double)), b.ctypes.data_as(POINTER(c_double)),
                                       st, c_void_p(cuda_stream) if cuda_stream else None, ctypes.byref(ctx)))
        self.ctx = ctx

    def close(self):
        if self.ctx:
            _lib().lbm3d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int):
        lbm._check(_lib().lbm3d_step(self.ctx, int(n)))

    def fields(self):
        out = [np.zeros((self.nz, self.ny, self.nx)) for _ in range(5)]
        self.fields_into(*out)
        return tuple(out)

    def fields_into(self, rho_A, rho_B, ux, uy, uz):
        """Fields into the given host float64 arrays of shape [nz][ny][nx] (any may be None)."""
        for a in (rho_A, rho_B, ux, uy, uz):
            assert a is None or (a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.nx * self.ny * self.nz)
        lbm._check(_lib().lbm3d_fields(self.ctx, *[lbm._ptr(o) for o in (rho_A, rho_B, ux, uy, uz)], 0))

    def populations(self) -> np.ndarray:
        f = np.zeros((2, 19, self.nz, self.ny, self.nx))
        lbm._check(_lib().lbm3d_get_populations(self.ctx, f.ctypes.data))
        return f

    def set_populations(self, f):
        f = _c(f, np.float64)
        assert f.shape == (2, 19, self.nz, self.ny, self.nx)
        lbm._check(_lib().lbm3d_set_populations(self.ctx, f.ctypes.data))

    def set_densities(self, rho_A, rho_B, on_device: bool = False):
        """f = f^eq(rho_k, 0) from new densities ([nz][ny][nx]; host arrays, or device buffers)."""
        if on_device:
            lbm._check(_lib().lbm3d_set_densities(self.ctx, lbm._ptr(rho_A), lbm._ptr(rho_B), 1))
        else:
            a, b = _c(rho_A, np.float64), _c(rho_B, np.float64)
            assert a.shape == b.shape == (self.nz, self.ny, self.nx)
            lbm._check(_lib().lbm3d_set_densities(self.ctx, a.ctypes.data, b.ctypes.data, 0))

    def set_densities_async(self, rho_A, rho_B):
        """lbm3d_set_densities from host arrays, enqueued: the arrays ([nz][ny][nx] float64,
        C-contiguous, ideally page-locked) must stay unchanged until sync() returns."""
        for a in (rho_A, rho_B):
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.nx * self.ny * self.nz
        lbm._check(_lib().lbm3d_set_densities_async(self.ctx, rho_A.ctypes.data, rho_B.ctypes.data))

    def fields_async_into(self, rho_A, rho_B, ux, uy, uz):
        """lbm3d_fields into host arrays, enqueued: read them after sync() returns."""
        for a in (rho_A, rho_B, ux, uy, uz):
            assert a is None or (a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.nx * self.ny * self.nz)
        lbm._check(_lib().lbm3d_fields_async(self.ctx, *[lbm._ptr(o) for o in (rho_A, rho_B, ux, uy, uz)]))

    def sync(self):
        lbm._check(_lib().lbm3d_synchronize(self.ctx))

    def diagnostics(self, allow_unstable: bool = False) -> dict:
        d = lbm3d_diag()
        st = _lib().lbm3d_diagnostics(self.ctx, ctypes.byref(d))
        if not (allow_unstable and st == lbm.LBM_EUNSTABLE):
            lbm._check(st)
        return d.as_dict()

    def contact_angle(self, sphere: dict):
        """(theta_deg, fit_rms, npoints) against the solid sphere {"c": (x, y, z), "R": R_eff}."""
        c = (c_double * 3)(*sphere["c"])
        th, rms, n = c_double(), c_double(), c_int64()
        lbm._check(_lib().lbm3d_contact_angle(self.ctx, c, float(sphere["R"]), ctypes.byref(th), ctypes.byref(rms),
                                              ctypes.byref(n)))
        return th.value, rms.value, n.value
