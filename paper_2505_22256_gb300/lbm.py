"""Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every function keeps the C name and forwards to ``_build/liblbm_gb300.so``; no computation happens
here.  Arrays are numpy arrays on the host or, where the C call takes device pointers, objects with
``data_ptr()`` (torch tensors) or plain integer addresses.  A non-zero status raises ``LbmError``
carrying the library's message.  The library is never replaced by anything else: if it has not been
built, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_uint8, c_uint32, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm_gb300.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE, LBM_EIO = range(8)
LBM_BC_PERIODIC, LBM_BC_WALL, LBM_BC_OPEN = 0, 1, 2
LBM_ADS_ORIGINAL, LBM_ADS_IMPROVED = 0, 1
LBM_STORE_F64, LBM_STORE_F32, LBM_STORE_F16_SHIFTED, LBM_STORE_BF16_SHIFTED = 0, 1, 2, 3
LBM_SURFACE_FLAT, LBM_SURFACE_CIRCLE, LBM_SURFACE_NONE = 0, 1, 2

STORAGE = {"f64": LBM_STORE_F64, "f32": LBM_STORE_F32, "f16": LBM_STORE_F16_SHIFTED,
           "bf16": LBM_STORE_BF16_SHIFTED}
BC = {"periodic": LBM_BC_PERIODIC, "wall": LBM_BC_WALL, "open": LBM_BC_OPEN}

# exported entry points (every one is declared in include/lbm.h)
SYMBOLS = ("lbm_create", "lbm_ensemble_create", "lbm_destroy", "lbm_step", "lbm_synchronize",
           "lbm_set_densities", "lbm_fields", "lbm_diagnostics", "lbm_contact_angle", "lbm_wall_list",
           "lbm_get_populations", "lbm_set_populations", "lbm_info", "lbm_set_launch", "lbm_autotune",
           "lbm_save", "lbm_load", "lbm_status_str", "lbm_last_error", "lbm_diagnostics_noalloc",
           "lbm_diagnostics_all", "lbm_contact_angle_all", "lbm_set_wall_path", "lbm_set_densities_all",
           "lbm_fields_all", "lbm_selftest_wait_timeout", "lbm_set_densities_all_async", "lbm_fields_all_async")


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("bc_x", c_int32), ("bc_y", c_int32)]


class lbm_params(ctypes.Structure):
    _fields_ = [("tau", c_double * 2), ("G_AB", c_double), ("mode", c_int32), ("lambda_", c_double),
                ("G_w2", c_double), ("delta", c_double), ("g", c_double * 2), ("u_in", c_double),
                ("rho_in", c_double * 2), ("rho0_store", c_double * 2), ("u_wall", c_double * 2),
                ("inlet_profile", c_int32), ("second_layer", c_int32), ("adhesion_stencil", c_int32),
                ("outlet", c_int32), ("rho_out", c_double * 2)]


class lbm_diag(ctypes.Structure):
    _fields_ = [("mass_A", c_double), ("mass_B", c_double), ("mom_x", c_double), ("mom_y", c_double),
                ("umax", c_double), ("rhoA_min", c_double), ("rhoA_max", c_double),
                ("rhoB_min", c_double), ("rhoB_max", c_double), ("n_fluid", c_int64),
                ("unstable", c_int32), ("pad_", c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class lbm_surface(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("normal", c_int32), ("y_w", c_double), ("cx", c_double),
                ("cy", c_double), ("R", c_double)]


class lbm_case(ctypes.Structure):
    _fields_ = [("grid", lbm_grid), ("solid", POINTER(c_uint8)), ("rho_A0", POINTER(c_double)),
                ("rho_B0", POINTER(c_double)), ("params", lbm_params)]


class lbm_info_t(ctypes.Structure):
    _fields_ = [("ncases", c_int32), ("storage", c_int32), ("nodes", c_int64), ("fluid_nodes", c_int64),
                ("wall_nodes", c_int64), ("steps", c_int64), ("state_bytes", c_int64),
                ("device_bytes", c_int64), ("block_threads", c_int32), ("block_rows", c_int32),
                ("grid_blocks", c_int32), ("work_items", c_int32), ("wall_inline", c_int32), ("pad_", c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load the CUDA library (once).  Raises when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    ctx_p = c_void_p
    d = POINTER(c_double)
    lib.lbm_create.argtypes = [POINTER(lbm_grid), POINTER(c_uint8), POINTER(lbm_params), d, d, c_int32,
                               c_void_p, POINTER(ctx_p)]
    lib.lbm_ensemble_create.argtypes = [c_int32, POINTER(lbm_case), c_int32, c_void_p, POINTER(ctx_p)]
    lib.lbm_destroy.argtypes = [ctx_p]
    lib.lbm_destroy.restype = None
    lib.lbm_step.argtypes = [ctx_p, c_int64]
    lib.lbm_synchronize.argtypes = [ctx_p, c_double]
    lib.lbm_set_densities.argtypes = [ctx_p, c_int32, c_void_p, c_void_p, c_int32]
    lib.lbm_fields.argtypes = [ctx_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int32]
    lib.lbm_diagnostics.argtypes = [ctx_p, c_int32, POINTER(lbm_diag)]
    lib.lbm_contact_angle.argtypes = [ctx_p, c_int32, POINTER(lbm_surface), d, d, POINTER(c_int64)]
    lib.lbm_wall_list.argtypes = [ctx_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  POINTER(c_int64)]
    lib.lbm_get_populations.argtypes = [ctx_p, c_int32, c_void_p]
    lib.lbm_set_populations.argtypes = [ctx_p, c_int32, c_void_p]
    lib.lbm_info.argtypes = [ctx_p, POINTER(lbm_info_t)]
    lib.lbm_set_launch.argtypes = [ctx_p, c_int32, c_int32]
    lib.lbm_set_wall_path.argtypes = [ctx_p, c_int32]
    lib.lbm_autotune.argtypes = [ctx_p, c_int32, d]
    lib.lbm_save.argtypes = [ctx_p, ctypes.c_char_p]
    lib.lbm_load.argtypes = [ctx_p, ctypes.c_char_p]
    lib.lbm_diagnostics_noalloc.argtypes = [c_void_p] * 5 + [c_int32, c_int32, c_void_p, POINTER(lbm_diag)]
    lib.lbm_diagnostics_all.argtypes = [ctx_p, POINTER(lbm_diag)]
    lib.lbm_set_densities_all.argtypes = [ctx_p, c_void_p, c_void_p, c_int32]
    lib.lbm_selftest_wait_timeout.argtypes = [ctx_p, c_double]
    lib.lbm_fields_all.argtypes = [ctx_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32]
    lib.lbm_set_densities_all_async.argtypes = [ctx_p, c_void_p, c_void_p]
    lib.lbm_fields_all_async.argtypes = [ctx_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.lbm_contact_angle_all.argtypes = [ctx_p, POINTER(lbm_surface), c_void_p, c_void_p, c_void_p]
    lib.lbm_status_str.argtypes = [c_int32]
    lib.lbm_status_str.restype = ctypes.c_char_p
    lib.lbm_last_error.argtypes = []
    lib.lbm_last_error.restype = ctypes.c_char_p
    for name in SYMBOLS:
        if name not in ("lbm_destroy", "lbm_status_str", "lbm_last_error"):
            getattr(lib, name).restype = c_int32
    _lib = lib
    return lib


def status_name(s: int) -> str:
    return load_library().lbm_status_str(int(s)).decode()


def _check(status: int):
    if status != LBM_OK:
        raise LbmError(status, load_library().lbm_last_error().decode())


def _ptr(a) -> int | None:
    """Address of a host numpy array, a device tensor (data_ptr) or an int; None for None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    return int(a.ctypes.data)


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


INLET = {"uniform": 0, "poiseuille": 1}
SECOND_LAYER = {"psi_and_solid": 0, "psi": 1}  # lbm_second_layer
ADHESION_STENCIL = {"e8": 0, "d2q9": 1}  # lbm_adhesion_stencil
OUTLET = {"copy": 0, "pressure": 1}  # lbm_outlet


def make_params(tau=(1.0, 1.0), G=1.205, scheme="improved", lam=1.0, Gw2=None, delta=0.8, g=(0.0, 0.0),
                u_in=0.0, rho_in=(1.0, 0.03), rho0_store=(0.0, 0.0), u_wall=(0.0, 0.0), inlet_profile="uniform",
                second_layer="psi_and_solid", adhesion_stencil="e8", outlet="copy", rho_out=(0.03, 1.0),
                **_ignored) -> lbm_params:
    p = lbm_params()
    p.tau[0], p.tau[1] = tau
    p.G_AB = G
    p.mode = LBM_ADS_IMPROVED if scheme == "improved" else LBM_ADS_ORIGINAL
    p.lambda_ = lam
    p.G_w2 = G if Gw2 is None else Gw2
    p.delta = delta
    p.g[0], p.g[1] = g
    p.u_in = u_in
    p.rho_in[0], p.rho_in[1] = rho_in
    p.rho0_store[0], p.rho0_store[1] = rho0_store
    p.u_wall[0], p.u_wall[1] = u_wall
    p.inlet_profile = INLET[inlet_profile]
    p.second_layer = SECOND_LAYER[second_layer]
    p.adhesion_stencil = ADHESION_STENCIL[adhesion_stencil]
    p.outlet = OUTLET[outlet]
    p.rho_out[0], p.rho_out[1] = rho_out
    return p


def make_grid(nx, ny, bc_x="periodic", bc_y="wall") -> lbm_grid:
    return lbm_grid(int(nx), int(ny), BC[bc_x], BC[bc_y])


# ------------------------------------------------------------------------------------------------
# entry points, same names as the C ABI
# ------------------------------------------------------------------------------------------------
def lbm_create(grid: lbm_grid, solid, params: lbm_params, rho_A0, rho_B0, storage: int = LBM_STORE_F32,
               cuda_stream: int | None = None) -> c_void_p:
    lib = load_library()
    s = _host(solid, np.uint8)
    a = _host(rho_A0, np.float64)
    b = _host(rho_B0, np.float64)
    ctx = c_void_p()
    _check(lib.lbm_create(ctypes.byref(grid), s.ctypes.data_as(POINTER(c_uint8)), ctypes.byref(params),
                          a.ctypes.data_as(POINTER(c_double)), b.ctypes.data_as(POINTER(c_double)), int(storage),
                          c_void_p(cuda_stream) if cuda_stream else None, ctypes.byref(ctx)))
    return ctx


def lbm_ensemble_create(cases: list, storage: int = LBM_STORE_F32, cuda_stream: int | None = None) -> c_void_p:
    """cases: list of (grid, solid, params, rho_A0, rho_B0)."""
    lib = load_library()
    keep = []
    arr = (lbm_case * len(cases))()
    for i, (grid, solid, params, ra, rb) in enumerate(cases):
        s, a, b = _host(solid, np.uint8), _host(ra, np.float64), _host(rb, np.float64)
        keep += [s, a, b]
        arr[i].grid = grid
        arr[i].solid = s.ctypes.data_as(POINTER(c_uint8))
        arr[i].rho_A0 = a.ctypes.data_as(POINTER(c_double))
        arr[i].rho_B0 = b.ctypes.data_as(POINTER(c_double))
        arr[i].params = params
    ctx = c_void_p()
    _check(lib.lbm_ensemble_create(len(cases), arr, int(storage), c_void_p(cuda_stream) if cuda_stream else None,
                                   ctypes.byref(ctx)))
    del keep
    return ctx


def lbm_destroy(ctx) -> None:
    load_library().lbm_destroy(ctx)


def lbm_step(ctx, n: int) -> None:
    _check(load_library().lbm_step(ctx, int(n)))


def lbm_synchronize(ctx, timeout_s: float = 0.0) -> None:
    _check(load_library().lbm_synchronize(ctx, float(timeout_s)))


def lbm_set_densities(ctx, case_index: int, rho_A0, rho_B0, on_device: bool = False) -> None:
    if on_device:
        _check(load_library().lbm_set_densities(ctx, case_index, _ptr(rho_A0), _ptr(rho_B0), 1))
    else:
        a, b = _host(rho_A0, np.float64), _host(rho_B0, np.float64)
        _check(load_library().lbm_set_densities(ctx, case_index, a.ctypes.data, b.ctypes.data, 0))


def lbm_fields(ctx, case_index: int, rho_A=None, rho_B=None, ux=None, uy=None, on_device: bool = False) -> None:
    """Writes into the given arrays (host float64 numpy arrays, or device buffers if on_device)."""
    for a in (rho_A, rho_B, ux, uy):
        if a is not None and not on_device:
            assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(load_library().lbm_fields(ctx, case_index, _ptr(rho_A), _ptr(rho_B), _ptr(ux), _ptr(uy),
                                     1 if on_device else 0))


def lbm_set_densities_all(ctx, rho_A0, rho_B0, on_device: bool = False) -> None:
    """All cases at once: cases back to back in case order, each [ny][nx] (flat float64 arrays of
    sum nx ny elements, or device buffers if on_device)."""
    if on_device:
        _check(load_library().lbm_set_densities_all(ctx, _ptr(rho_A0), _ptr(rho_B0), 1))
    else:
        a, b = _host(rho_A0, np.float64), _host(rho_B0, np.float64)
        _check(load_library().lbm_set_densities_all(ctx, a.ctypes.data, b.ctypes.data, 0))


def lbm_fields_all(ctx, rho_A=None, rho_B=None, ux=None, uy=None, on_device: bool = False) -> None:
    """Fields of all cases into the given arrays (cases back to back in case order)."""
    for a in (rho_A, rho_B, ux, uy):
        if a is not None and not on_device:
            assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(load_library().lbm_fields_all(ctx, _ptr(rho_A), _ptr(rho_B), _ptr(ux), _ptr(uy), 1 if on_device else 0))


def lbm_set_densities_all_async(ctx, rho_A0: np.ndarray, rho_B0: np.ndarray) -> None:
    """lbm_set_densities_all from host arrays, enqueued: the arrays (C-contiguous float64, ideally
    page-locked) must stay unchanged until lbm_synchronize returns."""
    for a in (rho_A0, rho_B0):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(load_library().lbm_set_densities_all_async(ctx, rho_A0.ctypes.data, rho_B0.ctypes.data))


def lbm_fields_all_async(ctx, rho_A=None, rho_B=None, ux=None, uy=None) -> None:
    """lbm_fields_all into host arrays, enqueued: read them after lbm_synchronize returns."""
    for a in (rho_A, rho_B, ux, uy):
        if a is not None:
            assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(load_library().lbm_fields_all_async(ctx, _ptr(rho_A), _ptr(rho_B), _ptr(ux), _ptr(uy)))


def lbm_selftest_wait_timeout(ctx, limit_ms: float) -> None:
    """Drive a kernel's bounded pipeline wait to its limit; raises the error a stalled step raises."""
    _check(load_library().lbm_selftest_wait_timeout(ctx, float(limit_ms)))


def lbm_diagnostics(ctx, case_index: int = 0, allow_unstable: bool = False) -> dict:
    d = lbm_diag()
    st = load_library().lbm_diagnostics(ctx, case_index, ctypes.byref(d))
    if not (allow_unstable and st == LBM_EUNSTABLE):
        _check(st)
    return d.as_dict()


def lbm_diagnostics_noalloc(rho_A, rho_B, ux, uy, solid, nx: int, ny: int, cuda_stream: int | None = None,
                            allow_unstable: bool = False) -> dict:
    """Diagnostics of device-resident fields without any device allocation (for callers that may
    not allocate: pool-owning frameworks, latency-bound loops, fully committed devices).  The five
    arrays are device buffers (tensors or addresses) of shape [ny][nx]; solid is uint8."""
    d = lbm_diag()
    st = load_library().lbm_diagnostics_noalloc(_ptr(rho_A), _ptr(rho_B), _ptr(ux), _ptr(uy), _ptr(solid), int(nx),
                                                int(ny), c_void_p(cuda_stream) if cuda_stream else None,
                                                ctypes.byref(d))
    if not (allow_unstable and st == LBM_EUNSTABLE):
        _check(st)
    return d.as_dict()


def _fill_surface(s, surface: dict | None) -> None:
    if surface is None:
        s.kind, s.normal = LBM_SURFACE_NONE, 1
    elif surface["kind"] == "flat":
        s.kind, s.normal, s.y_w = LBM_SURFACE_FLAT, int(surface.get("normal", 1)), float(surface["y_w"])
    else:
        s.kind, s.normal = LBM_SURFACE_CIRCLE, 1
        s.cx, s.cy, s.R = float(surface["cx"]), float(surface["cy"]), float(surface["R"])


def lbm_diagnostics_all(ctx, ncases: int, allow_unstable: bool = False) -> list:
    """Diagnostics of every case in one pass (one dict per case)."""
    d = (lbm_diag * ncases)()
    st = load_library().lbm_diagnostics_all(ctx, d)
    if not (allow_unstable and st == LBM_EUNSTABLE):
        _check(st)
    return [x.as_dict() for x in d]


def lbm_contact_angle_all(ctx, surfaces: list):
    """Contact angle of every case; a None surface skips its case.  Returns (theta_deg, fit_rms,
    npoints) as arrays, NaN where a case was skipped or had too few interface points."""
    n = len(surfaces)
    s = (lbm_surface * n)()
    for i, sf in enumerate(surfaces):
        _fill_surface(s[i], sf)
    th, rms, npts = np.zeros(n), np.zeros(n), np.zeros(n, np.int64)
    _check(load_library().lbm_contact_angle_all(ctx, s, th.ctypes.data, rms.ctypes.data, npts.ctypes.data))
    return th, rms, npts


def lbm_contact_angle(ctx, case_index: int, surface: dict):
    s = lbm_surface()
    _fill_surface(s, surface)
    th, rms, n = c_double(), c_double(), c_int64()
    _check(load_library().lbm_contact_angle(ctx, case_index, ctypes.byref(s), ctypes.byref(th), ctypes.byref(rms),
                                            ctypes.byref(n)))
    return th.value, rms.value, n.value


def lbm_wall_list(ctx, case_index: int = 0):
    lib = load_library()
    n = c_int64()
    _check(lib.lbm_wall_list(ctx, case_index, None, None, None, None, None, ctypes.byref(n)))
    node = np.zeros(n.value, np.int32)
    subst = np.zeros(n.value, np.uint32)
    seff = np.zeros(n.value, np.uint32)
    ax = np.zeros(n.value)
    ay = np.zeros(n.value)
    _check(lib.lbm_wall_list(ctx, case_index, node.ctypes.data, subst.ctypes.data, seff.ctypes.data, ax.ctypes.data,
                             ay.ctypes.data, ctypes.byref(n)))
    return node, subst, seff, ax, ay


def lbm_get_populations(ctx, case_index: int, ny: int, nx: int) -> np.ndarray:
    f = np.zeros((2, 9, ny, nx))
    _check(load_library().lbm_get_populations(ctx, case_index, f.ctypes.data))
    return f


def lbm_set_populations(ctx, case_index: int, f) -> None:
    a = _host(f, np.float64)
    _check(load_library().lbm_set_populations(ctx, case_index, a.ctypes.data))


def lbm_info(ctx) -> dict:
    i = lbm_info_t()
    _check(load_library().lbm_info(ctx, ctypes.byref(i)))
    return i.as_dict()


def lbm_set_launch(ctx, block_threads: int, block_rows: int) -> None:
    _check(load_library().lbm_set_launch(ctx, int(block_threads), int(block_rows)))


def lbm_set_wall_path(ctx, inline_correction: int) -> None:
    _check(load_library().lbm_set_wall_path(ctx, int(inline_correction)))


def lbm_autotune(ctx, steps: int = 5) -> float:
    ms = c_double()
    _check(load_library().lbm_autotune(ctx, int(steps), ctypes.byref(ms)))
    return ms.value


def lbm_save(ctx, path: str) -> None:
    _check(load_library().lbm_save(ctx, path.encode()))


def lbm_load(ctx, path: str) -> None:
    _check(load_library().lbm_load(ctx, path.encode()))


# ------------------------------------------------------------------------------------------------
# convenience wrapper over a context built from scenarios
# ------------------------------------------------------------------------------------------------
class Lattice:
    """Owns one context (one or several cases built from ``scenarios.Scenario`` objects)."""

    def __init__(self, scenarios, storage: str = "f32", cuda_stream: int | None = None, rho0_store=None):
        if not isinstance(scenarios, (list, tuple)):
            scenarios = [scenarios]
        self.scenarios = list(scenarios)
        self.storage = STORAGE[storage]
        cases = []
        for sc in self.scenarios:
            p = sc.params()
            p["rho0_store"] = tuple(rho0_store if rho0_store is not None else getattr(sc, "rho0_store", (0.0, 0.0)))
            cases.append((make_grid(sc.nx, sc.ny, sc.bc_x, sc.bc_y), sc.solid, make_params(**p), sc.rhoA0, sc.rhoB0))
        if len(cases) == 1:
            g, s, p, a, b = cases[0]
            self.ctx = lbm_create(g, s, p, a, b, self.storage, cuda_stream)
        else:
            self.ctx = lbm_ensemble_create(cases, self.storage, cuda_stream)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int):
        lbm_step(self.ctx, n)

    def sync(self, timeout_s: float = 0.0):
        lbm_synchronize(self.ctx, timeout_s)

    def fields(self, case: int = 0):
        sc = self.scenarios[case]
        out = [np.zeros((sc.ny, sc.nx)) for _ in range(4)]
        lbm_fields(self.ctx, case, *out)
        return tuple(out)

    def fields_all(self):
        """Fields of every case from one batched call: a list of (rho_A, rho_B, ux, uy) per case."""
        total = sum(sc.nx * sc.ny for sc in self.scenarios)
        out = [np.zeros(total) for _ in range(4)]
        lbm_fields_all(self.ctx, *out)
        res, o = [], 0
        for sc in self.scenarios:
            n = sc.nx * sc.ny
            res.append(tuple(a[o:o + n].reshape(sc.ny, sc.nx) for a in out))
            o += n
        return res

    def populations(self, case: int = 0) -> np.ndarray:
        sc = self.scenarios[case]
        return lbm_get_populations(self.ctx, case, sc.ny, sc.nx)

    def set_populations(self, f, case: int = 0):
        lbm_set_populations(self.ctx, case, f)

    def diagnostics(self, case: int = 0, allow_unstable: bool = False) -> dict:
        return lbm_diagnostics(self.ctx, case, allow_unstable)

    def wall_list(self, case: int = 0):
        return lbm_wall_list(self.ctx, case)

    def contact_angle(self, case: int = 0, surface: dict | None = None):
        return lbm_contact_angle(self.ctx, case, surface or self.scenarios[case].surface)

    def diagnostics_all(self, allow_unstable: bool = False) -> list:
        return lbm_diagnostics_all(self.ctx, len(self.scenarios), allow_unstable)

    def contact_angle_all(self, surfaces: list | None = None):
        return lbm_contact_angle_all(self.ctx, surfaces or [sc.surface for sc in self.scenarios])

    def info(self) -> dict:
        return lbm_info(self.ctx)
