"""C-ABI checks that need no GPU: the library loads, exports every entry point that include/lbm.h
declares, rejects invalid arguments with LBM_EINVAL before touching the device, and reports the
absence of a GB300 as LBM_ECUDA (there is no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_2505_22256_gb300 import build, lbm as binding

    build.build()
    binding.load_library()
    return binding


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_documented_calls():
    names = _declared_functions()
    for must in ("lbm_create", "lbm_step", "lbm_fields", "lbm_contact_angle", "lbm_diagnostics",
                 "lbm_wall_list", "lbm_ensemble_create", "lbm_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lbm):
    lib = ctypes.CDLL(lbm.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(lbm.SYMBOLS) == _declared_functions()


def test_struct_layouts_match_header(lbm, tmp_path):
    """Every field of the binding's ctypes structures sits at the offset the C compiler gives the
    header's struct (gcc, offsetof / sizeof), so layout changes cannot drift apart."""
    structs = {"lbm_grid": lbm.lbm_grid, "lbm_params": lbm.lbm_params, "lbm_diag": lbm.lbm_diag,
               "lbm_surface": lbm.lbm_surface, "lbm_info_t": lbm.lbm_info_t, "lbm_case": lbm.lbm_case}
    c_names = {"lambda_": "lambda"}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lbm.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            cf = c_names.get(fname, fname)
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {cf}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def _case(n=16):
    solid = np.zeros((n, n), np.uint8)
    solid[0] = solid[-1] = 1
    r = np.full((n, n), 0.5)
    return solid, r, r.copy()


@pytest.mark.parametrize("field,value", [("tau", (0.5, 1.0)), ("lambda_", 0.0), ("delta", 1.5),
                                         ("delta", 0.0), ("G_AB", float("nan")), ("mode", 7),
                                         ("second_layer", 2), ("adhesion_stencil", 2), ("adhesion_stencil", -1)])
def test_invalid_parameters_are_rejected(lbm, field, value):
    solid, a, b = _case()
    p = lbm.make_params()
    if field == "tau":
        p.tau[0], p.tau[1] = value
    else:
        setattr(p, field, value)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_grid(16, 16), solid, p, a, b)
    assert e.value.status == lbm.LBM_EINVAL


@pytest.mark.parametrize("bc_x,bc_y,field,value", [
    ("periodic", "wall", "inlet_profile", 2),           # no such profile
    ("periodic", "wall", "inlet_profile", 1),           # the Poiseuille inlet needs an open x
    ("open", "periodic", "inlet_profile", 1),           # ... and walls in y
    ("periodic", "periodic", "u_wall", (0.01, 0.0)),    # sliding walls need walls in y
    ("open", "wall", "u_wall", (0.0, 0.01)),            # ... and a closed x
    ("periodic", "wall", "u_wall", (float("inf"), 0.0)),
    ("periodic", "wall", "outlet", 1),                  # the pressure outlet needs an open x
    ("open", "wall", "outlet", 2),                      # no such outlet
    ("open", "wall", "rho_out", (0.0, 1.0)),            # outlet densities must be > 0
])
def test_inlet_profile_and_sliding_wall_parameters_are_checked(lbm, bc_x, bc_y, field, value):
    solid, a, b = _case()
    p = lbm.make_params()
    if field == "u_wall":
        p.u_wall[0], p.u_wall[1] = value
    elif field == "rho_out":
        p.outlet = 1
        p.rho_out[0], p.rho_out[1] = value
    else:
        setattr(p, field, value)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_grid(16, 16, bc_x, bc_y), solid, p, a, b)
    assert e.value.status == lbm.LBM_EINVAL


def test_invalid_grids_and_fields_are_rejected(lbm):
    solid, a, b = _case()
    p = lbm.make_params()
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_grid(4, 16), solid[:, :4], p, a[:, :4], b[:, :4])
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_grid(16, 16, "periodic", "open"), solid, p, a, b)
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_grid(16, 16), np.ones((16, 16), np.uint8), p, a, b)
    assert e.value.status == lbm.LBM_EINVAL and "no fluid" in str(e.value)
    bad = a.copy()
    bad[5, 5] = -1.0
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_grid(16, 16), solid, p, bad, b)
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_ensemble_create([], lbm.LBM_STORE_F32)
    assert e.value.status == lbm.LBM_EINVAL


def test_null_context_is_rejected(lbm):
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step(None, 1)
    assert e.value.status == lbm.LBM_EINVAL
    lbm.lbm_destroy(None)  # no-op
    a = np.zeros(4)
    for call in (lambda: lbm.lbm_set_densities_all_async(None, a, a), lambda: lbm.lbm_fields_all_async(None, a),
                 lambda: lbm.lbm_synchronize(None, 0.0)):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.status == lbm.LBM_EINVAL


def test_no_cpu_fallback_without_a_gb300(lbm):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    solid, a, b = _case()
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_grid(16, 16), solid, lbm.make_params(), a, b)
    assert e.value.status == lbm.LBM_ECUDA


def test_status_strings(lbm):
    assert lbm.status_name(0) == "LBM_OK"
    assert lbm.status_name(4) == "LBM_EUNSTABLE"
    assert lbm.status_name(99) == "LBM_UNKNOWN"


# ---------------------------------------------------------------------------------------------
# the 3-D ABI (include/lbm3d.h)
# ---------------------------------------------------------------------------------------------
def _declared3():
    text = open(os.path.join(ROOT, "include", "lbm3d.h")).read()
    return sorted(set(re.findall(r"\b(lbm3d_\w+)\s*\(", text)))


def test_3d_header_declarations_match_binding_and_exports(lbm):
    from paper_2505_22256_gb300 import lbm3d

    assert sorted(lbm3d.SYMBOLS3) == _declared3()
    lib = lbm.load_library()
    for name in lbm3d.SYMBOLS3:
        assert hasattr(lib, name), name


def test_3d_struct_layouts_match_header(lbm, tmp_path):
    from paper_2505_22256_gb300 import lbm3d

    structs = {"lbm3d_grid": lbm3d.lbm3d_grid, "lbm3d_params": lbm3d.lbm3d_params, "lbm3d_diag": lbm3d.lbm3d_diag}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lbm3d.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {cf}));')
    lines.append("return 0; }")
    src = tmp_path / "layout3.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout3"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_3d_null_context_is_rejected(lbm):
    from paper_2505_22256_gb300 import lbm3d

    lib = lbm3d._lib()
    a = np.zeros(4)
    for st in (lib.lbm3d_set_densities_async(None, a.ctypes.data, a.ctypes.data),
               lib.lbm3d_fields_async(None, a.ctypes.data, None, None, None, None), lib.lbm3d_synchronize(None),
               lib.lbm3d_step(None, 1)):
        assert st == lbm.LBM_EINVAL


@pytest.mark.parametrize("what", ["tau", "lambda", "delta", "mode", "adhesion", "size", "storage", "density",
                                  "allsolid"])
def test_3d_invalid_input_is_rejected_before_any_device_work(lbm, what):
    from paper_2505_22256_gb300 import lbm3d

    n = 8
    solid = np.zeros((n, n, n), np.uint8)
    a = np.full((n, n, n), 0.5)
    params = dict(tau=(1.0, 1.0), lam=1.0, delta=0.8, scheme="improved")
    storage = "f32"
    if what == "tau":
        params["tau"] = (0.5, 1.0)
    elif what == "lambda":
        params["lam"] = 0.0
    elif what == "delta":
        params["delta"] = 1.5
    elif what == "size":
        solid, a = solid[:, :, :4], a[:, :, :4]
    elif what == "density":
        a = a.copy()
        a[2, 3, 4] = -1.0
    elif what == "allsolid":
        solid = np.ones_like(solid)
    if what in ("mode", "adhesion", "storage"):
        p = lbm3d.make_params3()
        st_code = 1
        if what == "mode":
            p.mode = 5
        elif what == "adhesion":
            p.adhesion_stencil = 2
        else:
            st_code = 9
        g = lbm3d.lbm3d_grid(n, n, n)
        ctx = ctypes.c_void_p()
        st = lbm3d._lib().lbm3d_create(ctypes.byref(g), solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                       ctypes.byref(p), a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), st_code, None,
                                       ctypes.byref(ctx))
        assert st == lbm.LBM_EINVAL
        return
    with pytest.raises(lbm.LbmError) as e:
        lbm3d.Lattice3(solid, a, a, params, storage)
    assert e.value.status == lbm.LBM_EINVAL
