"""The allocation-free diagnostics entry point (lbm_diagnostics_noalloc), for callers that may not
allocate device memory (pool-owning frameworks, latency-bound loops, fully committed devices).

It must agree with the context-based lbm_diagnostics on the same state, call after call, even
though every call shares one fixed scratch array inside the library.  This file is collected last
so that a failure here leaves the rest of a stop-at-first-failure run already done."""
import numpy as np
import pytest

from paper_2505_22256_gb300 import lbm, scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2505_22256_gb300 import build

    build.build()
    lbm.load_library()


def _compare(got, ref):
    for k in ("mass_A", "mass_B", "rhoA_min", "rhoA_max", "rhoB_min", "rhoB_max", "umax"):
        assert got[k] == pytest.approx(ref[k], rel=1e-10), k
    for k in ("mom_x", "mom_y"):
        assert got[k] == pytest.approx(ref[k], rel=1e-8, abs=1e-12), k
    assert got["n_fluid"] == ref["n_fluid"] and got["unstable"] == ref["unstable"] == 0


def _check_consecutive_calls(cases, steps):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    # FP64 storage: both paths then form every sum in double precision and the FP64 diagnostics
    # tolerances of the parity tests apply
    lat = lbm.Lattice(cases, "f64")
    lat.step(steps)
    for case, sc in enumerate(cases):
        ref = lat.diagnostics(case)
        bufs = [torch.empty((sc.ny, sc.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
        lbm.lbm_fields(lat.ctx, case, *bufs, on_device=True)
        lat.sync()
        solid = torch.from_numpy(np.ascontiguousarray(sc.solid)).cuda()
        torch.cuda.synchronize()
        for _ in range(2):  # two calls in a row share the scratch array
            got = lbm.lbm_diagnostics_noalloc(*bufs, solid, sc.nx, sc.ny)
            _compare(got, ref)
        del bufs, solid
        torch.cuda.empty_cache()
    lat.close()


def test_noalloc_diagnostics_match_the_context_diagnostics_on_consecutive_calls():
    """Small lattices: 3 and 8 blocks of 4,096 nodes, fewer than one per lane of the final combine."""
    _check_consecutive_calls([S.cylinder_droplet(96, lam=0.6), S.flat_droplet(200, 150, r=30, lam=1.3)], 40)


def test_noalloc_diagnostics_on_a_1024_squared_lattice():
    """256 blocks: every lane of the final combine adds eight block records in block order."""
    _check_consecutive_calls([S.cylinder_droplet(1024, R=160.0, r=200.0, lam=0.7)], 6)


def test_noalloc_diagnostics_at_the_node_limit():
    """Exactly 16,777,216 nodes (4096 x 4096, periodic, one cylinder): all 4,096 block records of
    the scratch array are written and combined (128 per lane)."""
    sc = S.cylinder_in_box(nx=4096, ny=4096, R=600.0, centre=(2048.0, 1400.0), r=700.0, drop=(2048.0, 2600.0),
                           lam=1.2)
    assert sc.nx * sc.ny == 16_777_216
    _check_consecutive_calls([sc], 2)


def test_noalloc_diagnostics_reject_lattices_beyond_the_scratch_limit():
    torch = pytest.importorskip("torch")
    tiny = torch.zeros(4, dtype=torch.float64, device="cuda")
    mask = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_diagnostics_noalloc(tiny, tiny, tiny, tiny, mask, 8192, 4096)
    assert e.value.status == lbm.LBM_EINVAL and "limit" in str(e.value)
