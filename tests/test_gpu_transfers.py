"""Overlapped host transfers (lbm_set_densities_all_async, lbm_fields_all_async; include/lbm.h)
against the blocking calls, through the C ABI: the same states and fields, bit for bit, with the
copies of successive calls in flight beside the time steps."""
import numpy as np
import pytest

from paper_2505_22256_gb300 import lbm, scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2505_22256_gb300 import build

    build.build()
    lbm.load_library()


def pinned(n):
    import torch

    return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()


def cases():
    return S.lambda_sweep_cylinder(n=160, seed=5, angles=(40, 90, 140))


def inputs(cs, k):
    """Densities of cycle k: the cases' initial fields, scaled a little differently per cycle."""
    a = np.concatenate([c.rhoA0.ravel() for c in cs]) * (1.0 + 0.01 * k)
    b = np.concatenate([c.rhoB0.ravel() for c in cs]) * (1.0 - 0.005 * k)
    return a, b


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_overlapped_cycles_equal_blocking_cycles(storage):
    cs = cases()
    total = sum(c.nx * c.ny for c in cs)
    cycles = 4
    # blocking: set, step, fields, one cycle at a time
    ref = []
    lat = lbm.Lattice(cs, storage)
    for k in range(cycles):
        a, b = inputs(cs, k)
        lbm.lbm_set_densities_all(lat.ctx, a, b, False)
        lat.step(7)
        out = [np.zeros(total) for _ in range(4)]
        lbm.lbm_fields_all(lat.ctx, *out)
        ref.append(out)
    lat.close()
    # overlapped: every cycle enqueued before anything is waited for; staging buffers alternate,
    # so cycles 2 and 3 reuse the buffers of cycles 0 and 1
    lat = lbm.Lattice(cs, storage)
    hin = [(pinned(total), pinned(total)) for _ in range(cycles)]
    hout = [[pinned(total) for _ in range(4)] for _ in range(cycles)]
    for k in range(cycles):
        hin[k][0][...], hin[k][1][...] = inputs(cs, k)
        for o in hout[k]:
            o[...] = np.nan
    for k in range(cycles):
        lbm.lbm_set_densities_all_async(lat.ctx, *hin[k])
        lat.step(7)
        lbm.lbm_fields_all_async(lat.ctx, *hout[k])
    lat.sync()
    for k in range(cycles):
        for q in range(4):
            np.testing.assert_array_equal(hout[k][q], ref[k][q])
    # a blocking call after the overlapped ones sees the same state
    out = [np.zeros(total) for _ in range(4)]
    lbm.lbm_fields_all(lat.ctx, *out)
    for q in range(4):
        np.testing.assert_array_equal(out[q], ref[-1][q])
    lat.close()


def test_partial_outputs_and_a_continuing_run():
    """NULL field outputs are skipped; fields taken without re-initialising between cycles equal the
    blocking calls' on the same run."""
    cs = cases()
    total = sum(c.nx * c.ny for c in cs)
    ref = []
    lat = lbm.Lattice(cs, "f32")
    for _ in range(3):
        lat.step(5)
        out = [np.zeros(total) for _ in range(4)]
        lbm.lbm_fields_all(lat.ctx, *out)
        ref.append(out)
    lat.close()
    lat = lbm.Lattice(cs, "f32")
    ra = [pinned(total) for _ in range(3)]
    uy = [pinned(total) for _ in range(3)]
    for k in range(3):
        lat.step(5)
        lbm.lbm_fields_all_async(lat.ctx, ra[k], None, None, uy[k])
    lat.sync()
    for k in range(3):
        np.testing.assert_array_equal(ra[k], ref[k][0])
        np.testing.assert_array_equal(uy[k], ref[k][3])
    lat.close()
