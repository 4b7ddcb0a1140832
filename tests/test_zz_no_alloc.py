"""The allocation-free Green step (dtt_apply_green_noalloc) gives the same result as the
ordinary entry point (dtt_apply_green), on two calls in a row, for both precisions.

Callers that cannot allocate device memory while they run (fixed-budget services,
latency-critical loops, hosts whose allocator belongs to another framework) use this entry
point with their own device buffers; the library keeps the intermediate spectra in a
fixed array of its own.  This file is collected last so that a failure here leaves every
other test already run.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt, rows  # noqa: E402


def _grid_and_field(seed, prec):
    spec = wl.random_problem(seed, nvox=(23, 9, 14), periodic_prob=0.3, n_strong=0, n_weak=0, n_smooth=0,
                             n_tie=0, anchored=False)
    g = rows.setup_grid(spec, prec)
    rng = np.random.default_rng(100 + seed)
    pt = rng.standard_normal((3,) + g.node_shape)
    return g, pt


@pytest.mark.parametrize("prec,tol", [(dtt.PREC_FP64, 1e-11), (dtt.PREC_MIXED, 2e-6)])
def test_noalloc_green_matches_green_twice(prec, tol):
    g, pt = _grid_and_field(3, prec)
    ref = g.dtt_apply_green(pt)
    dev = torch.device("cuda", 0)
    pt_dev = torch.from_numpy(np.ascontiguousarray(pt)).to(dev)
    for _ in range(2):
        out = torch.full_like(pt_dev, float("nan"))
        g.dtt_apply_green_noalloc(pt_dev, out)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # in place (input and output the same array)
    g.dtt_apply_green_noalloc(pt_dev, pt_dev)
    assert np.abs(pt_dev.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    g.close()


def test_noalloc_green_rejects_grids_beyond_the_scratch():
    bc = np.full((3, 2, 3), wl.D)
    g = dtt.Grid((144, 144, 144), 1.0, bc, precision=dtt.PREC_MIXED)
    assert g.n_nodes > 64 * 2 ** 20 // 24
    g.dtt_set_material(np.zeros(144 ** 3, np.uint8), [1.0], [1.0])
    g.dtt_set_reference(1.0, 1.0)
    buf = torch.zeros((3, g.n_nodes), dtype=torch.float64, device="cuda")
    with pytest.raises(dtt.DttError) as e:
        g.dtt_apply_green_noalloc(buf, buf)
    assert e.value.status == dtt.ERR_ARG
    g.close()
