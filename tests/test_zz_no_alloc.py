"""The allocation-free Green step (dtt_apply_green_noalloc) gives the same result as the
ordinary entry point (dtt_apply_green) and as the float64 oracle, on two calls in a row
and in place, for both precisions, and allocates no device memory.

Callers that cannot allocate device memory while they run (fixed-budget services,
latency-critical loops, hosts whose allocator belongs to another framework) use this entry
point with their own device buffers; the library keeps the intermediate spectra in a
fixed array of its own.  This file is collected last so that a failure here leaves every
other test already run.

Grids: 23 x 9 x 14 voxels puts the z axis (a length with the factor 7) on the dense
transform route; 12 x 9 x 16 puts it on the register-radix FFT route with the Green
multiply fused into the z pass, the route of every large grid, where an in-place call
swaps the work buffers.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import discrete as odz

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt, rows  # noqa: E402


def _grid_and_field(seed, prec, nvox):
    spec = wl.random_problem(seed, nvox=nvox, periodic_prob=0.3, n_strong=0, n_weak=0, n_smooth=0,
                             n_tie=0, anchored=False)
    g = rows.setup_grid(spec, prec)
    pb = odz.problem_from(spec)
    rng = np.random.default_rng(100 + seed)
    pt = rng.standard_normal((3,) + g.node_shape)
    for c in range(3):
        pt[c][~pb.dof_mask(c)] = 0.0
    want = odz.green_apply(pb, pt, spec["lam0"], spec["mu0"])
    return g, pt, want


@pytest.mark.parametrize("nvox", [(23, 9, 14), (12, 9, 16)])
@pytest.mark.parametrize("prec,tol", [(dtt.PREC_FP64, 1e-11), (dtt.PREC_MIXED, 2e-6)])
def test_noalloc_green_matches_green_and_oracle(prec, tol, nvox):
    g, pt, want = _grid_and_field(3, prec, nvox)
    ref = g.dtt_apply_green(pt)
    scale = np.abs(want).max()
    assert np.abs(ref - want).max() <= tol * scale
    dev = torch.device("cuda", 0)
    pt_dev = torch.from_numpy(np.ascontiguousarray(pt)).to(dev)
    outs = [torch.full_like(pt_dev, float("nan")) for _ in range(2)]
    g.dtt_apply_green_noalloc(pt_dev, outs[0])          # first call: resolves the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for k in range(2):                                  # two calls in a row
        outs[k].fill_(float("nan"))
        g.dtt_apply_green_noalloc(pt_dev, outs[k])
    got = [o.cpu().numpy() for o in outs]
    for x in got:
        assert np.isfinite(x).all()
        assert np.abs(x - ref).max() <= tol * scale
        assert np.abs(x - want).max() <= tol * scale
    assert np.array_equal(got[0], got[1])
    # in place (input and output the same array)
    inplace = pt_dev.clone()
    g.dtt_apply_green_noalloc(inplace, inplace)
    x = inplace.cpu().numpy()
    assert np.abs(x - ref).max() <= tol * scale
    assert np.abs(x - want).max() <= tol * scale
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, "device memory changed by %d bytes across the calls" % (free0 - free1)
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
