"""Warp-register sweeps of the mixed Green step (k_wfft.cu) on the GPU.

The Green step (Section 3.2.2, Tables 2-3, Eq. 7: forward DTTs, the Paux Green multiply,
inverse DTTs) takes the warp-register route on grids whose axes are all non-periodic with
n in {32, 48, 64, 96, 128, 192, 256, 384, 512} voxels.  Checked here against the float64
oracle on such grids (every transform type along every axis, every stage-1 radix R = 2n /
32 of the kernels, both schemes), against the shared-memory Stockham route, in place and
out of place, and in converged solves at the mixed-precision bar: Algorithm 1 with
constraint rows against the oracle, Algorithm 2 increments against the Stockham route."""
import numpy as np
import pytest

import workloads as wl
from oracle import discrete as odz, solver as osv

from helpers import gpu_grid, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt  # noqa: E402

MIXED = dtt.PREC_MIXED
WARP = {"residual_zchunk": 0, "fft_generic": 0, "z_route": 0, "fft_warp": 1}
STOCKHAM = {"residual_zchunk": 0, "fft_generic": 0, "z_route": 0, "fft_warp": 0}
# stage-1 radices R (per axis): (4, 2, 6), (8, 3, 2), (2, 4, 12), (16, 2, 2), (24, 2, 2), (2, 2, 32)
SIZES = [(64, 32, 96), (128, 48, 32), (32, 64, 192), (256, 32, 32), (384, 32, 32), (32, 32, 512)]


def _spec(seed, nvox, scheme=wl.TETRA2, **kw):
    kw.setdefault("anchored", False)
    if kw["anchored"] is False:
        kw.update(n_strong=0, n_weak=0, n_smooth=0, n_tie=0)
    return wl.random_problem(seed, nvox=nvox, scheme=scheme, periodic_prob=0.0, **kw)


def _field(pb, seed):
    pt = np.random.default_rng(100 + seed).standard_normal((3,) + pb.node_shape)
    for c in range(3):
        pt[c][~pb.dof_mask(c)] = 0.0
    return pt


@pytest.mark.parametrize("nvox", SIZES)
@pytest.mark.parametrize("scheme", [wl.TETRA2, wl.HEX1])
def test_green_step_matches_oracle(nvox, scheme):
    """One Green step against the oracle: within 2e-6 of the field's maximum (one FP32
    pass, the bar of the mixed single operators), and not bit-identical to the Stockham
    route (a different code path)."""
    seed = sum(nvox) + scheme
    spec = _spec(seed, nvox, scheme)
    pb, _ = oracle_problem(spec)
    pt = _field(pb, seed)
    ref = odz.green_apply(pb, pt, spec["lam0"], spec["mu0"])
    g = gpu_grid(spec, MIXED)
    g.dtt_set_tuning(WARP)
    got = g.dtt_apply_green(pt)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
    g.dtt_set_tuning(STOCKHAM)
    other = g.dtt_apply_green(pt)
    assert np.abs(other - ref).max() <= 2e-6 * np.abs(ref).max()
    assert not np.array_equal(got, other)
    g.close()


@pytest.mark.parametrize("seed", range(3))
def test_every_type_on_every_axis(seed):
    """Random non-periodic BCs per face and component on a 64 x 96 x 32 grid: every
    (component, axis) pair draws its own transform type."""
    spec = _spec(seed, (64, 96, 32))
    pb, _ = oracle_problem(spec)
    pt = _field(pb, seed)
    ref = odz.green_apply(pb, pt, spec["lam0"], spec["mu0"])
    g = gpu_grid(spec, MIXED)
    got = g.dtt_apply_green(pt)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
    g.close()


def test_converged_solve_with_rows_matches_oracle():
    """Algorithm 1 on an anchored two-phase cell of 32 x 64 x 32 voxels with strong, weak,
    smooth and tie rows: displacement, stress and reactions within 1e-6 of the oracle
    converged to 1e-13 (the mixed path run to r < 1e-7, as the other converged cases)."""
    spec = _spec(4, (32, 64, 32), anchored=True)
    pb, rows = oracle_problem(spec)
    ref = osv.solve_alg1(pb, rows, spec["lam0"], spec["mu0"], 1e-13, 3000)
    g = gpu_grid(spec, MIXED)
    rep = g.dtt_solve_step(1e-7, 3000)
    assert rep.status == dtt.OK, rep.as_dict()
    u, sig = g.dtt_get_fields(sigma=True)
    assert rel_l2(u, ref.u) <= 1e-6
    sref = np.moveaxis(ref.sigma, (0, 1, 2), (3, 4, 5))     # (ip, 3, 3, z, y, x) -> (z, y, x, ip, 3, 3)
    s6 = np.stack([sref[..., a, b] for a, b in ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))], axis=-1)
    assert rel_l2(sig, s6) <= 1e-6
    per, _ = g.dtt_get_reactions(len(rows))
    assert rel_l2(per, ref.reactions) <= 1e-6
    g.close()


def test_routes_reach_the_same_solution():
    """Two increments of Algorithm 2 on a 64 x 64 x 32 block (DCT1 laterally, DST3 along
    z), solved on both routes to r < 1e-7: the warp-register route reaches the Stockham
    route's solution (itself checked against the oracle) within the bar, with the same
    contact set except at nodes whose gap is below 1e-8 R."""
    w = wl.indentation(64, 64, 32, R=16.0, steps=2, dmin=0.01, dmax=0.03)
    I = w.indenter
    out = []
    for t in (WARP, STOCKHAM):
        g = gpu_grid(w, MIXED)
        g.dtt_set_tuning(t)
        g.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])
        res = []
        for step, O in enumerate(I["centers"]):
            g.dtt_move_indenter(O)
            rep = g.dtt_solve_step(1e-7, 4000, acv_mod=3, init=dtt.INIT_PREVIOUS if step else dtt.INIT_ZERO)
            assert rep.status == dtt.OK, rep.as_dict()
            act, gap, fn, force = g.dtt_get_contact()
            res.append((g.dtt_get_fields(), act.copy(), gap.copy(), force.copy()))
        out.append(res)
        g.close()
    for (u0, a0, g0, f0), (u1, a1, g1, f1) in zip(*out):
        assert rel_l2(u0, u1) <= 1e-6
        assert np.abs(f0 - f1).max() <= 1e-6 * np.abs(f1).max()
        tie = np.abs(g1) < 1e-8 * I["radius"]
        assert np.array_equal(a0[~tie], a1[~tie])
