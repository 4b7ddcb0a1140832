"""GPU parity at full size: the 256x256x128 indentation block (8.5 M nodes) and the
384x384x192 block with inclusions (28.6 M nodes), whose transform lengths (512 / 256 and
768 / 384) run on the register-radix FFT kernels.  The oracle cannot run on these grids,
so the checks use properties that hold at any size:

  * Green step (Algorithm 1, Eq. 7 with the Paux symbol of Section 3.2.3): a separable
    DTT mode of one component is an eigenvector, mapped to itself divided by a_c(q).  The
    symbol comes from oracle.discrete.S_symbols; the whole output field is compared.
  * Residual operator (stress, divergence and the reference term A0 u~, Section 3.1): the
    value at an interior node depends only on the 27 nodes and 8 voxels around it, so the
    oracle evaluates it on a 2x2x2-voxel window cut from the full grid, at sampled nodes
    (half of them next to a phase interface), in small and in finite strain.
  * Contact (Algorithm 2): the first increment's converged state satisfies Eq. 33 and the
    force balance of Section 5.4.

Tolerances as in test_gpu_parity.py: FP64 1e-11 relative; mixed 2e-6 of the field scale
for the residual operator, 5e-6 for the Green step of a single mode on these long axes.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import discrete as odz, transforms as otr
from tests.helpers import gpu_grid

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt  # noqa: E402

FP64, MIXED = dtt.PREC_FP64, dtt.PREC_MIXED

CASES = {
    "indentation_256x256x128": lambda: wl.indentation(256, 256, 128, R=64.0, steps=2),
    "indentation_inclusions_384x384x192": lambda: wl.indentation_inclusions(3000, steps=2),
}


def _mode_factors(pb, c, ks):
    """1-D factors (x, y, z) of the DTT mode of component c with wave numbers ks: cosines
    on cosine-type axes, sines on sine-type axes, zero on a Dirichlet end node."""
    out = []
    for d in range(3):
        t = pb.types[c][d]
        j = np.arange(pb.nn[d])
        v = np.cos(ks[d] * j) if t in (otr.DCT1, otr.DCT3, otr.DFT) else np.sin(ks[d] * j)
        if t == otr.DCT3:
            v[pb.nvox[d]] = 0.0
        out.append(v)
    return out


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (MIXED, 5e-6)])
def test_green_step_full_size_eigenmodes(case, prec, tol):
    spec = CASES[case]()
    pb = odz.problem_from(spec)
    g = gpu_grid(spec, prec)
    rng = np.random.default_rng(17)
    for trial in range(2):
        p = np.zeros((3,) + pb.node_shape)
        a = np.zeros(3)
        for c in range(3):
            ks = []
            for d in range(3):
                q = otr.selection(pb.types[c][d], pb.nvox[d])[2]
                # one low and one high wave number per axis over the two trials
                ks.append(q[rng.integers(1, 8)] if trial == 0 else q[len(q) - 1 - rng.integers(0, 8)])
            fx, fy, fz = _mode_factors(pb, c, ks)
            p[c] = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
            S = odz.S_symbols(pb, np.array([ks[0]]), np.array([ks[1]]), np.array([ks[2]]))
            a[c] = (spec["lam0"] * S[c] + 2.0 * spec["mu0"] * (S[0] + S[1] + S[2])).item()
        assert a.min() > 0.0
        u = g.dtt_apply_green(p)
        for c in range(3):
            ref = p[c] / a[c]
            assert np.abs(u[c] - ref).max() <= tol * np.abs(ref).max(), (case, trial, c)
    g.close()


def _interface_nodes(phase, rng, count):
    """Interior nodes (k, j, i) with both phases among their 8 voxels."""
    mixed = np.zeros(tuple(s - 1 for s in phase.shape), bool)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                blk = phase[dk:dk + mixed.shape[0], dj:dj + mixed.shape[1], di:di + mixed.shape[2]]
                mixed |= blk != phase[:-1, :-1, :-1]
    cand = np.argwhere(mixed) + 1
    if len(cand) == 0:
        return np.zeros((0, 3), int)
    return cand[rng.choice(len(cand), size=min(count, len(cand)), replace=False)]


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kin", ["SS", "FS"])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (MIXED, 2e-6)])
def test_residual_operator_full_size_sampled(case, kin, prec, tol):
    spec = CASES[case]()
    spec["kinematics"] = kin
    pb = odz.problem_from(spec)
    g = gpu_grid(spec, prec)
    rng = np.random.default_rng(23)
    u = 1e-2 * rng.standard_normal((3,) + pb.node_shape)
    for c in range(3):
        u[c][~pb.dof_mask(c)] = 0.0
    p, pt, _ = g.dtt_apply_residual(u)
    g.close()
    nz, ny, nx = pb.node_shape
    nodes = np.stack([rng.integers(1, nz - 1, 100), rng.integers(1, ny - 1, 100), rng.integers(1, nx - 1, 100)], 1)
    nodes = np.concatenate([nodes, _interface_nodes(spec["phase"], rng, 100)])
    got_p, got_pt, ref_p, ref_pt = [], [], [], []
    for k, j, i in nodes:
        win = odz.Problem((2, 2, 2), pb.h, np.full((3, 2, 3), otr.BC_N), pb.scheme,
                          spec["phase"][k - 1:k + 1, j - 1:j + 1, i - 1:i + 1], spec["lam"], spec["mu"],
                          spec.get("eps_star"))
        uw = u[:, k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
        pw, _ = odz.residual(win, uw, kin)
        a0 = odz.apply_A0(win, uw, spec["lam0"], spec["mu0"])
        ref_p.append(pw[:, 1, 1, 1])
        ref_pt.append(pw[:, 1, 1, 1] + a0[:, 1, 1, 1])
        got_p.append(p[:, k, j, i])
        got_pt.append(pt[:, k, j, i])
    ref_p, ref_pt, got_p, got_pt = map(np.array, (ref_p, ref_pt, got_p, got_pt))
    scale_p = np.abs(p).max()
    scale_pt = max(scale_p, np.abs(ref_pt).max())
    assert np.abs(got_p - ref_p).max() <= tol * scale_p
    assert np.abs(got_pt - ref_pt).max() <= tol * scale_pt
    # the interface samples do see both phases
    assert len(nodes) > 100 or len(np.unique(spec["phase"])) == 1


@pytest.mark.parametrize("case", list(CASES))
def test_contact_full_size_first_increment(case):
    """Algorithm 2 on the full grid, mixed precision, first increment from u~ = 0 (d/R =
    0.001), in the runner's configuration (tolerance 1e-6, Anderson every 3 iterations):
    Eq. 33 complementarity at convergence (no penetration, no tensile reaction, zero gap on
    the contact set).  On the 256x256x128 block, the contact force equals the volume average
    of sigma_zz times the top face's area (Section 5.4)."""
    spec = CASES[case]()
    I = spec["indenter"]
    g = gpu_grid(spec, MIXED)
    g.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])
    g.dtt_move_indenter(I["centers"][0])
    rep = g.dtt_solve_step(1e-6, 20000, acv_mod=spec["acv_mod"], init=dtt.INIT_ZERO, graph_iters=16)
    assert rep.status == dtt.OK, rep.as_dict()
    act, gap, fn, force = g.dtt_get_contact()
    assert act.sum() >= 5
    assert gap.min() >= -1e-6 * I["radius"]
    assert np.abs(gap[act]).max() <= 1e-6 * I["radius"]
    assert (fn[act] <= 1e-8 * np.abs(fn).max()).all()
    assert force[2] < 0.0
    if case == "indentation_256x256x128":
        sig = g.dtt_get_stress_tensor()
        w = 0.5 if sig.shape[3] == 2 else 1.0
        mean_zz = w * sig[..., 2, 2].sum() / float(np.prod(spec["nvox"]))
        area = spec["nvox"][0] * spec["nvox"][1] * spec["h"] ** 2
        assert abs(mean_zz * area - force[2]) <= 1e-5 * abs(force[2])   # measured 2e-7
    g.close()
