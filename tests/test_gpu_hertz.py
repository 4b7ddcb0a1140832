"""Eq. 30 (Hertz) on the GPU: a rigid sphere of radius R = 64 voxels pressed into a
bottom-clamped block with traction-free sides (Section 5.4's geometry), seven geometric
increments d/R = 0.001 ... 0.01, mixed precision, r < 1e-7.

Hertz's law is for a half-space; a clamped block of depth H stiffens the response by a
relative amount that grows with a / H, a = sqrt(R d) the contact radius.  Measured F /
Hertz at d/R = 0.01: 1.059 (256 x 256 x 128), 1.044 (384 x 384 x 192), 1.037
(512 x 512 x 256), 1.029 (768 x 768 x 384); with R = 128 on the 512 x 512 x 256 block (the
same a / H as R = 64 on 256 x 256 x 128, twice the contact radius in voxels) 1.060, so the
excess follows a / H and not the voxel size.  On the 768 x 768 x 384 block (227 M nodes,
about 54 GB in mixed precision) every increment with d/R <= 0.01 is within 3 %."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26082_b300 import dtt, rows  # noqa: E402
from oracle import hertz  # noqa: E402


def _ratios(L, H, R):
    w = wl.indentation(L, L, H, R=R, steps=7, dmin=0.001, dmax=0.01)
    I = w.indenter
    g = rows.setup_grid(w, dtt.PREC_MIXED)
    g.dtt_set_indenter(I["axis"], I["face"], I["centers"][0], I["radius"])
    out = []
    for s, O in enumerate(I["centers"]):
        g.dtt_move_indenter(O)
        rep = g.dtt_solve_step(1e-7, 20000, acv_mod=3, init=dtt.INIT_PREVIOUS if s else dtt.INIT_ZERO,
                               graph_iters=16)
        assert rep.status == dtt.OK, rep.as_dict()
        act, gap, fn, force = g.dtt_get_contact()
        assert gap.min() >= -1e-6 * R                       # no penetration beyond rounding
        assert (fn[act] <= 1e-8 * np.abs(fn).max()).all()   # no tensile reaction
        d = I["ratios"][s] * R
        out.append(np.linalg.norm(force) / hertz.hertz_force(I["E"], I["nu"], R, d))
    g.close()
    return np.array(out)


def test_hertz_within_3_percent_on_a_large_block():
    small = _ratios(256, 128, 64.0)
    large = _ratios(768, 384, 64.0)
    assert np.all(np.abs(large - 1.0) <= 0.03), large
    # the finite-block excess shrinks with the block at the deepest increments
    assert np.all(large[-3:] < small[-3:])
