"""Host logic of the learned increment start (paper_2607_26082_b300.warmstart), on the CPU:
the indentation depths and depth triples, and the secant start without the network, which
scales the previous step like the Hertz force (F grows like d^(3/2), Eq. 30) and is exact
for a field that grows that way."""
import numpy as np
import pytest

import workloads as wl
from paper_2607_26082_b300 import warmstart

torch = pytest.importorskip("torch")


def test_depths_follow_the_sphere_centres():
    spec = wl.indentation_inclusions(3001, 48, 40, 24, steps=6)
    I = spec["indenter"]
    dk = warmstart.depths(spec)
    assert len(dk) == 6 and all(b > a > 0 for a, b in zip(dk, dk[1:]))
    nz = spec["nvox"][2]
    for d, c in zip(dk, I["centers"]):
        # the sphere's lowest point lies d below the top face
        assert c[2] - I["radius"] == pytest.approx(nz - d, abs=1e-12)
    assert warmstart.depth_triple(dk, 1) == (0.0, dk[0], dk[1])
    assert warmstart.depth_triple(dk, 4) == (dk[2], dk[3], dk[4])


def test_secant_start_is_exact_for_a_hertz_scaled_field():
    rng = np.random.default_rng(5)
    phi = torch.from_numpy(rng.standard_normal((3, 4, 5, 6)))
    dk = [0.05, 0.08, 0.13, 0.2]
    U = [d ** 1.5 * phi for d in dk]
    FN = [torch.from_numpy(-(d ** 1.5) * rng.random(7)) * torch.from_numpy((np.arange(7) % 3 == 0) * 1.0)
          for d in dk]
    for k in (2, 3):
        u, act = warmstart.secant_start(U, FN, dk, k)
        assert torch.allclose(u, U[k], rtol=1e-12, atol=1e-15)
        # the previous increment's contact zone: the nodes with a compressive reaction
        assert act.tolist() == [1 if i % 3 == 0 else 0 for i in range(7)]
    # the second increment extrapolates from the unloaded state (u = 0 at d = 0)
    u, _ = warmstart.secant_start(U, FN, dk, 1)
    assert torch.allclose(u, U[1], rtol=1e-12, atol=1e-15)


def test_lr_schedule_halves_every_quarter():
    f = warmstart.lr_schedule(1e-3, 8)
    assert [f(ep) for ep in range(8)] == [1e-3, 1e-3, 5e-4, 5e-4, 2.5e-4, 2.5e-4, 1.25e-4, 1.25e-4]
