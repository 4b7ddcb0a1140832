"""Pins of the float64 reference network (oracle/net.py) against facts outside it: the
convolution against scipy.ndimage.correlate, the backward pass against central finite
differences of the loss, the pooling / upsampling adjoint identities, and the input
features of a small cell checked channel by channel."""
import numpy as np
from scipy import ndimage

import workloads as wl
from oracle import net as onet


def _rand_layers(rng, c=(16, 16, 16), scale=0.15):
    return [(rng.standard_normal((27, co, ci)) * scale, rng.standard_normal(co) * 0.05)
            for ci, co in onet.layer_shapes(*c)]


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 6, 7, 3))
    W = rng.standard_normal((27, 4, 3))
    b = rng.standard_normal(4)
    y = onet.conv(x, W, b)
    for o in range(4):
        ref = np.full(x.shape[:3], b[o])
        for i in range(3):
            k = W[:, o, i].reshape(3, 3, 3)   # [dz + 1, dy + 1, dx + 1]
            ref += ndimage.correlate(x[..., i], k, mode="constant", cval=0.0)
        assert np.abs(y[..., o] - ref).max() < 1e-12


def test_pool_and_up_adjoints():
    rng = np.random.default_rng(1)
    for shape in [(5, 4, 7), (6, 6, 6), (3, 2, 1)]:
        a = rng.standard_normal(shape + (2,))
        pc = onet.pool(a)
        bcoarse = rng.standard_normal(pc.shape)
        assert np.isclose((pc * bcoarse).sum(), (a * onet.pool_adjoint(bcoarse, shape)).sum())
        f = rng.standard_normal(shape + (2,))
        uc = onet.up(bcoarse, shape)
        assert np.isclose((uc * f).sum(), (bcoarse * onet.up_adjoint(f, pc.shape[:3])).sum())
        # pooling a constant gives the constant (partial blocks averaged over their own cells)
        assert np.allclose(onet.pool(np.ones(shape + (1,)) * 3.0), 3.0)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    layers = _rand_layers(rng)
    x = rng.standard_normal((3, 4, 5, 16))
    t = rng.standard_normal((3, 4, 5, 3))
    w = 0.3
    loss, grads, _ = onet.loss_grad(layers, x, t, w)
    p0 = onet.pack(layers)
    g = onet.pack(grads)
    h = 1e-6
    idx = rng.choice(p0.size, 40, replace=False)
    idx = np.concatenate([idx, [onet.pack(layers[:10]).size + 1, 7]])   # include a last-layer and a first-layer entry
    for q in idx:
        pp, pm = p0.copy(), p0.copy()
        pp[q] += h
        pm[q] -= h
        lp = onet.loss_grad(onet.unpack(pp, 16, 16, 16), x, t, w)[0]
        lm = onet.loss_grad(onet.unpack(pm, 16, 16, 16), x, t, w)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9, (q, fd, g[q])


def test_features_of_a_small_cell():
    c = wl.batch_cell(77, sizes=(8,))
    x = onet.features(c)
    nn = [c["nvox"][d] if c["bc"][d][0][0] == wl.P else c["nvox"][d] + 1 for d in range(3)]
    assert x.shape == (nn[2], nn[1], nn[0], 16)
    assert 0.0 < x[..., 0].min() and x[..., 0].max() <= 1.0 + 1e-15
    # a Dirichlet face fixes its component on every node of the face
    for comp in range(3):
        for d in range(3):
            for f in range(2):
                if c["bc"][d][f][comp] == wl.D:
                    sl = [slice(None)] * 3
                    sl[2 - d] = 0 if f == 0 else nn[d] - 1
                    assert (x[tuple(sl) + (1 + comp,)] == 1.0).all()
    for it in c["intents"]:
        i, j, k = it["ijk"]
        assert x[k, j, i, 1 + it["comp"]] == 1.0
    e = c["eps_star"]
    assert np.allclose(x[..., 4], 1000 * e[0, 0]) and np.allclose(x[..., 9], 1000 * e[0, 1])
    assert x[..., 10].max() == (nn[0] - 1) / c["nvox"][0] and (x[..., 13:] == 0).all()


def test_increment_loss_backward_matches_finite_differences():
    rng = np.random.default_rng(5)
    layers = _rand_layers(rng)
    x = rng.standard_normal((3, 4, 5, 16))
    t = rng.standard_normal((3, 4, 5, 4))
    m = np.zeros((3, 4, 5))
    m[-1] = 1.0                                   # the top layer is the surface
    wp = 0.7
    loss, grads, _ = onet.increment_loss_grad(layers, x, t, m, wp)
    p0 = onet.pack(layers)
    g = onet.pack(grads)
    h = 1e-6
    for q in np.concatenate([rng.choice(p0.size, 30, replace=False), [onet.pack(layers[:10]).size + 3]]):
        pp, pm = p0.copy(), p0.copy()
        pp[q] += h
        pm[q] -= h
        fd = (onet.increment_loss_grad(onet.unpack(pp, 16, 16, 16), x, t, m, wp)[0] -
              onet.increment_loss_grad(onet.unpack(pm, 16, 16, 16), x, t, m, wp)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9, (q, fd, g[q])
    # the pressure term sees only surface nodes: changing the target elsewhere changes nothing
    t2 = t.copy()
    t2[0, ..., 3] += 5.0
    assert onet.increment_loss_grad(layers, x, t2, m, wp)[0] == loss


def test_increment_features_closed_forms():
    """Channels of the increment mode on a hand-made state: the secant factor of d^1.5,
    the gap of a surface node right below the sphere, the pressure normalisation."""
    nz, ny, nx = 3, 4, 5
    x = np.zeros((nz, ny, nx, 16))
    u1 = np.zeros((3, nz, ny, nx))
    u2 = np.zeros((3, nz, ny, nx))
    u1[2] = -0.3
    u2[2] = -0.1
    depth = (1.0, 2.0, 3.0)
    s = (3.0 ** 1.5 - 2.0 ** 1.5) / (2.0 ** 1.5 - 1.0)
    surf = [(2, 1, 2), (0, 0, 2)]
    R = 10.0
    center = (2.0, 1.0, 2.0 + R + 0.5)      # 0.5 above the top node (2, 1, 2) before it moves
    f = onet.increment_features(x, u1, u2, [-2.0, -0.5], depth, surf, center, R)
    assert np.allclose(f[..., 6], -0.2 * s)   # secant over dd = 1
    assert np.allclose(f[..., 4:6], 0.0)
    # node (2, 1, 2) moves by -0.3 + (-0.2 s): its gap is 0.5 + 0.3 + 0.2 s
    assert np.isclose(f[2, 1, 2, 8], 0.5 + 0.3 + 0.2 * s)
    assert f[2, 1, 2, 7] == 1.0 and f[2, 0, 0, 7] == 1.0 and f[1, 1, 2, 7] == 0.0
    assert np.isclose(f[2, 1, 2, 9], 1.0) and np.isclose(f[2, 0, 0, 9], 0.25)
