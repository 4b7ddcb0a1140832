"""Float64 reference of the warm-start network (TEST INFRASTRUCTURE: only tests and the
smoke check use it).  The architecture, feature layout and parameter packing are those
stated in include/dtt_net.h; everything here is written from that definition with plain
numpy (no blocking, no reduced precision):

  conv(x)[v, o] = b[o] + sum_tap sum_i W[tap, o, i] x[v + off(tap), i]   (zero outside),
  tap = 9 (dz + 1) + 3 (dy + 1) + (dx + 1);
  pool = mean over 2x2x2 blocks (partial blocks at odd edges); up = nearest-neighbour.

The paper names a learned initialisation only as a prospect (Section 5.4, conclusion); the
network itself has no printed counterpart, so its pins are mathematical: the convolution
against scipy.ndimage.correlate, the backward pass against finite differences of the
loss, and the pooling / upsampling adjoint identities.
"""
import numpy as np

CIN, COUT = 16, 16


def layer_shapes(c1=16, c2=32, c3=64):
    return [(CIN, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c3), (c3, c2), (c2, c2), (c2, c1), (c1, c1),
            (c1, COUT)]


def unpack(p, c1=16, c2=32, c3=64):
    """Packed vector -> list of (W[27, cout, cin], b[cout])."""
    out, off = [], 0
    for cin, cout in layer_shapes(c1, c2, c3):
        n = 27 * cin * cout
        W = np.asarray(p[off:off + n], dtype=np.float64).reshape(27, cout, cin)
        off += n
        b = np.asarray(p[off:off + cout], dtype=np.float64)
        off += cout
        out.append((W, b))
    assert off == len(p)
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def _shift(x, dx, dy, dz):
    """s[z, y, x] = x[z + dz, y + dy, x + dx] (zero outside)."""
    nz, ny, nx = x.shape[:3]
    s = np.zeros_like(x)
    zs, ys, xs = slice(max(0, -dz), min(nz, nz - dz)), slice(max(0, -dy), min(ny, ny - dy)), \
        slice(max(0, -dx), min(nx, nx - dx))
    zt, yt, xt = slice(max(0, dz), min(nz, nz + dz)), slice(max(0, dy), min(ny, ny + dy)), \
        slice(max(0, dx), min(nx, nx + dx))
    s[zs, ys, xs] = x[zt, yt, xt]
    return s


def taps():
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                yield 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1), dx, dy, dz


def conv(x, W, b):
    y = np.zeros(x.shape[:3] + (W.shape[1],))
    for t, dx, dy, dz in taps():
        y += _shift(x, dx, dy, dz) @ W[t].T
    return y + b


def conv_backward(x, W, g):
    """g = dL/dy -> (dL/dx, dL/dW, dL/db)."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for t, dx, dy, dz in taps():
        xs = _shift(x, dx, dy, dz)
        gW[t] = np.einsum("zyxo,zyxi->oi", g, xs)
        gx += _shift(g @ W[t], -dx, -dy, -dz)
    return gx, gW, g.sum(axis=(0, 1, 2))


def pool(x):
    nz, ny, nx, C = x.shape
    cz, cy, cx = (nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2
    s = np.zeros((cz, cy, cx, C))
    cnt = np.zeros((cz, cy, cx, 1))
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                part = x[oz::2, oy::2, ox::2]
                s[:part.shape[0], :part.shape[1], :part.shape[2]] += part
                cnt[:part.shape[0], :part.shape[1], :part.shape[2]] += 1
    return s / cnt


def pool_adjoint(g, fine_shape):
    nz, ny, nx = fine_shape
    C = g.shape[3]
    cz, cy, cx = g.shape[:3]
    counts = np.zeros((cz, cy, cx, 1))
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                part = np.ones((nz, ny, nx, 1))[oz::2, oy::2, ox::2]
                counts[:part.shape[0], :part.shape[1], :part.shape[2]] += 1
    out = np.zeros((nz, ny, nx, C))
    q = g / counts
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                tgt = out[oz::2, oy::2, ox::2]
                tgt += q[:tgt.shape[0], :tgt.shape[1], :tgt.shape[2]]
    return out


def up(c, fine_shape):
    nz, ny, nx = fine_shape
    iz, iy, ix = np.arange(nz) // 2, np.arange(ny) // 2, np.arange(nx) // 2
    return c[iz][:, iy][:, :, ix]


def up_adjoint(g, coarse_shape):
    out = np.zeros(tuple(coarse_shape) + (g.shape[3],))
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                part = g[oz::2, oy::2, ox::2]
                out[:part.shape[0], :part.shape[1], :part.shape[2]] += part
    return out


def relu(a):
    return np.maximum(a, 0.0)


def forward(layers, x):
    """Returns (y, cache) with y [nz, ny, nx, 16]."""
    L = layers
    c = {"x": x}
    c["z0"] = conv(x, *L[0]); c["a0"] = relu(c["z0"])
    c["z1"] = conv(c["a0"], *L[1]); c["e1"] = relu(c["z1"])
    c["p1"] = pool(c["e1"])
    c["z2"] = conv(c["p1"], *L[2]); c["a2"] = relu(c["z2"])
    c["z3"] = conv(c["a2"], *L[3]); c["e2"] = relu(c["z3"])
    c["p2"] = pool(c["e2"])
    c["z4"] = conv(c["p2"], *L[4]); c["a4"] = relu(c["z4"])
    c["z5"] = conv(c["a4"], *L[5]); c["e3"] = relu(c["z5"])
    c["u2"] = up(c["e3"], c["e2"].shape[:3])
    c["z6"] = conv(c["u2"], *L[6]); c["d2a"] = relu(c["z6"]) + c["e2"]
    c["z7"] = conv(c["d2a"], *L[7]); c["d2"] = relu(c["z7"])
    c["u1"] = up(c["d2"], c["e1"].shape[:3])
    c["z8"] = conv(c["u1"], *L[8]); c["d1a"] = relu(c["z8"]) + c["e1"]
    c["z9"] = conv(c["d1a"], *L[9]); c["d1"] = relu(c["z9"])
    y = conv(c["d1"], *L[10])
    return y, c


def loss_and_output_grad(y, target, w=0.0):
    """loss = mean over nodes and channels 0..2 of d^2 + w s^2 sum_axis (forward difference
    of d)^2, d = y - target, s = largest node count; returns (loss, dloss/dy)."""
    V = np.prod(y.shape[:3])
    s2 = w * float(max(y.shape[:3])) ** 2
    d = y[..., :3] - target
    total = (d * d).sum()
    for ax in range(3):
        f = np.diff(d, axis=ax)
        total += s2 * (f * f).sum()
    # gradient: 2 d + 2 s^2 D^T D d, D the forward differences along each axis
    g = d.copy()
    for ax in range(3):
        f = np.diff(d, axis=ax)
        lo = [slice(None)] * 4
        hi = [slice(None)] * 4
        lo[ax] = slice(0, d.shape[ax] - 1)
        hi[ax] = slice(1, d.shape[ax])
        g[tuple(lo)] -= s2 * f
        g[tuple(hi)] += s2 * f
    gy = np.zeros_like(y)
    gy[..., :3] = 2.0 * g / (3 * V)
    return float(total / (3 * V)), gy


def loss_grad(layers, x, target, w=0.0):
    """Loss of loss_and_output_grad and its gradients per layer."""
    return loss_grad_with(layers, x, lambda y: loss_and_output_grad(y, target, w))


def increment_loss_and_output_grad(y, target, pmask, wp=1.0):
    """Increment mode (include/dtt_net.h): mean over nodes and channels 0..2 of
    (y - t)^2 plus wp times the mean over the surface nodes (pmask = 1) of (y_3 - t_3)^2;
    returns (loss, dloss/dy)."""
    V = np.prod(y.shape[:3])
    ns = float((pmask != 0).sum())
    d = y[..., :3] - target[..., :3]
    dp = (y[..., 3] - target[..., 3]) * (pmask != 0)
    loss = (d * d).sum() / (3 * V) + (wp * (dp * dp).sum() / ns if ns > 0 else 0.0)
    gy = np.zeros_like(y)
    gy[..., :3] = 2.0 * d / (3 * V)
    if ns > 0:
        gy[..., 3] = 2.0 * wp * dp / ns
    return float(loss), gy


def increment_loss_grad(layers, x, target, pmask, wp=1.0):
    return loss_grad_with(layers, x, lambda y: increment_loss_and_output_grad(y, target, pmask, wp))


def increment_features(x, u1, u2, fn_prev, depth, surface_ijk, center, radius, eps=None):
    """Channels 4..9 of the increment mode over base features x [nz, ny, nx, 16] (a copy is
    returned): u1, u2 the fields of increments k-1 and k-2 ([3, nz, ny, nx]; u2 None =
    zero), fn_prev the normal reactions of increment k-1 at surface_ijk (a list of node
    (i, j, k)), depth = (d_(k-2), d_(k-1), d_k), the sphere of increment k (centre, radius),
    eps the macroscopic strain of the affine lift (h = 1)."""
    x = np.array(x, dtype=np.float64)
    d0, d1, d2 = depth
    s = (d2 ** 1.5 - d1 ** 1.5) / (d1 ** 1.5 - d0 ** 1.5)
    dd = d2 - d1
    du = u1 - (0.0 if u2 is None else u2)
    w = du * s / dd                              # secant prediction over dd
    x[..., 4:7] = np.moveaxis(w, 0, -1)
    x[..., 7:10] = 0.0
    e = np.zeros((3, 3)) if eps is None else np.asarray(eps, float)
    fmax = max(0.0, float(np.max(-np.asarray(fn_prev)))) if len(fn_prev) else 0.0
    for q, (i, j, k) in enumerate(surface_ijk):
        X = np.array([i, j, k], float)
        M = X + e @ X + u1[:, k, j, i] + dd * w[:, k, j, i]
        gap = np.linalg.norm(M - np.asarray(center, float)) - radius
        x[k, j, i, 7] = 1.0
        x[k, j, i, 8] = min(8.0, max(-8.0, gap / dd))
        x[k, j, i, 9] = -fn_prev[q] / fmax if fmax > 0 else 0.0
    return x


def loss_grad_with(layers, x, loss_fn):
    """Loss of loss_fn(y) -> (loss, dloss/dy) and its gradients per layer."""
    y, c = forward(layers, x)
    loss, gy = loss_fn(y)
    grads = [None] * 11
    L = layers

    def step(k, inp, g, z):
        gz = g * (z > 0) if z is not None else g
        gx, gW, gb = conv_backward(inp, L[k][0], gz)
        grads[k] = (gW, gb)
        return gx

    g = step(10, c["d1"], gy, None)
    g = step(9, c["d1a"], g, c["z9"])
    ge1 = g.copy()
    g = step(8, c["u1"], g, c["z8"])
    g = up_adjoint(g, c["d2"].shape[:3])
    g = step(7, c["d2a"], g, c["z7"])
    ge2 = g.copy()
    g = step(6, c["u2"], g, c["z6"])
    g = up_adjoint(g, c["e3"].shape[:3])
    g = step(5, c["a4"], g, c["z5"])
    g = step(4, c["p2"], g, c["z4"])
    ge2 = ge2 + pool_adjoint(g, c["e2"].shape[:3])
    g = step(3, c["a2"], ge2, c["z3"])
    g = step(2, c["p1"], g, c["z2"])
    ge1 = ge1 + pool_adjoint(g, c["e1"].shape[:3])
    g = step(1, c["a0"], ge1, c["z1"])
    step(0, c["x"], g, c["z0"])
    return loss, grads, y


def features(spec):
    """Input features of a workload's nodes, [nz, ny, nx, 16] (layout of include/dtt_net.h)."""
    nvox = spec["nvox"]
    bc = np.asarray(spec["bc"])
    per = [bool(bc[d][0][0] == 0) for d in range(3)]
    nn = [nvox[d] if per[d] else nvox[d] + 1 for d in range(3)]
    lam, mu = np.asarray(spec["lam"], float), np.asarray(spec["mu"], float)
    E = np.where(lam + mu > 0, mu * (3 * lam + 2 * mu) / np.where(lam + mu > 0, lam + mu, 1.0), 0.0)
    En = E / E.max()
    ph = np.asarray(spec["phase"])           # [nz, ny, nx] voxels
    Ev = En[ph]
    x = np.zeros((nn[2], nn[1], nn[0], 16))
    acc = np.zeros((nn[2], nn[1], nn[0]))
    cnt = np.zeros((nn[2], nn[1], nn[0]))
    for oz in (-1, 0):
        for oy in (-1, 0):
            for ox in (-1, 0):
                for k in range(nn[2]):
                    vz = k + oz
                    if per[2]:
                        vz %= nvox[2]
                    elif vz < 0 or vz >= nvox[2]:
                        continue
                    for j in range(nn[1]):
                        vy = j + oy
                        if per[1]:
                            vy %= nvox[1]
                        elif vy < 0 or vy >= nvox[1]:
                            continue
                        for i in range(nn[0]):
                            vx = i + ox
                            if per[0]:
                                vx %= nvox[0]
                            elif vx < 0 or vx >= nvox[0]:
                                continue
                            acc[k, j, i] += Ev[vz, vy, vx]
                            cnt[k, j, i] += 1
    x[..., 0] = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0.0)
    fixed = np.zeros((nn[2], nn[1], nn[0], 3), bool)
    if spec.get("intents"):
        from . import constraints as ocs, discrete as odz
        pb = odz.problem_from(spec)
        for row in ocs.rows_from_intents(pb, spec["intents"]):
            for node, comp in zip(row.nodes, row.comps):
                i, j, k = node % nn[0], (node // nn[0]) % nn[1], node // (nn[0] * nn[1])
                fixed[k, j, i, comp] = True
    ind = spec.get("indenter")
    if ind:   # the contact surface's DOFs count as constrained
        sl = [slice(None)] * 3
        sl[2 - ind["axis"]] = 0 if ind["face"] == 0 else nn[ind["axis"]] - 1
        fixed[tuple(sl)] = True
    for c in range(3):
        for d in range(3):
            if per[d]:
                continue
            for f, idx in ((0, 0), (1, nn[d] - 1)):
                if bc[d][f][c] == 1:
                    sl = [slice(None)] * 3
                    sl[2 - d] = idx
                    fixed[tuple(sl) + (c,)] = True
        x[..., 1 + c] = fixed[..., c]
    e = np.asarray(spec.get("eps_star", np.zeros((3, 3))), float)
    e = 0.5 * (e + e.T)
    for q, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]):
        x[..., 4 + q] = 1000.0 * e[a, b]
    k, j, i = np.meshgrid(np.arange(nn[2]), np.arange(nn[1]), np.arange(nn[0]), indexing="ij")
    x[..., 10] = i / nvox[0]
    x[..., 11] = j / nvox[1]
    x[..., 12] = k / nvox[2]
    return x
