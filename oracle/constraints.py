"""Oracle: local kinematic constraints (strong, weak, smooth, ties) and their two
projections, plus the frictionless rigid-sphere contact geometry.

Test infrastructure only (see oracle/__init__.py).  Plain float64 numpy.

A constraint row r is a list of entries (node, component, a, b) and a target value U_r
on the TOTAL displacement u = u* + u~ (Section 4.1: the paper sets u* = 0 and prescribes
u~ directly; with a non-zero lift the natural reading is to prescribe u, so the target
on u~ is U_r - sum a u*).  Matrix A (Eq. 21, 22) holds the a's, matrix B (Eq. 23) the
b's; B = A^T except for smoothly applied rows.

  proj_U (Eq. 9, 11, 15):  u~ <- u~ + A^T (A A^T)^-1 (U - A u~)
  proj_P (Eq. 9, 14, 17):  lambda = (A B)^-1 A p,  p <- p - B lambda,  f = -lambda
Rows must have pairwise disjoint supports, so each row is projected on its own.

Row builders:
  strong  (Section 4.1.1, Eq. 21): a = b = 1 on one (node, component).
  weak    (Section 4.2.1, Eq. 10-14, Eq. 22): a = b = 1/8 on the 8 corners of a
          voxel, or 1/4 on the 4 corners of a boundary voxel face.
  smooth  (Section 4.2.2, Eq. 15-17, Table 2 of Section 4.2.2): a = 1 on the node;
          b = 1 on the node and w = 2^-m on each of its 26 (volume) or 8 (surface)
          neighbours, m = number of non-zero offsets -- which is w_MF = 1/2,
          w_ME = 1/4, w_Co = 1/8 in the volume and w_ME = 1/2, w_Co = 1/4 on a face.
  tie     (Section 4.2.3, the line-of-elements set V*): a = b = 1/|V*| on a node set.
"""
import itertools
import numpy as np


class Row:
    def __init__(self, nodes, comps, a, b, value):
        self.nodes = np.asarray(nodes, dtype=np.int64)
        self.comps = np.asarray(comps, dtype=np.int64)
        self.a = np.asarray(a, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.value = float(value)


def flat(pb, i, j, k):
    return int(i + pb.nn[0] * (j + pb.nn[1] * k))


def unflat(pb, n):
    i = n % pb.nn[0]
    j = (n // pb.nn[0]) % pb.nn[1]
    k = n // (pb.nn[0] * pb.nn[1])
    return int(i), int(j), int(k)


def strong_row(pb, ijk, comp, value):
    return Row([flat(pb, *ijk)], [comp], [1.0], [1.0], value)


def weak_voxel_row(pb, vox, comp, value):
    """Eq. 10: mean of the 8 corners of voxel vox = (i, j, k) (lower corner)."""
    nodes = []
    for dz, dy, dx in itertools.product((0, 1), repeat=3):
        ijk = [(vox[0] + dx) % pb.nn[0], (vox[1] + dy) % pb.nn[1], (vox[2] + dz) % pb.nn[2]]
        nodes.append(flat(pb, *ijk))
    return Row(nodes, [comp] * 8, [0.125] * 8, [0.125] * 8, value)


def weak_face_row(pb, axis, face_node, lower, comp, value):
    """Section 4.2.1 surface variant: mean of the 4 corners of a voxel face on the
    boundary plane  x_axis = face_node; lower = lower corner (the two in-plane indices)."""
    others = [d for d in range(3) if d != axis]
    nodes = []
    for o0, o1 in itertools.product((0, 1), repeat=2):
        ijk = [0, 0, 0]
        ijk[axis] = face_node
        ijk[others[0]] = lower[0] + o0
        ijk[others[1]] = lower[1] + o1
        nodes.append(flat(pb, *ijk))
    return Row(nodes, [comp] * 4, [0.25] * 4, [0.25] * 4, value)


def smooth_row(pb, ijk, comp, value):
    """Eq. 15-17: strong kinematic condition, reaction spread on the neighbours."""
    on_face = []
    for d in range(3):
        if not pb.periodic[d] and (ijk[d] == 0 or ijk[d] == pb.nn[d] - 1):
            on_face.append(d)
    if len(on_face) > 1:
        raise ValueError("smooth rows on edges/corners are not defined by the paper")
    nodes, a, b = [flat(pb, *ijk)], [1.0], [1.0]
    for off in itertools.product((-1, 0, 1), repeat=3):
        if off == (0, 0, 0):
            continue
        if on_face and off[on_face[0]] != 0:
            continue
        q = [ijk[d] + off[d] for d in range(3)]
        ok = True
        for d in range(3):
            if pb.periodic[d]:
                q[d] %= pb.nn[d]
            elif q[d] < 0 or q[d] >= pb.nn[d]:
                ok = False
        if not ok:
            raise ValueError("smooth row support leaves the grid")
        m = sum(1 for o in off if o != 0)
        nodes.append(flat(pb, *q))
        a.append(0.0)
        b.append(2.0 ** (-m))
    return Row(nodes, [comp] * len(nodes), a, b, value)


def tie_row(pb, node_list, comp, value):
    """Section 4.2.3: one averaged condition over a node set V*."""
    k = len(node_list)
    return Row([flat(pb, *n) for n in node_list], [comp] * k, [1.0 / k] * k, [1.0 / k] * k, value)


def check_rows(pb, rows):
    """Disjoint supports, no entry on a Dirichlet-face unknown, and no entry on a
    component whose Green symbol has null modes (discrete.has_null_modes)."""
    from .discrete import has_null_modes
    seen = set()
    masks = [pb.dof_mask(c).ravel() for c in range(3)]
    null = [has_null_modes(pb, c) for c in range(3)]
    for r in rows:
        for n, c in zip(r.nodes, r.comps):
            if null[c]:
                raise ValueError("constraint on a component with Green null modes")
            if not masks[c][n]:
                raise ValueError("constraint entry on a Dirichlet-face node")
            if (int(n), int(c)) in seen:
                raise ValueError("constraint rows overlap")
            seen.add((int(n), int(c)))


def targets(pb, rows):
    """U_r - A u* : the value each row prescribes on the fluctuation."""
    ustar = pb.lift().reshape(3, -1)
    return np.array([r.value - np.sum(r.a * ustar[r.comps, r.nodes]) for r in rows])


def proj_U(pb, u, rows, tgt):
    uf = u.reshape(3, -1)
    for r, t in zip(rows, tgt):
        aa = np.sum(r.a * r.a)
        corr = (t - np.sum(r.a * uf[r.comps, r.nodes])) / aa
        uf[r.comps, r.nodes] += r.a * corr
    return u


def proj_P(pb, p, rows):
    """Returns the multipliers f_r = -lambda_r (Eq. 17 first line for smooth rows)."""
    pf = p.reshape(3, -1)
    f = np.zeros(len(rows))
    for idx, r in enumerate(rows):
        ab = np.sum(r.a * r.b)
        lam = np.sum(r.a * pf[r.comps, r.nodes]) / ab
        pf[r.comps, r.nodes] -= r.b * lam
        f[idx] = -lam
    return f


def row_reactions(pb, rows, f):
    """Reaction force of each row, R_r = h^3 f_r sum_i W_i b_i (face nodes halved,
    edge nodes quartered, Section 4.1.3), and the total force vector."""
    Wf = [pb.weight_W(c).ravel() for c in range(3)]
    per = np.zeros(len(rows))
    tot = np.zeros(3)
    h3 = pb.h ** 3
    for idx, r in enumerate(rows):
        for n, c, b in zip(r.nodes, r.comps, r.b):
            v = h3 * Wf[c][n] * b * f[idx]
            per[idx] += v
            tot[c] += v
    return per, tot


# ---------------------------------------------------------------------------------
# Contact with a rigid sphere (Section 5.1, Eq. 24-28, Algorithm 2)
# ---------------------------------------------------------------------------------
class Indenter:
    """Sphere of centre O and radius R; the potential contact surface is face `face`
    (0 or 1) of axis `axis` -- all nodes of that face."""

    def __init__(self, pb, axis, face, center, radius):
        self.axis, self.face = int(axis), int(face)
        self.center = np.asarray(center, dtype=np.float64)
        self.radius = float(radius)
        shape = pb.node_shape
        m = np.zeros(shape, dtype=bool)
        sl = [slice(None)] * 3
        sl[2 - self.axis] = 0 if self.face == 0 else pb.nn[self.axis] - 1
        m[tuple(sl)] = True
        self.nodes = np.flatnonzero(m.ravel())


def contact_geometry(pb, ind, u):
    """Gap g = |O - M'| - R and normal n_c = (O - M')/|O - M'| at the surface nodes,
    M' = M + u*(M) + u~(M) (Section 5.1, definitions after Eq. 24 and Section 5.1.2)."""
    X = pb.node_positions().reshape(3, -1)[:, ind.nodes]
    tot = (pb.lift() + u).reshape(3, -1)[:, ind.nodes]
    Mp = X + tot
    v = ind.center[:, None] - Mp
    dist = np.sqrt(np.sum(v * v, axis=0))
    return dist - ind.radius, v / dist


def contact_proj_U(pb, ind, u, active):
    """Eq. 28 first line, sign read so that the projected point lies on the sphere:
    M' <- O - R n_c (the radial projection of M'), i.e. u(M) = O - R n_c - M.
    (The printed u~(M) = MO' + R n_c puts M' on the far side of the sphere.)"""
    _, n = contact_geometry(pb, ind, u)
    X = pb.node_positions().reshape(3, -1)[:, ind.nodes]
    ustar = pb.lift().reshape(3, -1)[:, ind.nodes]
    uf = u.reshape(3, -1)
    masks = [pb.dof_mask(c).ravel() for c in range(3)]
    target = ind.center[:, None] - ind.radius * n - X - ustar
    for q in np.flatnonzero(active):
        node = ind.nodes[q]
        for c in range(3):
            if masks[c][node]:
                uf[c, node] = target[c, q]
    return u


def contact_proj_P(pb, ind, u, p, active):
    """Eq. 28 proj_P on the active set: p <- p - (p.n_c) n_c.  Returns the normal
    reaction f = -h^3 sum_c W_c p_c n_c of every surface node, evaluated before the
    projection (Section 5.1.2: one-sided divergence with a null-stress layer outside)."""
    _, n = contact_geometry(pb, ind, u)
    pf = p.reshape(3, -1)
    W = np.stack([pb.weight_W(c).ravel()[ind.nodes] for c in range(3)])
    masks = np.stack([pb.dof_mask(c).ravel()[ind.nodes] for c in range(3)])
    pv = pf[:, ind.nodes]
    f = -(pb.h ** 3) * np.sum(W * pv * n, axis=0)
    pn = np.sum(pv * n, axis=0)
    for q in np.flatnonzero(active):
        node = ind.nodes[q]
        for c in range(3):
            if masks[c, q]:
                pf[c, node] -= pn[q] * n[c, q]
    return f, n


def rows_from_intents(pb, intents):
    """Build oracle rows from constraint intents (dicts with 'kind' in strong,
    weak_voxel, weak_face, smooth, tie)."""
    rows = []
    for it in intents:
        k = it["kind"]
        if k == "strong":
            rows.append(strong_row(pb, it["ijk"], it["comp"], it["value"]))
        elif k == "weak_voxel":
            rows.append(weak_voxel_row(pb, it["vox"], it["comp"], it["value"]))
        elif k == "weak_face":
            rows.append(weak_face_row(pb, it["axis"], it["face_node"], it["lower"], it["comp"], it["value"]))
        elif k == "smooth":
            rows.append(smooth_row(pb, it["ijk"], it["comp"], it["value"]))
        elif k == "tie":
            rows.append(tie_row(pb, it["nodes"], it["comp"], it["value"]))
        else:
            raise ValueError(k)
    return rows
