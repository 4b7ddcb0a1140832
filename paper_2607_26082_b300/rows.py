"""Host-side construction of constraint rows for dtt_set_constraints (CSR arrays).

Row kinds (each prescribes sum_e a_e u(node_e, comp) = value on the total displacement):
  strong  -- Section 4.1.1 / Eq. 21: one node, a = b = 1.
  weak    -- Section 4.2.1 / Eq. 10, 22: mean over the 8 corners of a voxel (a = b = 1/8)
             or over the 4 corners of a voxel face lying on the boundary (a = b = 1/4).
  smooth  -- Section 4.2.2 / Eq. 15-17: a = 1 on the node only; the reaction is spread with
             b = 1 on the node and 2^-m on each neighbour of the 3x3x3 block (3x3 on a
             boundary face), m = number of non-zero offsets (w_MF = 1/2, w_ME = 1/4,
             w_Co = 1/8 in the volume, w_ME = 1/2, w_Co = 1/4 on a face).
  tie     -- Section 4.2.3: mean over a node set V*, a = b = 1/|V*|.
"""
import numpy as np


def _nn(nvox, bc):
    bc = np.asarray(bc).reshape(3, 2, 3)
    return [nvox[d] if bc[d, 0, 0] == 0 else nvox[d] + 1 for d in range(3)]


class RowBuilder:
    def __init__(self, nvox, bc):
        self.nvox = tuple(int(v) for v in nvox)
        self.bc = np.asarray(bc).reshape(3, 2, 3)
        self.nn = _nn(self.nvox, self.bc)
        self.periodic = [self.bc[d, 0, 0] == 0 for d in range(3)]
        self.ptr = [0]
        self.node, self.comp, self.a, self.b, self.value = [], [], [], [], []

    def index(self, ijk):
        q = []
        for d in range(3):
            v = int(ijk[d])
            if self.periodic[d]:
                v %= self.nn[d]
            if v < 0 or v >= self.nn[d]:
                raise ValueError("node outside the grid")
            q.append(v)
        return q[0] + self.nn[0] * (q[1] + self.nn[1] * q[2])

    def _row(self, entries, value):
        for n, c, a, b in entries:
            self.node.append(n)
            self.comp.append(c)
            self.a.append(a)
            self.b.append(b)
        self.ptr.append(len(self.node))
        self.value.append(float(value))

    def strong(self, ijk, comp, value):
        self._row([(self.index(ijk), comp, 1.0, 1.0)], value)

    def weak_voxel(self, vox, comp, value):
        ent = []
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    ent.append((self.index((vox[0] + dx, vox[1] + dy, vox[2] + dz)), comp, 0.125, 0.125))
        self._row(ent, value)

    def weak_face(self, axis, face_node, lower, comp, value):
        o = [d for d in range(3) if d != axis]
        ent = []
        for s1 in (0, 1):
            for s0 in (0, 1):
                ijk = [0, 0, 0]
                ijk[axis] = face_node
                ijk[o[0]] = lower[0] + s0
                ijk[o[1]] = lower[1] + s1
                ent.append((self.index(ijk), comp, 0.25, 0.25))
        self._row(ent, value)

    def smooth(self, ijk, comp, value):
        faces = [d for d in range(3) if not self.periodic[d] and ijk[d] in (0, self.nn[d] - 1)]
        if len(faces) > 1:
            raise ValueError("smooth condition on an edge or corner")
        ent = [(self.index(ijk), comp, 1.0, 1.0)]
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    off = (ox, oy, oz)
                    m = sum(1 for v in off if v)
                    if m == 0 or (faces and off[faces[0]] != 0):
                        continue
                    ent.append((self.index([ijk[d] + off[d] for d in range(3)]), comp, 0.0, 0.5 ** m))
        self._row(ent, value)

    def tie(self, nodes, comp, value):
        k = float(len(nodes))
        self._row([(self.index(n), comp, 1.0 / k, 1.0 / k) for n in nodes], value)

    def add_intent(self, it):
        kind = it["kind"]
        if kind == "strong":
            self.strong(it["ijk"], it["comp"], it["value"])
        elif kind == "weak_voxel":
            self.weak_voxel(it["vox"], it["comp"], it["value"])
        elif kind == "weak_face":
            self.weak_face(it["axis"], it["face_node"], it["lower"], it["comp"], it["value"])
        elif kind == "smooth":
            self.smooth(it["ijk"], it["comp"], it["value"])
        elif kind == "tie":
            self.tie(it["nodes"], it["comp"], it["value"])
        else:
            raise ValueError(kind)

    def arrays(self):
        return (np.array(self.ptr, np.int32), np.array(self.node, np.int32), np.array(self.comp, np.int8),
                np.array(self.a, np.float64), np.array(self.b, np.float64), np.array(self.value, np.float64))


def csr_from_intents(nvox, bc, intents):
    rb = RowBuilder(nvox, bc)
    for it in intents:
        rb.add_intent(it)
    return rb.arrays()


def setup_grid(spec, precision, stream=None):
    """Create and configure a Grid from a mapping with keys nvox, h, bc, scheme, phase,
    lam, mu, eps_star, lam0, mu0, intents (and optionally indenter, kinematics "SS" or
    "FS", and medium "paux" or "iso")."""
    from . import dtt
    g = dtt.Grid(spec["nvox"], spec["h"], spec["bc"], spec["scheme"], precision, stream)
    g.dtt_set_material(spec["phase"], spec["lam"], spec["mu"])
    g.dtt_set_reference(spec["lam0"], spec["mu0"])
    g.dtt_set_load(np.asarray(spec.get("eps_star", np.zeros((3, 3)))))
    if spec.get("kinematics", "SS") == "FS":
        g.dtt_set_kinematics(dtt.FINITE_STRAIN)
    if spec.get("medium", "paux") == "iso":
        g.dtt_set_reference_medium(dtt.MEDIUM_ISOTROPIC)
    if spec.get("intents"):
        ptr, node, comp, a, b, val = csr_from_intents(spec["nvox"], spec["bc"], spec["intents"])
        g.dtt_set_constraints(ptr, node, comp, a, b, val)
        g.n_rows = len(val)
    else:
        g.n_rows = 0
    return g
