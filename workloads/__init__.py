"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws and lays out inputs (grid sizes, boundary-condition codes,
phase maps, material constants, constraint *intents*, indenter positions).  It holds
none of the solver's arithmetic: the constraint rows (their weights) are built from the
intents separately by the oracle and by the CUDA package's own host helpers.

Boundary-condition codes: 0 periodic, 1 Dirichlet, 2 Neumann; bc[axis][face][component].
Schemes: 0 TETRA2, 1 HEX1.

The paper measures on synthetic geometries of its own (a half compact-tension-like
specimen, Section 4.1.2; a spherical indentation of a cube, Section 5.4) and uses no
public dataset; the workloads below are seeded stand-ins with those structures.
"""
import numpy as np

P, D, N = 0, 1, 2
TETRA2, HEX1 = 0, 1


def lame(E, nu):
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


class Workload(dict):
    """nvox, h, bc, scheme, phase (nz,ny,nx) uint8, lam, mu, eps_star (3x3),
    intents (list of dicts), lam0, mu0, tol, acv_mod, optional indenter."""
    __getattr__ = dict.__getitem__


def node_counts(nvox, bc):
    return tuple(nvox[d] if bc[d][0][0] == P else nvox[d] + 1 for d in range(3))


def on_dirichlet(nvox, bc, ijk, c):
    """True if node ijk of component c lies on a Dirichlet face (no unknown there)."""
    for d in range(3):
        if bc[d][0][c] == P:
            continue
        if ijk[d] == 0 and bc[d][0][c] == D:
            return True
        if ijk[d] == nvox[d] and bc[d][1][c] == D:
            return True
    return False


# ---------------------------------------------------------------------------
# Cube 16^3 with a half-clamped bottom and 5 pinned interior nodes
# ---------------------------------------------------------------------------
def cube16(seed=1, n=16, scheme=TETRA2):
    """16x16x16 voxels, E=1, nu=0.3.  Bottom face z=0: u=0 on nodes with x<n/2 (strong
    rows), free elsewhere; top face: u_z = -0.01 (Dirichlet through the lift
    u*_z = -0.01 z / n); lateral faces: normal component Dirichlet (symmetry),
    tangential components Neumann; 5 seeded interior nodes pinned at u = 0."""
    rng = np.random.default_rng(seed)
    bc = np.full((3, 2, 3), N, dtype=np.int64)
    bc[0, :, 0] = D
    bc[1, :, 1] = D
    bc[2, 1, 2] = D
    lam, mu = lame(1.0, 0.3)
    eps = np.zeros((3, 3))
    eps[2, 2] = -0.01 / n
    nvox = (n, n, n)
    intents = []
    for i in range(n // 2):
        for j in range(n + 1):
            for c in range(3):
                if not on_dirichlet(nvox, bc, (i, j, 0), c):
                    intents.append(dict(kind="strong", ijk=(i, j, 0), comp=c, value=0.0))
    pins = set()
    while len(pins) < 5:
        pins.add(tuple(int(v) for v in rng.integers(1, n, size=3)))
    for ijk in sorted(pins):
        for c in range(3):
            intents.append(dict(kind="strong", ijk=ijk, comp=c, value=0.0))
    return Workload(name="cube16 + 5 pinned nodes", nvox=nvox, h=1.0, bc=bc, scheme=scheme,
                    phase=np.zeros((n, n, n), np.uint8), lam=np.array([lam]), mu=np.array([mu]),
                    eps_star=eps, intents=intents, lam0=lam, mu0=mu, tol=1e-8, acv_mod=3)


# ---------------------------------------------------------------------------
# Compact-tension-like plate
# ---------------------------------------------------------------------------
def ct_plate(nx=128, ny=128, nz=32, scheme=TETRA2, notch_scale=0.0, r0_factor=1.0):
    """Half compact-tension-like specimen in the paper's device (Section 4.1.2, Fig. 2),
    nx x ny x nz voxels (default 128 x 128 x 32), E = 210 (GPa, h = 1), nu = 0.3:
      * voxel row y in [0, 1): buffer layer of null stiffness; u_y is Dirichlet on the
        face y = 0 behind it (the buffer transmits no force);
      * crack plane y = 1: ligament nodes x >= 40 s (s = nx / 128) held at u_y = 0 (strong
        rows); notch voxels x < 40 s, y in [1, 3) are void (stiffness notch_scale * E), so
        the crack faces are traction-free;
      * one pin, a disk of radius 6 s through the thickness centred at (20 s, 1 + 24 s),
        pulled to u_y = +0.05 (strong rows) -- the specimen is the upper half of a plate whose
        two pins are pulled apart symmetrically;
      * u_z Dirichlet on z = 0 (mid-thickness symmetry plane); all other faces traction-free.
    Reference medium R0 = r0_factor * (lambda, mu) (Paux form, Section 3.2.3); tol 1e-6,
    Anderson on p~ every 2 iterations."""
    s = nx / 128.0
    bc = np.full((3, 2, 3), N, dtype=np.int64)
    bc[1, 0, 1] = D
    bc[2, 0, 2] = D
    E = 210.0
    lam, mu = lame(E, 0.3)
    lv, mv = lame(notch_scale * E, 0.3)
    xn = int(round(40 * s))
    phase = np.zeros((nz, ny, nx), np.uint8)
    phase[:, 1:3, :xn] = 1
    phase[:, 0, :] = 2
    intents = []
    for k in range(nz + 1):
        for i in range(xn, nx + 1):
            intents.append(dict(kind="strong", ijk=(i, 1, k), comp=1, value=0.0))
    r = 6.0 * s
    cx, cy = 20.0 * s, 1.0 + 24.0 * s
    for k in range(nz + 1):
        for j in range(ny + 1):
            for i in range(nx + 1):
                if (i - cx) ** 2 + (j - cy) ** 2 <= r * r:
                    intents.append(dict(kind="strong", ijk=(i, j, k), comp=1, value=0.05))
    return Workload(name="half CT-like specimen %dx%dx%d" % (nx, ny, nz), nvox=(nx, ny, nz), h=1.0,
                    bc=bc, scheme=scheme, phase=phase, lam=np.array([lam, lv, 0.0]),
                    mu=np.array([mu, mv, 0.0]), eps_star=np.zeros((3, 3)), intents=intents,
                    lam0=r0_factor * lam, mu0=r0_factor * mu, tol=1e-6, acv_mod=2,
                    ligament_rows=(nz + 1) * (nx + 1 - xn))


def indentation_inclusions(seed, nx=384, ny=384, nz=192, steps=20, contrast=5.0, scheme=TETRA2):
    """The large indentation configuration: a block of nx x ny x nz voxels (bottom clamped,
    lateral faces free, top face the contact surface) holding 2-8 non-overlapping spherical
    inclusions of radius U[8, 32] voxels (capped at half the smallest edge) and stiffness `contrast` times the matrix's
    (E = 1, nu = 0.3 both), indented by a rigid sphere of radius nx / 4 to a depth ratio
    d/R drawn from U[0.005, 0.05], reached in `steps` geometric increments from d/R = 0.001
    (or from the final ratio if it is smaller).  Reference medium 5 (lambda, mu) of the
    matrix, Anderson on p~ every 3 iterations, tolerance 1e-6."""
    rng = np.random.default_rng(seed)
    R = nx / 4.0
    w = indentation(nx, ny, nz, R=R, steps=steps, dmin=0.001, dmax=0.05, scheme=scheme)
    dR = float(rng.uniform(0.005, 0.05))
    ratios = np.geomspace(min(0.001, dR), dR, steps)
    w["indenter"]["ratios"] = ratios
    w["indenter"]["centers"] = [np.array([nx / 2.0, ny / 2.0, nz + R - r * R]) for r in ratios]
    ninc = int(rng.integers(2, 9))
    spheres = []
    tries = 0
    while len(spheres) < ninc and tries < 10000:
        tries += 1
        r = float(rng.uniform(8.0, min(32.0, min(nx, ny, nz) / 2.0 - 1.0)))
        c = np.array([rng.uniform(r, nx - r), rng.uniform(r, ny - r), rng.uniform(r, nz - r)])
        if all(np.linalg.norm(c - c2) >= r + r2 for c2, r2 in spheres):
            spheres.append((c, r))
    phase = np.zeros((nz, ny, nx), np.uint8)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    for c, r in spheres:
        phase[(x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r] = 1
    lam, mu = lame(np.array([1.0, contrast]), 0.3)
    w["phase"], w["lam"], w["mu"] = phase, lam, mu
    w["lam0"], w["mu0"] = 5 * float(lam[0]), 5 * float(mu[0])
    w["spheres"], w["d_over_R"] = spheres, dR
    w["name"] = "indentation of a %dx%dx%d block with %d inclusions, R=%g, d/R=%.4f" % (nx, ny, nz, len(spheres), R, dR)
    return w


def normal_mixed_bc(normal):
    """bc[axis][face][component] from normal[axis][face] in (D, N): the normal component takes
    that condition and the tangential components the other one (sliding wall or its
    reverse, the conditions of the isotropic reference medium, Section 3.2.3)."""
    bc = np.zeros((3, 2, 3), dtype=np.int64)
    for d in range(3):
        for f in range(2):
            for c in range(3):
                bc[d, f, c] = normal[d][f] if c == d else (N if normal[d][f] == D else D)
    return bc


def iso_cell(seed, nvox=(12, 10, 8), scheme=TETRA2, n_strong=3, eps_scale=1e-3, contrast=4.0, periodic=(0, 0, 0)):
    """Two-phase cell for the isotropic reference medium: every face normal mixed (drawn at
    random) except on the axes flagged in `periodic`, which are periodic for every
    component; a random two-phase map of stiffness ratio `contrast` (nu = 0.3), random eps*,
    and up to n_strong interior strong rows on components that have a Dirichlet face.
    Reference media: (lambda0, mu0) = the mean of the phases' Lame coefficients."""
    rng = np.random.default_rng(seed)
    normal = rng.choice([D, N], size=(3, 2))
    bc = normal_mixed_bc(normal)
    for d in range(3):
        if periodic[d]:
            bc[d] = P
    phase = (rng.random((nvox[2], nvox[1], nvox[0])) < 0.35).astype(np.uint8)
    lam, mu = lame(np.array([1.0, contrast]), 0.3)
    e = rng.uniform(-eps_scale, eps_scale, size=(3, 3))
    intents = []
    for _ in range(n_strong):
        c = int(rng.integers(0, 3))
        if not (bc[:, :, c] == D).any():
            continue
        ijk = tuple(int(rng.integers(1, nvox[d])) for d in range(3))
        if all(it["ijk"] != ijk or it["comp"] != c for it in intents):
            intents.append(dict(kind="strong", ijk=ijk, comp=c, value=float(rng.uniform(-1e-3, 1e-3))))
    return Workload(name="normal-mixed two-phase cell %dx%dx%d" % tuple(nvox), nvox=tuple(nvox), h=1.0, bc=bc,
                    scheme=scheme, phase=phase, lam=lam, mu=mu, eps_star=0.5 * (e + e.T), intents=intents,
                    lam0=float(lam.mean()), mu0=float(mu.mean()), tol=1e-6, acv_mod=2, medium="iso")


CT_LOADS = ("strong_line", "weak_line", "strong_node", "weak_node", "smooth_node")


def ct_specimen(load="strong_line", scheme=TETRA2, tol=1e-4):
    """The paper's half CT-like specimen (Section 4.1.2, Fig. 2; Section 4.2.3), axes
    (e1, e2, e3) = (x, y, z), 10 x 100 x (50 + 1) voxels:
      * voxel layer z in [0, 1) is the void buffer (null Lame coefficients); u_z is
        Dirichlet on its outer face z = 0, every other face and component is traction-free;
      * the specimen is z in [1, 51), lambda = 4.04e4, mu = 2.70e4; the paper's height
        x3 is z - 1;
      * the ligament, nodes (0:10, 50:100) of the plane x3 = 0, is held at u_z = 0 by
        strong rows; the crack (0:10, 0:50) of that plane is free;
      * the load pulls by 10 in e3 at (x2, x3) = (24, 24):
          strong_line  strong rows on the line of nodes (0:10, 24, 24);
          weak_line    one row over the 44 nodes of the line of elements with centres
                       (0.5:9.5, 24.5, 24.5): their mean u_z = 10, reaction spread evenly
                       (Eq. 10-14 with V(i0) replaced by the 44-node set);
          strong_node  one strong row at node (2, 24, 24);
          weak_node    one weak row at the element centre (2.5, 24.5, 24.5) (Eq. 10-14);
          smooth_node  one smooth row at node (2, 24, 24) (Eq. 15-17).
    Reference medium (lambda / 2, mu / 2), Anderson on p~ every 2 iterations, tol 1e-4
    (the tolerance of the paper's acceleration table)."""
    if load not in CT_LOADS:
        raise ValueError(load)
    nx, ny, nz = 10, 100, 51
    bc = np.full((3, 2, 3), N, dtype=np.int64)
    bc[2, 0, 2] = D
    lam, mu = 4.04e4, 2.70e4
    phase = np.zeros((nz, ny, nx), np.uint8)
    phase[0] = 1
    intents = []
    for j in range(50, ny + 1):
        for i in range(nx + 1):
            intents.append(dict(kind="strong", ijk=(i, j, 1), comp=2, value=0.0))
    jl, kl, U = 24, 24 + 1, 10.0
    if load == "strong_line":
        for i in range(nx + 1):
            intents.append(dict(kind="strong", ijk=(i, jl, kl), comp=2, value=U))
    elif load == "weak_line":
        nodes = [(i, jl + dy, kl + dz) for dz in (0, 1) for dy in (0, 1) for i in range(nx + 1)]
        intents.append(dict(kind="tie", nodes=nodes, comp=2, value=U))
    elif load == "strong_node":
        intents.append(dict(kind="strong", ijk=(2, jl, kl), comp=2, value=U))
    elif load == "weak_node":
        intents.append(dict(kind="weak_voxel", vox=(2, jl, kl), comp=2, value=U))
    else:
        intents.append(dict(kind="smooth", ijk=(2, jl, kl), comp=2, value=U))
    return Workload(name="CT-like specimen 10x100x(50+1), %s load" % load, nvox=(nx, ny, nz), h=1.0,
                    bc=bc, scheme=scheme, phase=phase, lam=np.array([lam, 0.0]), mu=np.array([mu, 0.0]),
                    eps_star=np.zeros((3, 3)), intents=intents, lam0=lam / 2, mu0=mu / 2, tol=tol,
                    acv_mod=2, ligament_rows=51 * (nx + 1))


# ---------------------------------------------------------------------------
# Rigid-sphere indentation
# ---------------------------------------------------------------------------
def indentation(nx=256, ny=256, nz=128, R=64.0, steps=10, dmin=0.001, dmax=0.05,
                scheme=TETRA2):
    """Elastic block (E=1, nu=0.3), bottom z=0 clamped (Dirichlet, all components),
    lateral faces traction-free, top face z=nz the potential contact surface.  Sphere of
    radius R centred above the middle of the top face; the indentation depths d/R are
    geometrically spaced from dmin to dmax over `steps` increments."""
    bc = np.full((3, 2, 3), N, dtype=np.int64)
    bc[2, 0, :] = D
    lam, mu = lame(1.0, 0.3)
    ratios = np.geomspace(dmin, dmax, steps)
    centers = [np.array([nx / 2.0, ny / 2.0, nz + R - r * R]) for r in ratios]
    return Workload(name="sphere indentation %dx%dx%d R=%g" % (nx, ny, nz, R), nvox=(nx, ny, nz),
                    h=1.0, bc=bc, scheme=scheme, phase=np.zeros((nz, ny, nx), np.uint8),
                    lam=np.array([lam]), mu=np.array([mu]), eps_star=np.zeros((3, 3)), intents=[],
                    lam0=5 * lam, mu0=5 * mu, tol=1e-6, acv_mod=3,
                    indenter=dict(axis=2, face=1, radius=R, centers=centers, ratios=ratios,
                                  E=1.0, nu=0.3))


def indentation_cube(n=65, steps=80, dmax=0.2, scheme=TETRA2):
    """Section 5.4's benchmark geometry: a cube of n^3 voxels, bottom face clamped, the
    other faces traction-free, a rigid sphere of diameter equal to the cube edge (R = n/2
    voxels) centred over the top face, pushed in `steps` equal increments to d/R = dmax.
    nu = 0.3 as for the paper's steel (lambda = 120, mu = 80 GPa), with E = 1: forces scale
    with E and iteration counts do not.  The reference medium is 1 x (lambda, mu), so that
    a multiplier of it is the paper's R0 factor."""
    w = indentation(n, n, n, R=n / 2.0, steps=steps, dmin=dmax / steps, dmax=dmax, scheme=scheme)
    ratios = np.linspace(dmax / steps, dmax, steps)
    R = n / 2.0
    w["indenter"]["ratios"] = ratios
    w["indenter"]["centers"] = [np.array([n / 2.0, n / 2.0, n + R - r * R]) for r in ratios]
    w["lam0"] = float(w["lam"][0])
    w["mu0"] = float(w["mu"][0])
    w["name"] = "sphere indentation of a %d^3 cube, R=%g, %d equal steps to d/R=%g" % (n, R, steps, dmax)
    return w


# ---------------------------------------------------------------------------
# Batches of uneven two-phase cells (training-data generation workload)
# ---------------------------------------------------------------------------
def batch_cell(seed, sizes=(32, 48, 64, 96), scheme=TETRA2, contrast=10.0, nu=0.3, max_pins=16):
    """One cubic two-phase cell: edge drawn uniformly from `sizes`; non-overlapping
    spherical inclusions (radius U[3, 10] voxels, kept inside the cell) added in random
    order until the inclusion volume fraction reaches a target drawn from U[0.1, 0.3]
    (or the placements run out); E_matrix = 1, E_inclusion = contrast, nu = 0.3 both;
    per axis the faces are periodic with probability 1/3 (all components), else each face
    and component is Dirichlet or Neumann at random, redrawn until every component has a
    Dirichlet face (no null modes); 0..max_pins interior nodes pinned at u = 0 (strong
    rows, one random component each); eps* symmetric with entries U[-1e-3, 1e-3];
    reference medium the mean of the two phases' Lame constants; Anderson on p~ every 2
    iterations, tol 1e-6."""
    rng = np.random.default_rng(seed)
    n = int(rng.choice(sizes))
    nvox = (n, n, n)
    while True:
        bc = np.zeros((3, 2, 3), dtype=np.int64)
        for d in range(3):
            if rng.random() < 1.0 / 3.0:
                bc[d] = P
            else:
                bc[d] = rng.choice([D, N], size=(2, 3))
        if all(any(bc[d, f, c] == D for d in range(3) for f in range(2)) for c in range(3)):
            break
    phase = np.zeros((n, n, n), np.uint8)
    target = rng.uniform(0.1, 0.3)
    filled = 0
    spheres = []
    tries = 0
    while filled < target * n ** 3 and tries < 2000:
        tries += 1
        r = rng.uniform(3.0, 10.0)
        if 2 * r >= n:
            continue
        c = rng.uniform(r, n - r, size=3)
        if any(np.linalg.norm(c - c2) < r + r2 for c2, r2 in spheres):
            continue
        spheres.append((c, r))
        lo = np.maximum(np.floor(c - r).astype(int), 0)
        hi = np.minimum(np.ceil(c + r).astype(int) + 1, n)
        z, y, x = np.meshgrid(np.arange(lo[2], hi[2]) + 0.5, np.arange(lo[1], hi[1]) + 0.5,
                              np.arange(lo[0], hi[0]) + 0.5, indexing="ij")
        m = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r
        phase[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]][m] = 1
        filled += int(m.sum())
    lm, mm = lame(1.0, nu)
    li, mi = lame(contrast, nu)
    npin = int(rng.integers(0, max_pins + 1))
    intents, used = [], set()
    tries = 0
    nn = node_counts(nvox, bc)
    while len(intents) < npin and tries < 1000:
        tries += 1
        ijk = tuple(int(rng.integers(1, nn[d] - 1)) for d in range(3))
        c = int(rng.integers(3))
        if (ijk, c) in used or on_dirichlet(nvox, bc, ijk, c):
            continue
        used.add((ijk, c))
        intents.append(dict(kind="strong", ijk=ijk, comp=c, value=0.0))
    a = rng.uniform(-1e-3, 1e-3, size=(3, 3))
    eps = 0.5 * (a + a.T)
    return Workload(name="two-phase cell %d^3 (seed %d)" % (n, seed), nvox=nvox, h=1.0, bc=bc, scheme=scheme,
                    phase=phase, lam=np.array([lm, li]), mu=np.array([mm, mi]), eps_star=eps, intents=intents,
                    lam0=0.5 * (lm + li), mu0=0.5 * (mm + mi), tol=1e-6, acv_mod=2,
                    spheres=spheres, vf_target=target)


def batch_cells(n_cells=256, seed0=1000, sizes=(32, 48, 64, 96), **kw):
    """n_cells cells drawn by batch_cell with seeds seed0, seed0 + 1, ..."""
    return [batch_cell(seed0 + i, sizes=sizes, **kw) for i in range(n_cells)]


# ---------------------------------------------------------------------------
# Random small problems for parity tests
# ---------------------------------------------------------------------------
def random_bc(rng, periodic_prob=0.25):
    bc = np.zeros((3, 2, 3), dtype=np.int64)
    for d in range(3):
        if rng.random() < periodic_prob:
            bc[d] = P
        else:
            bc[d] = rng.choice([D, N], size=(2, 3))
    return bc


def random_problem(seed, nvox=None, nphase=2, n_strong=3, n_weak=2, n_smooth=1, n_tie=1,
                   scheme=TETRA2, periodic_prob=0.25, eps_scale=1e-3, anchored=True):
    """Random cell with random per-face BCs, a random two-phase map, a random eps* and
    a few random constraints of every kind (disjoint supports, none on a Dirichlet-face
    unknown).  anchored=True redraws until every component has a Dirichlet face on
    two axes (no rigid or hourglass null modes)."""
    rng = np.random.default_rng(seed)
    if nvox is None:
        nvox = tuple(int(v) for v in rng.integers(4, 9, size=3))
    while True:
        bc = random_bc(rng, periodic_prob)
        if not anchored:
            break
        ok = all(sum(1 for d in range(3) if D in bc[d, :, c]) >= 2 for c in range(3))
        if ok:
            break
    nn = node_counts(nvox, bc)
    phase = rng.integers(0, nphase, size=(nvox[2], nvox[1], nvox[0])).astype(np.uint8)
    Es = np.array([1.0, 3.0, 0.5][:nphase])
    lam, mu = lame(Es, 0.3)
    e = rng.uniform(-eps_scale, eps_scale, size=(3, 3))
    eps = 0.5 * (e + e.T)
    used = set()
    intents = []

    def free(nodes_comps):
        for ijk, c in nodes_comps:
            if (tuple(ijk), c) in used or on_dirichlet(nvox, bc, ijk, c):
                return False
        return True

    def take(nodes_comps):
        for ijk, c in nodes_comps:
            used.add((tuple(ijk), c))

    def rand_node(lo=0, hi_pad=0):
        return tuple(int(rng.integers(lo, nn[d] - hi_pad)) for d in range(3))

    tries = 0
    while n_strong > 0 and tries < 1000:
        tries += 1
        ijk, c = rand_node(), int(rng.integers(3))
        if free([(ijk, c)]):
            take([(ijk, c)])
            intents.append(dict(kind="strong", ijk=ijk, comp=c, value=float(rng.uniform(-0.02, 0.02))))
            n_strong -= 1
    while n_weak > 0 and tries < 2000:
        tries += 1
        vox = tuple(int(rng.integers(0, nvox[d])) for d in range(3))
        c = int(rng.integers(3))
        sup = [(((vox[0] + a) % nn[0], (vox[1] + b) % nn[1], (vox[2] + g) % nn[2]), c)
               for g in (0, 1) for b in (0, 1) for a in (0, 1)]
        if free(sup):
            take(sup)
            intents.append(dict(kind="weak_voxel", vox=vox, comp=c, value=float(rng.uniform(-0.02, 0.02))))
            n_weak -= 1
    while n_smooth > 0 and tries < 3000:
        tries += 1
        ijk = tuple(int(rng.integers(1, nn[d] - 1)) for d in range(3))
        c = int(rng.integers(3))
        sup = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    q = [ijk[0] + dx, ijk[1] + dy, ijk[2] + dz]
                    q = [q[d] % nn[d] if bc[d][0][0] == P else q[d] for d in range(3)]
                    sup.append((tuple(q), c))
        if all(0 <= s[0][d] < nn[d] for s in sup for d in range(3)) and free(sup):
            take(sup)
            intents.append(dict(kind="smooth", ijk=ijk, comp=c, value=float(rng.uniform(-0.02, 0.02))))
            n_smooth -= 1
    while n_tie > 0 and tries < 4000:
        tries += 1
        c = int(rng.integers(3))
        base = rand_node(0, 1)
        nodes = [base, (base[0] + 1, base[1], base[2]), (base[0], base[1] + 1, base[2])]
        sup = [(n_, c) for n_ in nodes]
        if free(sup):
            take(sup)
            intents.append(dict(kind="tie", nodes=nodes, comp=c, value=float(rng.uniform(-0.02, 0.02))))
            n_tie -= 1
    return Workload(name="random cell seed %d" % seed, nvox=nvox, h=1.0, bc=bc, scheme=scheme,
                    phase=phase, lam=lam, mu=mu, eps_star=eps, intents=intents,
                    lam0=float(np.max(lam)), mu0=float(np.max(mu)), tol=1e-10, acv_mod=3)


def random_field(seed, shape, scale=1.0):
    """A seeded float64 field of the given shape."""
    return scale * np.random.default_rng(seed).standard_normal(shape)
