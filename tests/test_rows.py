"""The host-side constraint rows handed to dtt_set_constraints (paper_2607_26082_b300.rows)
against the oracle's own rows (oracle/constraints.py), built separately from the same
intents: every row prescribes the same combination A u = U (Sections 4.1-4.2: strong,
weak, smooth and tie rows) and spreads its reaction with the same B, entry by entry, on
random cells of every boundary kind (periodic axes included), the paper's CT-like
specimen under each loading, and the 16^3 cube."""
import numpy as np
import pytest

import workloads as wl
from oracle import constraints as ocs, discrete as odz
from paper_2607_26082_b300 import rows


def _csr_rows(spec):
    ptr, node, comp, a, b, val = rows.csr_from_intents(spec["nvox"], spec["bc"], spec["intents"])
    out = []
    for r in range(len(val)):
        ent = {}
        for e in range(ptr[r], ptr[r + 1]):
            k = (int(node[e]), int(comp[e]))
            pa, pb = ent.get(k, (0.0, 0.0))
            ent[k] = (pa + float(a[e]), pb + float(b[e]))
        out.append((ent, float(val[r])))
    return out, (ptr, node, comp, a, b, val)


def _oracle_rows(spec):
    pb = odz.problem_from(spec)
    out = []
    for row in ocs.rows_from_intents(pb, spec["intents"]):
        ent = {}
        for n, c, a, b in zip(row.nodes, row.comps, row.a, row.b):
            k = (int(n), int(c))
            pa, pbb = ent.get(k, (0.0, 0.0))
            ent[k] = (pa + float(a), pbb + float(b))
        out.append((ent, row.value))
    return out


def _assert_same(spec):
    got, arrays = _csr_rows(spec)
    want = _oracle_rows(spec)
    assert len(got) == len(want)
    for (ge, gv), (we, wv) in zip(got, want):
        assert gv == wv
        keys = set(ge) | set(we)
        for k in keys:
            ga, gb = ge.get(k, (0.0, 0.0))
            wa, wb = we.get(k, (0.0, 0.0))
            assert abs(ga - wa) <= 1e-15 and abs(gb - wb) <= 1e-15, (k, ge.get(k), we.get(k))
    ptr, node, comp, a, b, val = arrays
    assert ptr[0] == 0 and np.all(np.diff(ptr) >= 1) and ptr[-1] == len(node)
    nn = wl.node_counts(spec["nvox"], spec["bc"])
    assert node.min() >= 0 and node.max() < int(np.prod(nn))
    assert set(np.unique(comp)) <= {0, 1, 2}
    return len(got)


@pytest.mark.parametrize("seed", range(24))
def test_random_cells(seed):
    spec = wl.random_problem(seed, periodic_prob=0.4)
    _assert_same(spec)


@pytest.mark.parametrize("load", wl.CT_LOADS)
def test_ct_specimen_loadings(load):
    assert _assert_same(wl.ct_specimen(load)) > 0


def test_cube16():
    assert _assert_same(wl.cube16()) > 0


def test_face_rows_and_periodic_wrap():
    """Rows the workloads do not draw: weak rows over boundary faces (Eq. 10 with the four
    face nodes), smooth rows on a boundary face (the face's 3 x 3 weights), and weak-voxel,
    smooth and tie rows that wrap across periodic axes."""
    spec = wl.random_problem(3, nvox=(6, 5, 7), periodic_prob=0.0, anchored=False)
    nn = wl.node_counts(spec["nvox"], spec["bc"])
    spec["intents"] = [
        {"kind": "weak_face", "axis": 2, "face_node": 0, "lower": (1, 1), "comp": 0, "value": 0.01},
        {"kind": "weak_face", "axis": 0, "face_node": nn[0] - 1, "lower": (2, 3), "comp": 2, "value": -0.02},
        {"kind": "weak_face", "axis": 1, "face_node": nn[1] - 1, "lower": (4, 5), "comp": 1, "value": 0.0},
        {"kind": "smooth", "ijk": (0, 2, 3), "comp": 1, "value": 0.03},
        {"kind": "smooth", "ijk": (3, 2, nn[2] - 1), "comp": 0, "value": 0.0},
        {"kind": "smooth", "ijk": (3, 3, 3), "comp": 2, "value": 0.5},
    ]
    assert _assert_same(spec) == 6
    spec = wl.random_problem(4, nvox=(6, 5, 7), periodic_prob=1.0, anchored=False)
    bc = np.asarray(spec["bc"]).reshape(3, 2, 3)
    assert (bc[:, :, 0] == 0).all()
    spec["intents"] = [
        {"kind": "weak_voxel", "vox": (5, 4, 6), "comp": 0, "value": 0.1},
        {"kind": "smooth", "ijk": (0, 0, 3), "comp": 1, "value": 0.2},
        {"kind": "tie", "nodes": [(0, 1, 1), (5, 1, 1), (2, 4, 6)], "comp": 2, "value": -0.1},
    ]
    assert _assert_same(spec) == 3
