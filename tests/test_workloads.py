"""The seeded generator of the batched-cell workload draws what its recipe states."""
import numpy as np

import workloads as wl


def test_batch_cells_follow_the_recipe():
    cells = wl.batch_cells(24, seed0=1000)
    sizes = set()
    for c in cells:
        n = c["nvox"][0]
        sizes.add(n)
        assert c["nvox"] == (n, n, n) and n in (32, 48, 64, 96)
        bc = c["bc"]
        for d in range(3):
            per = bc[d] == wl.P
            assert per.all() or not per.any()       # periodic axes: all faces, all components
        for comp in range(3):
            assert (bc[:, :, comp] == wl.D).any()   # a Dirichlet face per component
        # inclusions: inside the cell, radius in [3, 10], pairwise disjoint
        sp = c["spheres"]
        for k, (ctr, r) in enumerate(sp):
            assert 3.0 <= r <= 10.0 and np.all(ctr >= r) and np.all(ctr <= n - r)
            for ctr2, r2 in sp[:k]:
                assert np.linalg.norm(ctr - ctr2) >= r + r2
        vf = c["phase"].mean()
        assert 0.1 <= c["vf_target"] <= 0.3
        assert vf >= c["vf_target"] or len(sp) > 0
        # pins: interior nodes, not on a Dirichlet face of their component, distinct
        seen = set()
        assert len(c["intents"]) <= 16
        for it in c["intents"]:
            assert it["kind"] == "strong" and it["value"] == 0.0
            assert all(1 <= it["ijk"][d] <= n - 1 for d in range(3))
            assert not wl.on_dirichlet(c["nvox"], bc, it["ijk"], it["comp"])
            key = (it["ijk"], it["comp"])
            assert key not in seen
            seen.add(key)
        e = c["eps_star"]
        assert np.allclose(e, e.T) and np.abs(e).max() <= 1e-3
        assert c["lam"][1] / c["lam"][0] == 10.0 and c["mu"][1] / c["mu"][0] == 10.0
    assert len(sizes) >= 3


def test_batch_cells_are_reproducible():
    a = wl.batch_cell(1234)
    b = wl.batch_cell(1234)
    assert np.array_equal(a["phase"], b["phase"]) and np.array_equal(a["bc"], b["bc"])
    assert a["intents"] == b["intents"]


def test_indentation_cube_follows_the_benchmark_geometry():
    w = wl.indentation_cube(65, steps=80, dmax=0.2)
    I = w["indenter"]
    assert w["nvox"] == (65, 65, 65) and I["radius"] == 32.5
    assert np.allclose(np.diff(I["ratios"]), 0.2 / 80) and np.isclose(I["ratios"][-1], 0.2)
    # depth d = (n + R) - centre_z, measured from the undeformed top face
    d = np.array([65 + 32.5 - c[2] for c in I["centers"]])
    assert np.allclose(d, I["ratios"] * 32.5)
    assert np.allclose([c[:2] for c in I["centers"]], 32.5)
    assert (w["bc"][2, 0] == wl.D).all() and (w["bc"][2, 1] == wl.N).all()
    assert (w["bc"][:2] == wl.N).all()
    assert w["lam0"] == w["lam"][0] and w["mu0"] == w["mu"][0]


def test_ct_specimen_follows_the_paper_set_up():
    for load in wl.CT_LOADS:
        w = wl.ct_specimen(load)
        assert w["nvox"] == (10, 100, 51)
        assert (w["phase"][0] == 1).all() and (w["phase"][1:] == 0).all()
        assert w["lam"][1] == 0.0 and w["mu"][1] == 0.0
        assert w["bc"][2, 0, 2] == wl.D and (np.delete(w["bc"].reshape(-1), 2 * 6 + 2) == wl.N).all()
        lig = w["intents"][:w["ligament_rows"]]
        assert len(lig) == 561
        assert all(it["kind"] == "strong" and it["comp"] == 2 and it["value"] == 0.0 and it["ijk"][2] == 1
                   and 50 <= it["ijk"][1] <= 100 for it in lig)
        load_rows = w["intents"][w["ligament_rows"]:]
        assert all(it["comp"] == 2 and it["value"] == 10.0 for it in load_rows)
        if load == "strong_line":
            assert sorted(it["ijk"] for it in load_rows) == [(i, 24, 25) for i in range(11)]
        elif load == "weak_line":
            (row,) = load_rows
            assert row["kind"] == "tie" and len(set(row["nodes"])) == 44
            assert {n[1] for n in row["nodes"]} == {24, 25} and {n[2] for n in row["nodes"]} == {25, 26}
        else:
            (row,) = load_rows
            kind = {"strong_node": "strong", "weak_node": "weak_voxel", "smooth_node": "smooth"}[load]
            assert row["kind"] == kind
            assert row.get("ijk", row.get("vox")) == (2, 24, 25)


def test_indentation_with_inclusions_follows_the_recipe():
    for seed in (2000, 2001):
        w = wl.indentation_inclusions(seed, 96, 96, 48, steps=10)
        sp = w["spheres"]
        assert 2 <= len(sp) <= 8
        for k, (c, r) in enumerate(sp):
            assert 8 <= r <= 32 and np.all(c >= r) and np.all(c <= np.array([96, 96, 48]) - r)
            for c2, r2 in sp[:k]:
                assert np.linalg.norm(c - c2) >= r + r2
        assert 0.005 <= w["d_over_R"] <= 0.05 and np.isclose(w["indenter"]["ratios"][-1], w["d_over_R"])
        assert w["indenter"]["radius"] == 24.0 and w["lam"][1] / w["lam"][0] == 5.0
        assert w["phase"].any() and (w["bc"][2, 0] == wl.D).all()
