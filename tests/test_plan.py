"""The library's host model (nesa_plan: RWG functions, octree, lists, Q) against the
oracle's, on the CPU: the integer structure nesa_build would upload, with no GPU.

Counted from the oracle's tree: boxes and interaction pairs per level, Q per level,
and the near-field pattern.  An RWG pair is near when some quadrature point of one
and some point of the other lie in touching leaves (Sec. 2 split, 7 points per
triangle); a triangle pair likewise; a V column is an (RWG, leaf) pair where the
function has a point in the leaf.
"""
import numpy as np
import pytest

from oracle.nesa import NesaOracle
from workloads import get_config


def _touching(ijk_a, ijk_b):
    return (np.abs(ijk_a[:, None, :] - ijk_b[None, :, :]) <= 1).all(-1)


@pytest.mark.parametrize("name", ["tiny", "C1", "C1b"])
def test_host_model_matches_oracle(name):
    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    info = nesa.plan(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"])
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    t = o.tree
    assert info["device_bytes"] == 0
    assert info["n_unknowns"] == o.n and info["n_triangles"] == len(c["triangles"])
    assert info["n_points"] == 7 * len(c["triangles"])
    assert info["l0"] == o.l0 and info["n_levels"] == o.L + 1
    for l in range(o.l0, o.L + 1):
        assert info["q"][l] == o.Q[l]
        assert info["n_boxes"][l] == len(t.boxes[l])
        assert info["n_interactions"][l] == sum(len(t.interaction_list(l, b)) for b in t.boxes[l])
    # near pattern and V columns from the leaves of the quadrature points
    pl = np.asarray(t.point_leaf_ijk).reshape(len(c["triangles"]), 7, 3)
    leaves, lid = np.unique(pl.reshape(-1, 3), axis=0, return_inverse=True)
    lid = lid.reshape(len(c["triangles"]), 7)
    nl = len(leaves)
    touch = _touching(leaves, leaves)
    tri_in = np.zeros((len(c["triangles"]), nl), bool)
    tri_in[np.arange(len(c["triangles"]))[:, None], lid] = True
    tri_near = (tri_in.astype(np.int64) @ touch.astype(np.int64) @ tri_in.T.astype(np.int64)) > 0
    assert info["near_tri_pairs"] == int(tri_near.sum())
    tri = np.asarray(o.rwg["tri"])
    rwg_in = tri_in[tri[:, 0]] | tri_in[tri[:, 1]]
    rwg_near = (rwg_in.astype(np.int64) @ touch.astype(np.int64) @ rwg_in.T.astype(np.int64)) > 0
    assert info["near_nnz"] == int(rwg_near.sum())
    assert info["v_columns"] == int(rwg_in.sum())
    assert info["max_leaf_columns"] == int(rwg_in.sum(0).max())


def test_plan_rejects_bad_arguments():
    import paper_1801_03589_gb300 as nesa
    c = get_config("tiny")
    with pytest.raises(nesa.NesaError):
        nesa.plan(c["vertices"], c["triangles"], -1.0, leaf_size=c["leaf_size"], n_levels=c["n_levels"])
    with pytest.raises(nesa.NesaError):  # a triangle with a vertex index out of range
        bad = np.array(c["triangles"]).copy()
        bad[0, 0] = len(c["vertices"]) + 5
        nesa.plan(c["vertices"], bad, c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"])


@pytest.mark.parametrize("name,P", [("C1", 100), ("C1b", 150), ("C3c", 120)])
def test_points_per_leaf_depth_rule_matches_oracle(name, P):
    """The paper's depth rule (Sec. 3: subdivide while the groups average at least P
    sources), chosen by leaf_size = 0 and points_per_leaf = P: the library's host model
    and the oracle's tree pick the same depth and the same boxes and lists."""
    import paper_1801_03589_gb300 as nesa
    from oracle.tree import Tree
    c = get_config(name)
    info = nesa.plan(c["vertices"], c["triangles"], c["k"], leaf_size=0.0, n_levels=0, points_per_leaf=P)
    t = Tree(c["vertices"], c["triangles"], 0.0, 0, points_per_leaf=P)
    npts = 7 * len(c["triangles"])
    assert npts >= P * len(t.boxes[t.L])  # the rule itself, on the oracle's boxes
    deeper = Tree(c["vertices"], c["triangles"], t.width(t.L) / 2, t.L + 2)
    assert npts < P * len(deeper.boxes[deeper.L])
    assert info["n_levels"] == t.L + 1 and info["l0"] == t.l0
    for l in range(t.L + 1):
        assert info["n_boxes"][l] == len(t.boxes[l])
    for l in range(t.l0, t.L + 1):
        assert info["n_interactions"][l] == sum(len(t.interaction_list(l, b)) for b in t.boxes[l])


def test_auto_levels_from_leaf_size():
    """n_levels = 0 with a leaf size: the fewest levels whose root cube spans the mesh."""
    import paper_1801_03589_gb300 as nesa
    from oracle.tree import Tree
    c = get_config("C1b")  # r = 1 sphere: extent 2, leaf 0.25 -> root 2 = 0.25 * 2^3
    info = nesa.plan(c["vertices"], c["triangles"], c["k"], leaf_size=0.25, n_levels=0)
    t = Tree(c["vertices"], c["triangles"], 0.25, 0)
    assert info["n_levels"] == t.L + 1 == 4
    assert info["n_boxes"][t.L] == len(t.boxes[t.L])
