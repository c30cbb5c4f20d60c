"""The octree and its box lists built on the device (nesa_build) against the host model
(nesa_plan, itself pinned to the oracle's tree on the CPU) and the oracle's leaf
coordinates: every structural count equal, the leaf of every quadrature point and the
RWG numbering bit-exact.  Workloads of different shapes: spheres, a plate, the aircraft
body, and the paper's points-per-leaf depth rule."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.quadrature import triangle_points  # noqa: E402
from oracle.rwg import build_rwg  # noqa: E402
from oracle.tree import leaf_geometry, point_leaf_coords  # noqa: E402
from workloads import get_config  # noqa: E402

KEYS = ("n_unknowns", "n_points", "n_levels", "l0", "q", "n_boxes", "n_interactions", "n_offsets", "near_nnz",
        "near_tri_pairs", "v_columns", "max_leaf_columns")


@pytest.mark.parametrize("name", ["tiny", "C1", "C1b", "C3a", "C3c", "C4"])
def test_device_tree_equals_host_model(name):
    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    kw = dict(leaf_size=c["leaf_size"], n_levels=c["n_levels"])
    host = nesa.plan(c["vertices"], c["triangles"], c["k"], **kw)
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], **kw)
    dev = g.info()
    for k in KEYS:
        assert dev[k] == host[k], k
    pts = triangle_points(c["vertices"], c["triangles"]).reshape(-1, 3)
    origin, w = leaf_geometry(c["vertices"], c["leaf_size"], c["n_levels"])
    assert np.array_equal(g.export_point_leaf(), point_leaf_coords(pts, origin, w, c["n_levels"]))
    rw = g.export_rwg()
    r = build_rwg(c["vertices"], c["triangles"])
    assert np.array_equal(rw[:, :2], r["edge"]) and np.array_equal(rw[:, 2:], r["tri"])
    split = dev["build_split"]
    print("%s build split (s): %s" % (name, {k: round(v, 3) for k, v in split.items()}))
    assert split["tree_lists_device"] > 0.0
    g.close()


def test_device_tree_points_per_leaf():
    import paper_1801_03589_gb300 as nesa
    c = get_config("C1b")
    kw = dict(leaf_size=0.0, n_levels=0, points_per_leaf=150)
    host = nesa.plan(c["vertices"], c["triangles"], c["k"], **kw)
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], **kw)
    dev = g.info()
    for k in KEYS:
        assert dev[k] == host[k], k
    g.close()
