"""Failure detection on the host, through the C ABI (no GPU): meshes the library must
refuse come back as NESA_ERR_MESH with the reason in nesa_last_error, from the host
part of the build (nesa_plan runs it without a device)."""
import numpy as np
import pytest

from workloads import get_config


@pytest.fixture(scope="module")
def nesa():
    from paper_1801_03589_gb300 import build
    build.build()
    import paper_1801_03589_gb300 as m
    return m


def _refused(nesa, v, t, what):
    with pytest.raises(nesa.NesaError) as e:
        nesa.plan(v, t, 2 * np.pi)
    assert e.value.status == nesa.ERR_MESH
    assert what in nesa.lib().nesa_last_error().decode()


def test_repeated_vertex_is_a_degenerate_triangle(nesa):
    c = get_config("tiny")
    t = c["triangles"].copy()
    t[5] = (t[5, 0], t[5, 0], t[5, 1])
    _refused(nesa, c["vertices"], t, "degenerate triangle")


def test_zero_area_triangle_is_degenerate(nesa):
    c = get_config("tiny")
    v0 = c["vertices"][0]
    nv = len(c["vertices"])
    # three collinear points (exactly: the edges have zero y and z components) ...
    v = np.vstack([c["vertices"], v0 + [1e-3, 0, 0], v0 + [2e-3, 0, 0]])
    t = np.vstack([c["triangles"], [[0, nv, nv + 1]]]).astype(np.int32)
    _refused(nesa, v, t, "degenerate triangle")
    # ... and nearly collinear ones, whose area is at the rounding level of the edges
    v = np.vstack([c["vertices"], v0 * 1.0001, v0 * 1.0002])
    _refused(nesa, v, t, "degenerate triangle")


def test_vertex_index_out_of_range(nesa):
    c = get_config("tiny")
    t = c["triangles"].copy()
    t[3, 2] = len(c["vertices"])
    _refused(nesa, c["vertices"], t, "out of range")


def test_edge_of_three_triangles_is_non_manifold(nesa):
    c = get_config("tiny")
    v = np.vstack([c["vertices"], [[0.0, 0.0, 0.0]]])
    a, b = c["triangles"][0, 0], c["triangles"][0, 1]
    t = np.vstack([c["triangles"], [[a, b, len(v) - 1]]]).astype(np.int32)  # a third triangle on edge (a, b)
    _refused(nesa, v, t, "non-manifold")


def test_good_mesh_is_planned(nesa):
    c = get_config("tiny")
    info = nesa.plan(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"])
    assert info["n_unknowns"] == 480


def test_build_batch_names_the_failing_mesh(nesa):
    """nesa_build_batch returns the first failing mesh's status and index (the host part
    of the build fails before any device work)."""
    c = get_config("tiny")
    t = c["triangles"].copy()
    t[5] = (t[5, 0], t[5, 0], t[5, 1])
    with pytest.raises(nesa.NesaError) as e:
        nesa.build_batch([(c["vertices"], t), (c["vertices"], c["triangles"])], [c["k"], c["k"]])
    assert e.value.status == nesa.ERR_MESH
    msg = nesa.lib().nesa_last_error().decode()
    assert "mesh 0" in msg and "degenerate" in msg
