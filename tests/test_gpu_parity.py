"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: 1e-10 relative 2-norm for every floating-point result (the operator is
built independently on both sides; differences come from rounding order only).
Integer structure (RWG numbering, leaf of every quadrature point) is bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nesa import NesaOracle  # noqa: E402
from oracle.rhs import planewave_rhs  # noqa: E402
from workloads import get_config, plane_wave_directions, random_coefficients  # noqa: E402

TOL = 1e-10


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


_cache = {}


def pair(name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        import paper_1801_03589_gb300 as nesa
        c = get_config(name)
        o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"], **kw)
        pk = {}
        if "q_mode" in kw:
            pk["q_mode"] = nesa.Q_FIXED if kw["q_mode"] == "fixed" else nesa.Q_AUTO
        if "q_fixed" in kw:
            pk["q_fixed"] = kw["q_fixed"]
        g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"], **pk)
        _cache[key] = (c, o, g)
    return _cache[key]


@pytest.mark.parametrize("name", ["tiny", "C1", "C1b", "C3a"])
def test_structure_bit_exact(name):
    c, o, g = pair(name)
    info = g.info()
    assert info["n_unknowns"] == o.n
    assert info["l0"] == o.l0 and info["n_levels"] == o.L + 1
    rw = g.export_rwg()
    assert np.array_equal(rw[:, :2], o.rwg["edge"])
    assert np.array_equal(rw[:, 2:], o.rwg["tri"])
    assert np.array_equal(g.export_point_leaf(), o.tree.point_leaf_ijk)
    for l in range(o.l0, o.L + 1):
        assert info["q"][l] == o.Q[l]
        assert info["n_boxes"][l] == len(o.tree.boxes[l])
        assert info["n_interactions"][l] == sum(len(o.tree.interaction_list(l, b)) for b in o.tree.boxes[l])


@pytest.mark.parametrize("name", ["tiny", "C1"])
def test_near_far_full_parity(name):
    import paper_1801_03589_gb300 as nesa
    c, o, g = pair(name)
    x = random_coefficients(o.n, 1, seed=11)[0]
    xd = torch.from_numpy(x).cuda().view(1, -1)
    yn = g.matvec(xd, parts=nesa.PART_NEAR).cpu().numpy()[0]
    yf = g.matvec(xd, parts=nesa.PART_FAR).cpu().numpy()[0]
    y = g.matvec(xd).cpu().numpy()[0]
    on = o.near_matrix() @ x
    of = o.far_rows(x)
    assert rel(yn, on) < TOL
    assert rel(yf, of) < TOL
    assert rel(y, on + of) < TOL


def test_fixed_q_parity():
    c, o, g = pair("tiny", q_mode="fixed", q_fixed=64)
    x = random_coefficients(o.n, 1, seed=12)[0]
    y = g.matvec(torch.from_numpy(x).cuda().view(1, -1)).cpu().numpy()[0]
    assert rel(y, o.matvec(x)) < TOL


@pytest.mark.parametrize("name", ["C1b", "C3a"])
def test_multilevel_rows_parity(name):
    c, o, g = pair(name)
    x = random_coefficients(o.n, 1, seed=13)[0]
    y = g.matvec(torch.from_numpy(x).cuda().view(1, -1)).cpu().numpy()[0]
    rows = np.unique(np.linspace(0, o.n - 1, 40).astype(np.int64))
    assert rel(y[rows], o.matvec_rows(x, rows)) < TOL


def test_multi_rhs_matches_single():
    c, o, g = pair("C1b")
    X = random_coefficients(o.n, 3, seed=14)
    Y = g.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    for r in range(3):
        y1 = g.matvec(torch.from_numpy(X[r:r + 1].copy()).cuda()).cpu().numpy()[0]
        assert rel(Y[r], y1) < 1e-14


def test_host_pointer_product():
    c, o, g = pair("C1")
    x = random_coefficients(o.n, 2, seed=15)
    yh = g.matvec_host(x)
    yd = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(yh, yd)


def test_rhs_planewave_parity():
    c, o, g = pair("C1")
    kh, pol = plane_wave_directions(3, seed=5)
    b = g.rhs_planewave(kh, pol).cpu().numpy()
    ob = planewave_rhs(c["vertices"], c["triangles"], o.rwg, c["k"], kh, pol)
    assert rel(b, ob) < TOL


def test_full_size_sampled_rows():
    # the benchmark workload (r = 3 sphere, 122,880 unknowns, 6 levels) in the launch
    # configuration the benchmark times; the oracle computes sampled rows one by one
    c, o, g = pair("C2")
    x = random_coefficients(o.n, 1, seed=16)[0]
    y = g.matvec(torch.from_numpy(x).cuda().view(1, -1)).cpu().numpy()[0]
    rows = np.unique(np.linspace(0, o.n - 1, 12).astype(np.int64))
    assert rel(y[rows], o.matvec_rows(x, rows)) < TOL


def test_invalid_arguments_rejected():
    import paper_1801_03589_gb300 as nesa
    c, o, g = pair("tiny")
    x = torch.zeros((1, o.n), dtype=torch.complex128, device="cuda")
    assert nesa.lib().nesa_matvec(g._h, x.data_ptr(), x.data_ptr() + 16, 0) == nesa.ERR_INVALID_ARG
    assert nesa.lib().nesa_matvec(g._h, x.data_ptr(), x.data_ptr(), 65) == nesa.ERR_INVALID_ARG
    with pytest.raises(nesa.NesaError) as e:
        nesa.Nesa(c["vertices"], c["triangles"][:, [0, 0, 1]], c["k"])
    assert e.value.status == nesa.ERR_MESH
    with pytest.raises(nesa.NesaError) as e:
        nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=0.01, n_levels=9)
    assert e.value.status == nesa.ERR_MESH
    with pytest.raises(nesa.NesaError) as e:
        nesa.Nesa(c["vertices"], c["triangles"], -1.0)
    assert e.value.status == nesa.ERR_INVALID_ARG


@pytest.mark.parametrize("name,P", [("C1", 100), ("C1b", 150)])
def test_points_per_leaf_build_bit_exact_and_product(name, P):
    """The paper's depth rule (Sec. 3, points_per_leaf = P with leaf_size = 0): the leaf
    of every quadrature point equals the oracle's tree built with the same rule, and the
    FP64 product matches the oracle's NESA on that tree."""
    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], 0.0, 0, points_per_leaf=P)
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=0.0, n_levels=0, points_per_leaf=P)
    info = g.info()
    assert info["n_levels"] == o.L + 1 and info["l0"] == o.l0
    assert np.array_equal(g.export_point_leaf(), o.tree.point_leaf_ijk)
    x = random_coefficients(o.n, 1, seed=17)[0]
    y = g.matvec(torch.from_numpy(x).cuda().view(1, -1)).cpu().numpy()[0]
    rows = np.unique(np.linspace(0, o.n - 1, 24).astype(np.int64))
    assert rel(y[rows], o.matvec_rows(x, rows)) < TOL
    g.close()


@pytest.mark.parametrize("name", ["tiny", "C1"])
def test_self_only_singular_mode_parity(name):
    """singular_mode = self (extraction for T = T' only): near and whole FP64 products
    against the oracle built with the same rule."""
    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"], singular_mode="self")
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"],
                  singular_mode=nesa.SINGULAR_SELF)
    x = random_coefficients(o.n, 1, seed=18)[0]
    xd = torch.from_numpy(x).cuda().view(1, -1)
    yn = g.matvec(xd, parts=nesa.PART_NEAR).cpu().numpy()[0]
    assert rel(yn, o.near_matrix() @ x) < TOL
    y = g.matvec(xd).cpu().numpy()[0]
    assert rel(y, o.matvec(x)) < TOL
    # and it differs from the default rule (the mode is not ignored)
    _, _, gt = pair(name)
    yt = gt.matvec(xd, parts=nesa.PART_NEAR).cpu().numpy()[0]
    assert rel(yn, yt) > 1e-4
    g.close()
