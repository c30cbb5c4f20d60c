"""Translations generated when used instead of stored per offset (Eq. 12: D_l(o) is the
Green's-function matrix between the equivalent points of two boxes).

* FP64 product: D filled chunk by chunk into a bounded work buffer just before the
  translations that use it.  Same values as the stored table (same formula, same
  rounding); the sum over a box's interaction list runs chunk by chunk, so the result
  equals the stored-table product up to the summation order (1e-13), and the oracle to
  the FP64 tolerance (1e-10).
* Tensor-core product: each BF16 hi/lo tile formed in the GEMM's producer warps in FP32
  (phase relative to the offset's centre distance).  Bound: the mixed tolerance 5e-5
  against the FP64 product, as for stored tiles; the far part within 2^-16.
* The complex64 CUDA-core engine on generated levels (complex64 work buffer), 1e-5.
* The export of a generated D_l(o) equals the stored one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nesa import NesaOracle  # noqa: E402
from workloads import get_config, random_coefficients  # noqa: E402

TOL = 1e-10
TOL_TC = 5e-5
_cache = {}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def ctx(name, tables, **kw):
    import paper_1801_03589_gb300 as nesa
    key = (name, tables, tuple(sorted(kw.items())))
    if key not in _cache:
        c = get_config(name)
        _cache[key] = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"],
                                n_levels=c["n_levels"], translation_tables=tables, **kw)
    return _cache[key]


@pytest.mark.parametrize("name", ["C1b", "C3a"])
def test_generated_fp64_product_equals_stored(name):
    import paper_1801_03589_gb300 as nesa
    gs, gg = ctx(name, nesa.TABLES_STORED), ctx(name, nesa.TABLES_GENERATED)
    for nrhs in (1, 3):
        x = torch.from_numpy(random_coefficients(gs.n, nrhs, seed=70 + nrhs)).cuda()
        ys, yg = gs.matvec(x).cpu().numpy(), gg.matvec(x).cpu().numpy()
        e = rel(yg, ys)
        print("%s FP64 generated vs stored, %d RHS: %.2e" % (name, nrhs, e))
        assert e < 1e-13
    info = gg.info()
    assert info["device_bytes"] < gs.info()["device_bytes"]


def test_generated_fp64_product_vs_oracle():
    import paper_1801_03589_gb300 as nesa
    c = get_config("C3a")
    g = ctx("C3a", nesa.TABLES_GENERATED)
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    x = random_coefficients(g.n, 1, seed=72)[0]
    y = g.matvec(torch.from_numpy(x).cuda().view(1, -1)).cpu().numpy()[0]
    rows = np.unique(np.linspace(0, g.n - 1, 20).astype(np.int64))
    assert rel(y[rows], o.matvec_rows(x, rows)) < TOL


@pytest.mark.parametrize("name,nrhs", [("C1b", 1), ("C3a", 1), ("C3a", 2), ("C3a", 32)])
def test_generated_tensor_product_vs_fp64(name, nrhs):
    """Every level's tiles generated in the producers (offset-grouped below 32 right-hand
    sides, target-grouped from 32)."""
    import paper_1801_03589_gb300 as nesa
    g = ctx(name, nesa.TABLES_GENERATED, precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    gs = ctx(name, nesa.TABLES_STORED, precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    x = torch.from_numpy(random_coefficients(g.n, nrhs, seed=73)).cuda()
    mixed = nesa.PART_ALL | nesa.PART_MIXED
    y64 = gs.matvec(x).cpu().numpy()
    yg = g.matvec(x, parts=mixed).cpu().numpy()
    ys = gs.matvec(x, parts=mixed).cpu().numpy()
    yfg = g.matvec(x, parts=nesa.PART_FAR | nesa.PART_MIXED).cpu().numpy()
    yf64 = gs.matvec(x, parts=nesa.PART_FAR).cpu().numpy()
    assert g.device_status() == nesa.OK
    e, es, ef = rel(yg, y64), rel(ys, y64), rel(yfg, yf64)
    print("%s %d RHS tensor product, generated tiles: %.2e vs FP64 (stored tiles %.2e), far part %.2e"
          % (name, nrhs, e, es, ef))
    assert e < TOL_TC and ef < 2.0 ** -16


def test_auto_stores_the_tables_that_fit():
    """Automatic choice: levels whose FP64 tables fit the budget (every level here) are
    stored, so the product is the stored-table product bit for bit."""
    import paper_1801_03589_gb300 as nesa
    c = get_config("C3a")
    ga, gs = [nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"],
                        precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR, translation_tables=t)
              for t in (nesa.TABLES_AUTO, nesa.TABLES_STORED)]
    assert ga.info()["device_bytes"] == gs.info()["device_bytes"]  # both fresh: nothing generated
    x = torch.from_numpy(random_coefficients(ga.n, 1, seed=74)).cuda()
    mixed = nesa.PART_ALL | nesa.PART_MIXED
    assert torch.equal(ga.matvec(x), gs.matvec(x))
    ya, ys = ga.matvec(x, parts=mixed), gs.matvec(x, parts=mixed)
    assert rel(ya.cpu().numpy(), ys.cpu().numpy()) < 1e-6  # tile widths are tuned per context
    ga.close()
    gs.close()


def test_generated_fp32_engine():
    import paper_1801_03589_gb300 as nesa
    g = ctx("C1b", nesa.TABLES_GENERATED, precision=nesa.MIXED, translate=nesa.TRANSLATE_FP32)
    x = torch.from_numpy(random_coefficients(g.n, 2, seed=75)).cuda()
    y64 = g.matvec(x).cpu().numpy()
    y32 = g.matvec(x, parts=nesa.PART_ALL | nesa.PART_MIXED).cpu().numpy()
    assert rel(y32, y64) < 1e-5


def test_export_of_generated_translation_equals_stored():
    import paper_1801_03589_gb300 as nesa
    gs, gg = ctx("C1b", nesa.TABLES_STORED), ctx("C1b", nesa.TABLES_GENERATED)
    info = gs.info()
    for l in range(info["l0"], info["n_levels"]):
        for slot in (0, info["n_offsets"][l] // 2, info["n_offsets"][l] - 1):
            assert np.array_equal(gg.export_offset(l, slot), gs.export_offset(l, slot))
            assert np.array_equal(gg.export_D(l, slot), gs.export_D(l, slot))
