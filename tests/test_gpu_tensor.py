"""Mixed product with the translations on the tensor cores (tcgen05, BF16 hi/lo).

The error of the product against the FP64 oracle is printed per workload and bounded;
the bound (5e-5) is derived from the arithmetic: each operand is split into two BF16
numbers (8 significant bits each), the dropped lo.lo product and the rounding of the lo
part leave about 2^-16 relative error per product, accumulated in FP32, on the far
part only (the near part is complex64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nesa import NesaOracle  # noqa: E402
from workloads import get_config, plane_wave_directions, random_coefficients  # noqa: E402

TOL_TC = 5e-5
_cache = {}


def build(name):
    import paper_1801_03589_gb300 as nesa
    if name not in _cache:
        c = get_config(name)
        g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"],
                      precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
        _cache[name] = (c, g)
    return _cache[name]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", ["tiny", "C1", "C1b", "C3a"])
def test_tensor_product_vs_fp64(name):
    import paper_1801_03589_gb300 as nesa
    c, g = build(name)
    x = torch.from_numpy(random_coefficients(g.n, 1, seed=51)).cuda()
    yt = g.matvec(x, parts=nesa.PART_ALL | nesa.PART_MIXED).cpu().numpy()[0]
    y64 = g.matvec(x).cpu().numpy()[0]
    ytf = g.matvec(x, parts=nesa.PART_FAR | nesa.PART_MIXED).cpu().numpy()[0]
    yf64 = g.matvec(x, parts=nesa.PART_FAR).cpu().numpy()[0]
    assert nesa.lib().nesa_device_status(g._h) == nesa.OK
    e, ef = rel(yt, y64), rel(ytf, yf64)
    print("%s tensor-core mixed product: rel err vs FP64 product %.2e (far part %.2e)" % (name, e, ef))
    assert e < TOL_TC and ef < 10 * TOL_TC


def test_tensor_product_vs_oracle_rows():
    import paper_1801_03589_gb300 as nesa
    c, g = build("C1b")
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    x = random_coefficients(g.n, 1, seed=52)[0]
    y = g.matvec(torch.from_numpy(x).cuda().view(1, -1), parts=nesa.PART_ALL | nesa.PART_MIXED).cpu().numpy()[0]
    rows = np.unique(np.linspace(0, g.n - 1, 30).astype(np.int64))
    e = rel(y[rows], o.matvec_rows(x, rows))
    print("C1b tensor-core mixed product: rel err vs oracle (30 rows) %.2e" % e)
    assert e < TOL_TC


def test_tensor_multi_rhs_columns_independent():
    import paper_1801_03589_gb300 as nesa
    c, g = build("C1b")
    X = torch.from_numpy(random_coefficients(g.n, 3, seed=53)).cuda()
    Y = g.matvec(X, parts=nesa.PART_ALL | nesa.PART_MIXED).cpu().numpy()
    for r in range(3):
        y1 = g.matvec(X[r:r + 1].contiguous(), parts=nesa.PART_ALL | nesa.PART_MIXED).cpu().numpy()[0]
        assert rel(Y[r], y1) < 1e-6


def test_refined_solve_with_tensor_product():
    c, g = build("C1b")
    kh, pol = plane_wave_directions(1, seed=54)
    B = g.rhs_planewave(kh, pol)
    x, info = g.solve(B, tol=1e-5, mixed=True, restart=60, inner_tol=1e-3)
    assert info["converged"] == 1 and info["rel_residual"][0] <= 1e-5
    r = B - g.matvec(x)
    assert float(r.abs().pow(2).sum().sqrt() / B.abs().pow(2).sum().sqrt()) <= 1e-5


def test_many_rhs_near_field_partial_group():
    # 40 right-hand sides: the near field runs four rows at a time and the per-leaf
    # reception product a leaf's columns at a time, both with two right-hand sides per
    # lane (lanes 20-31 idle); every column must match its own single product
    # (different summation order in FP32: bounded by the mixed tolerance)
    import paper_1801_03589_gb300 as nesa
    c, g = build("C1b")
    X = torch.from_numpy(random_coefficients(g.n, 40, seed=57)).cuda()
    for parts in (nesa.PART_ALL, nesa.PART_NEAR, nesa.PART_FAR):
        p = parts | nesa.PART_MIXED
        Y = g.matvec(X, parts=p).cpu().numpy()
        for r in (0, 31, 32, 39):
            y1 = g.matvec(X[r:r + 1].contiguous(), parts=p).cpu().numpy()[0]
            assert rel(Y[r], y1) < TOL_TC, (parts, r, rel(Y[r], y1))


def test_many_rhs_reception_large_leaves():
    # Three levels on the r = 1 sphere: leaves a quarter of the domain wide hold more V
    # columns than the 64 of one column block of the per-leaf reception product (several
    # blocks per leaf, the last one ragged).  40 right-hand sides against their single products (the row
    # kernel's reception) and, for one column, against the oracle.
    import paper_1801_03589_gb300 as nesa
    c = get_config("C1b")
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=3,
                  precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    mc = g.info()["max_leaf_columns"]
    assert mc > 64, mc
    X = torch.from_numpy(random_coefficients(g.n, 40, seed=58)).cuda()
    for parts in (nesa.PART_ALL, nesa.PART_FAR):
        p = parts | nesa.PART_MIXED
        Y = g.matvec(X, parts=p).cpu().numpy()
        assert nesa.lib().nesa_device_status(g._h) == nesa.OK
        for r in (0, 33, 39):
            y1 = g.matvec(X[r:r + 1].contiguous(), parts=p).cpu().numpy()[0]
            assert rel(Y[r], y1) < TOL_TC, (parts, r, rel(Y[r], y1))
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], 3)
    rows = np.unique(np.linspace(0, g.n - 1, 12).astype(np.int64))
    Y = g.matvec(X, parts=nesa.PART_ALL | nesa.PART_MIXED).cpu().numpy()
    xh = X.cpu().numpy()
    e = rel(Y[39, rows], o.matvec_rows(xh[39], rows))
    print("C1b at 3 levels (max %d V columns per leaf), 40 RHS: rel err vs oracle (12 rows) %.2e" % (mc, e))
    assert e < TOL_TC


@pytest.mark.parametrize("nrhs", [16, 21, 33, 64])
def test_many_rhs_grouped_near_field(nrhs):
    # 16 or more right-hand sides: the near field runs four rows at a time over the union
    # of their columns (a row's value 0 where it lacks a column), two right-hand sides
    # per lane (all four rows per lane from 32 right-hand sides, one row per lane below,
    # where a CTA serves 16 and 21 needs a second, partly filled one); an odd count pads
    # the x rows to an even stride with zeros.  Every column
    # of the near part against the FP64 near part (complex64 values and x, FP32 sums:
    # 1e-5 as for one right-hand side), every column of the whole product against the
    # FP64 product (the mixed tolerance), and sampled rows of the last column against the
    # oracle's near rows (Eq. 9).
    import paper_1801_03589_gb300 as nesa
    c, g = build("C3a")
    X = torch.from_numpy(random_coefficients(g.n, nrhs, seed=60 + nrhs)).cuda()
    Yn = g.matvec(X, parts=nesa.PART_NEAR | nesa.PART_MIXED).cpu().numpy()
    Yn64 = g.matvec(X, parts=nesa.PART_NEAR).cpu().numpy()
    assert nesa.lib().nesa_device_status(g._h) == nesa.OK
    en = [rel(Yn[r], Yn64[r]) for r in range(nrhs)]
    Y = g.matvec(X, parts=nesa.PART_ALL | nesa.PART_MIXED).cpu().numpy()
    Y64 = g.matvec(X, parts=nesa.PART_ALL).cpu().numpy()
    ea = [rel(Y[r], Y64[r]) for r in range(nrhs)]
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    rows = np.unique(np.linspace(0, g.n - 1, 9).astype(np.int64))
    xh = X[nrhs - 1].cpu().numpy()
    eo = rel(Yn[nrhs - 1, rows], o.near_rows(rows) @ xh)
    print("C3a grouped near field, %d RHS: max rel err vs FP64 near %.2e, whole product %.2e, "
          "near rows vs oracle %.2e" % (nrhs, max(en), max(ea), eo))
    assert max(en) < 1e-5 and eo < 1e-5
    assert max(ea) < TOL_TC


@pytest.mark.parametrize("name", ["C1b", "C3a"])
def test_target_grouped_gemm_vs_fp64(name):
    # 64 right-hand sides run the transfers and translations target-grouped (a work item
    # per target box and 32 right-hand sides, its list summed in TMEM in chunks of about
    # 32 K steps that the epilogue adds in FP32): every column against the FP64 product.
    # The far part alone stays within 2^-16, the error of one BF16 hi/lo product; one
    # accumulation over a whole interaction list (thousands of MMAs) measured 2.7e-5
    # there, the chunked form 5e-6, the offset-grouped form 4e-6.
    import paper_1801_03589_gb300 as nesa
    c, g = build(name)
    X = torch.from_numpy(random_coefficients(g.n, 64, seed=59)).cuda()
    for parts in (nesa.PART_ALL, nesa.PART_FAR):
        Y = g.matvec(X, parts=parts | nesa.PART_MIXED).cpu().numpy()
        Y64 = g.matvec(X, parts=parts).cpu().numpy()
        assert nesa.lib().nesa_device_status(g._h) == nesa.OK
        errs = [rel(Y[r], Y64[r]) for r in range(64)]
        print("%s target-grouped tensor product, 64 RHS, parts %d: max rel err vs FP64 %.2e"
              % (name, parts, max(errs)))
        assert max(errs) < (TOL_TC if parts == nesa.PART_ALL else 2.0 ** -16)
