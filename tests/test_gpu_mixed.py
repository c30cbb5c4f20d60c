"""Mixed-precision product and FP64 iterative refinement.

* The low-precision product (complex64 operator copy) is compared with the FP64
  oracle; its error is printed per workload and bounded at 1e-5.
* The refined mixed solve must reach a true FP64 relative residual <= 1e-5, and, solved
  to 1e-8, agree with the FP64 solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nesa import NesaOracle  # noqa: E402
from workloads import get_config, plane_wave_directions, random_coefficients  # noqa: E402

_cache = {}


def build(name, oracle=False):
    import paper_1801_03589_gb300 as nesa
    if name not in _cache:
        c = get_config(name)
        g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"],
                      precision=nesa.MIXED)
        o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"]) if oracle else None
        _cache[name] = (c, g, o)
    return _cache[name]


@pytest.mark.parametrize("name", ["C1", "C1b"])
def test_mixed_product_error_vs_oracle(name):
    import paper_1801_03589_gb300 as nesa
    c, g, o = build(name, oracle=True)
    x = random_coefficients(g.n, 1, seed=31)[0]
    xd = torch.from_numpy(x).cuda().view(1, -1)
    ym = g.matvec(xd, parts=nesa.PART_ALL | nesa.PART_MIXED).cpu().numpy()[0]
    y64 = g.matvec(xd).cpu().numpy()[0]
    ref = o.matvec(x) if name == "C1" else None
    if ref is None:
        rows = np.unique(np.linspace(0, g.n - 1, 30).astype(np.int64))
        ref_rows = o.matvec_rows(x, rows)
        err = np.linalg.norm(ym[rows] - ref_rows) / np.linalg.norm(ref_rows)
    else:
        err = np.linalg.norm(ym - ref) / np.linalg.norm(ref)
    err64 = np.linalg.norm(ym - y64) / np.linalg.norm(y64)
    print("%s mixed product: rel err vs oracle %.2e, vs FP64 product %.2e" % (name, err, err64))
    assert err < 1e-5 and err64 < 1e-5


def test_mixed_parts_match_fp64_parts():
    import paper_1801_03589_gb300 as nesa
    c, g, _ = build("C1b")
    x = torch.from_numpy(random_coefficients(g.n, 2, seed=32)).cuda()
    for part in (nesa.PART_NEAR, nesa.PART_FAR):
        a = g.matvec(x, parts=part | nesa.PART_MIXED)
        b = g.matvec(x, parts=part)
        assert float((a - b).abs().pow(2).sum().sqrt() / b.abs().pow(2).sum().sqrt()) < 1e-5


def test_refined_solve_reaches_fp64_residual():
    c, g, _ = build("C1b")
    kh, pol = plane_wave_directions(2, seed=33)
    B = g.rhs_planewave(kh, pol)
    xm, im = g.solve(B, tol=1e-5, mixed=True, restart=50, inner_tol=1e-3)
    assert im["converged"] == 2 and max(im["rel_residual"]) <= 1e-5
    assert im["refinements"] >= 1 and im["fp64_matvecs"] == im["refinements"]
    # independent check of the true residual with the FP64 product
    r = B - g.matvec(xm)
    rel = (r.abs().pow(2).sum(1).sqrt() / B.abs().pow(2).sum(1).sqrt()).cpu().numpy()
    assert np.all(rel <= 1e-5)


def test_refined_solution_matches_fp64_solution():
    c, g, _ = build("C1b")
    kh, pol = plane_wave_directions(1, seed=34)
    B = g.rhs_planewave(kh, pol)
    x64, i64 = g.solve(B, tol=1e-8, restart=100, max_iters=3000)
    xm, im = g.solve(B, tol=1e-8, mixed=True, restart=100, max_iters=3000, max_refine=20, inner_tol=1e-4)
    d = float((xm - x64).abs().pow(2).sum().sqrt() / x64.abs().pow(2).sum().sqrt())
    print("C1b: |x_mixed - x_fp64| / |x_fp64| = %.2e (both to 1e-8); iterations fp64 %d, mixed %d (+%d FP64 products)"
          % (d, i64["iterations"], im["iterations"], im["fp64_matvecs"]))
    assert d < 1e-5
