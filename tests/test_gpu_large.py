"""The two large workloads at full size, in the configuration the benchmark times (mixed
context, translation tables chosen automatically):

* the sphere of radius 16 wavelengths (icosphere subdivision 8: 1,310,720 triangles,
  1,966,080 RWG unknowns, 9 levels, Q up to 4,096 at 8-wavelength boxes; the two
  coarsest far levels, whose FP64 tables would take 85 and 10.5 GB, are generated);
* the aircraft body scaled to 52 wavelengths (344,676 triangles, 516,413 RWG, 9 levels,
  Q = 12,544 at its 16-wavelength coarsest level, whose tables would take 181 GB).

The whole oracle product is out of reach here (its coarsest translations alone are
hundreds of 4,096 x 4,096 Green's matrices per box), so the outputs are checked in parts:

* structure: RWG numbering and the leaf of every quadrature point, bit-exact;
* near field (Eq. 9) on sampled rows against the oracle's entries, to the FP64 tolerance;
* far field (Eqs. 10-14) on sampled rows against the exact sum over the far point pairs
  (no equivalent sources at all): the NESA approximation error, bounded by 1e-3;
* the mixed product against the FP64 product on all rows, to the mixed tolerance, with
  one and with 16 right-hand sides (column 0).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.efie import ETA0, efie_rows  # noqa: E402
from oracle.nesa import channel_sources, green, apply_testing  # noqa: E402
from oracle.quadrature import triangle_points  # noqa: E402
from oracle.rwg import build_rwg  # noqa: E402
from oracle.tree import leaf_geometry, point_leaf_coords  # noqa: E402
from workloads import get_config, random_coefficients  # noqa: E402

TOL = 1e-10
TOL_TC = 5e-5
TOL_NESA = 1e-3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module", params=["C5", "C4L"])
def big(request):
    import paper_1801_03589_gb300 as nesa
    c = get_config(request.param)
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"],
                  precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    rwg = build_rwg(c["vertices"], c["triangles"])
    pts = triangle_points(c["vertices"], c["triangles"]).reshape(-1, 3)
    origin, w = leaf_geometry(c["vertices"], c["leaf_size"], c["n_levels"])
    leaf = point_leaf_coords(pts, origin, w, c["n_levels"])
    x = random_coefficients(g.n, 1, seed=2024)[0]
    xd = torch.from_numpy(x).cuda().view(1, -1)
    rows = np.unique(np.linspace(0, g.n - 1, 12).astype(np.int64))
    yield dict(nesa=nesa, c=c, g=g, rwg=rwg, pts=pts, leaf=leaf, x=x, xd=xd, rows=rows, name=request.param)
    g.close()


def test_large_structure_bit_exact(big):
    g, rwg = big["g"], big["rwg"]
    assert g.n == rwg["n"] == {"C5": 1966080, "C4L": 516413}[big["name"]]
    rw = g.export_rwg()
    assert np.array_equal(rw[:, :2], rwg["edge"]) and np.array_equal(rw[:, 2:], rwg["tri"])
    assert np.array_equal(g.export_point_leaf(), big["leaf"])


def test_large_near_rows_vs_oracle(big):
    nesa, c, g, rows = big["nesa"], big["c"], big["g"], big["rows"]
    yn = g.matvec(big["xd"], parts=nesa.PART_NEAR).cpu().numpy()[0]
    ref = efie_rows(c["vertices"], c["triangles"], big["rwg"], c["k"], rows=rows,
                    near_leaf_ijk=big["leaf"].reshape(-1, 7, 3)) @ big["x"]
    e = rel(yn[rows], ref)
    print("%s near field, 12 rows: rel err vs oracle %.2e" % (big["name"], e))
    assert e < TOL


def test_large_far_rows_vs_exact_far_field(big):
    """Far part of 6 rows against the exact sum over the far point pairs: F_p = sum over
    points q whose leaves do not touch the leaf of p of g(p, q) J_q."""
    nesa, c, g = big["nesa"], big["c"], big["g"]
    rows = big["rows"][::2]
    rwg, pts, leaf = big["rwg"], big["pts"], big["leaf"]
    J = channel_sources(c["vertices"], c["triangles"], rwg, pts, big["x"])
    F = np.zeros((len(pts), 4), np.complex128)
    for m in rows:
        for t in rwg["tri"][m]:
            for p in range(7 * t, 7 * t + 7):
                far = np.abs(leaf - leaf[p]).max(1) > 1
                F[p] = green(c["k"], pts[p:p + 1], pts[far])[0] @ J[far]
    exact = apply_testing(c["vertices"], c["triangles"], rwg, pts, c["k"], ETA0, F, rows)
    yf = g.matvec(big["xd"], parts=nesa.PART_FAR).cpu().numpy()[0][rows]
    yfm = g.matvec(big["xd"], parts=nesa.PART_FAR | nesa.PART_MIXED).cpu().numpy()[0][rows]
    e, em = rel(yf, exact), rel(yfm, exact)
    print("%s far field, 6 rows: NESA (FP64) vs exact far sum %.2e, mixed %.2e" % (big["name"], e, em))
    assert e < TOL_NESA and em < TOL_NESA


def test_large_mixed_vs_fp64(big):
    nesa, g = big["nesa"], big["g"]
    mixed = nesa.PART_ALL | nesa.PART_MIXED
    y64 = g.matvec(big["xd"]).cpu().numpy()[0]
    ym = g.matvec(big["xd"], parts=mixed).cpu().numpy()[0]
    nrhs = big["c"]["nrhs"]
    xm = torch.from_numpy(random_coefficients(g.n, nrhs, seed=2025)).cuda()
    xm[0] = big["xd"][0]
    y16 = g.matvec(xm, parts=mixed).cpu().numpy()[0]
    assert g.device_status() == nesa.OK
    e1, e16 = rel(ym, y64), rel(y16, y64)
    print("%s mixed product vs FP64: 1 RHS %.2e, column 0 of %d RHS %.2e" % (big["name"], e1, nrhs, e16))
    assert e1 < TOL_TC and e16 < TOL_TC
