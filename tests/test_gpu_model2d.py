"""The 2D model problem of Sec. 3 on the GPU (real FP64) against its oracle.

Structure, exactly: the finest level, the occupied groups, the interaction pairs per
level and the number of stored near-field entries.  Products, through the C ABI:
the near part (Eq. 9), the far part (Eqs. 10-14) and their sum within 1e-10 (relative
2-norm) of the oracle's NESA product, which is itself pinned to the dense potential
(tests/test_oracle_2d.py); several right-hand sides equal their single products.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nesa2d import Nesa2D  # noqa: E402
from workloads.curve2d import charges, curve_points  # noqa: E402

TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("n,P,Q", [(3000, 30, 16), (20000, 50, 10)])
def test_model2d_parity(n, P, Q):
    import paper_1801_03589_gb300 as nesa
    x = curve_points(n, seed=1)
    q = charges(n, seed=1)
    g = nesa.Model2D(x, P, Q)
    o = Nesa2D(x, P, Q)
    t = o.tree
    info = g.info()
    assert (info["l0"], info["L"]) == (t.l0, t.L)
    for l in range(t.l0, t.L + 1):
        assert info["n_boxes"][l] == len(t.boxes[l])
        assert info["n_interactions"][l] == sum(len(t.interaction_list(l, a)) for a in t.boxes[l])
    assert info["near_entries"] == sum(len(t.leaf_points[a]) * len(t.leaf_points[b])
                                       for a in t.boxes[t.L] for b in t.near(t.L, a))
    qd = torch.from_numpy(q).cuda()
    yn = g.matvec(qd, parts=nesa.PART2D_NEAR).cpu().numpy()
    yf = g.matvec(qd, parts=nesa.PART2D_FAR).cpu().numpy()
    y = g.matvec(qd).cpu().numpy()
    on, of = o.near(q), o.far(q)
    errs = (rel(yn, on), rel(yf, of), rel(y, on + of))
    print("2D model N=%d P=%d Q=%d (L=%d): rel err near %.1e, far %.1e, whole %.1e"
          % (n, P, Q, t.L, *errs))
    assert max(errs) < TOL
    Q3 = torch.from_numpy(np.stack([charges(n, seed=s) for s in (2, 3, 4)])).cuda()
    Y3 = g.matvec(Q3).cpu().numpy()
    for r in range(3):
        assert rel(Y3[r], g.matvec(Q3[r].contiguous()).cpu().numpy()) < 1e-14
    g.close()
