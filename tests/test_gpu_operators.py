"""Operator blocks exported through nesa_export_op against the oracle's (FP64).

D_l(o) (Eq. 12) is a Green's-function matrix between the equivalent points of two
boxes: compared entrywise, 1e-12.  C_l (Eq. 11) holds the regularised pseudo-inverse
K_{l-1}, whose directions of tiny singular value depend on how it is factorised (QR of
the augmented matrix here, the normal equations in the oracle).  It is compared on
what the product applies it to: equivalent sources of point currents inside the child
box, 1e-11 (measured 9e-14 on C1b; 1.2e-15 for D).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nesa import NesaOracle, green  # noqa: E402
from workloads import get_config  # noqa: E402


def test_translation_and_transfer_blocks():
    import paper_1801_03589_gb300 as nesa
    c = get_config("C1b")
    g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"])
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    info = g.info()
    l0, L = info["l0"], info["n_levels"] - 1
    assert (l0, L) == (o.l0, o.L) and L > l0
    errs_d, errs_c = [], []
    for l in range(l0, L + 1):
        noff = info["n_offsets"][l]
        for slot in sorted({0, noff // 2, noff - 1}):
            off = tuple(int(v) for v in g.export_offset(l, slot))
            Do = o.D(l, off)
            errs_d.append((l, slot, off, float(np.linalg.norm(g.export_D(l, slot) - Do) / np.linalg.norm(Do))))
    rng = np.random.default_rng(7)
    for l in range(l0 + 1, L + 1):
        w = o.tree.width(l)
        P = (rng.random((40, 3)) - 0.5) * w  # point currents inside the child box (centre 0)
        J = rng.standard_normal((40, 4)) + 1j * rng.standard_normal((40, 4))
        s = o.K[l] @ (green(o.k, o.T[l], P) @ J)
        for oc in range(8):
            Co = o.C(l, (oc & 1, (oc >> 1) & 1, (oc >> 2) & 1))
            ref = Co @ s
            errs_c.append((l, oc, float(np.linalg.norm(g.export_C(l, oc) @ s - ref) / np.linalg.norm(ref))))
    print("D blocks: max rel err %.2e over %d; C on equivalent sources: max rel err %.2e over %d"
          % (max(e[-1] for e in errs_d), len(errs_d), max(e[-1] for e in errs_c), len(errs_c)))
    assert all(e[-1] < 1e-12 for e in errs_d), errs_d
    assert all(e[-1] < 1e-11 for e in errs_c), errs_c
    with pytest.raises(nesa.NesaError):  # slot out of range
        g.export_offset(l0, info["n_offsets"][l0])
    with pytest.raises(nesa.NesaError):  # no source transfer into the coarsest far level
        g.export_C(l0, 0)
