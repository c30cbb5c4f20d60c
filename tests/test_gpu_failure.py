"""Failure detection on the GPU without a GPU fault (through the C ABI).

* A right-hand side holding NaN stops GMRES with NESA_ERR_NUMERIC (FP64 and mixed).
* A degenerate triangle is refused by nesa_build with NESA_ERR_MESH.
* The tensor-core GEMM's bounded waits: with the producers stalled by the host-set
  hook (they issue nothing), the consumers' waits run out after a short limit, the
  kernel leaves early, nesa_device_status reports NESA_ERR_TIMEOUT, and the next
  product on the same context is correct again.  Nothing traps, faults or hangs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads import get_config, random_coefficients  # noqa: E402


def _ctx(name, **kw):
    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    return nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"], **kw)


@pytest.mark.parametrize("mixed", [False, True])
def test_nan_right_hand_side_is_a_numeric_error(mixed):
    import paper_1801_03589_gb300 as nesa
    g = _ctx("tiny", precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    b = g.rhs_planewave([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]], [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    b[1, 17] = complex(np.nan, 0.0)
    _, info = g.solve(b, tol=1e-6, check=False, mixed=mixed, max_iters=50)
    assert info["status"] == nesa.ERR_NUMERIC
    assert not np.isfinite(info["rel_residual"][1])
    g.close()


def test_degenerate_triangle_refused_by_build():
    import paper_1801_03589_gb300 as nesa
    c = get_config("tiny")
    v0, nv = c["vertices"][0], len(c["vertices"])
    v = np.vstack([c["vertices"], v0 + [1e-3, 0, 0], v0 + [2e-3, 0, 0]])
    t = np.vstack([c["triangles"], [[0, nv, nv + 1]]]).astype(np.int32)
    with pytest.raises(nesa.NesaError) as e:
        nesa.Nesa(v, t, c["k"])
    assert e.value.status == nesa.ERR_MESH
    assert b"degenerate" in nesa.lib().nesa_last_error()


@pytest.mark.parametrize("nrhs", [1, 32])
def test_stalled_tensor_gemm_times_out_and_recovers(nrhs):
    import paper_1801_03589_gb300 as nesa
    g = _ctx("C1b", precision=nesa.MIXED, translate=nesa.TRANSLATE_TENSOR)
    mixed = nesa.PART_ALL | nesa.PART_MIXED
    x = torch.from_numpy(random_coefficients(g.n, nrhs, seed=90)).cuda()
    ref = g.matvec(x, parts=mixed)  # first product: allocations and tile tuning
    torch.cuda.synchronize()
    assert g.device_status() == nesa.OK
    g.inject_stall(1, wait_limit=4096)
    y = g.matvec(x, parts=mixed)
    assert g.device_status() == nesa.ERR_TIMEOUT
    g.inject_stall(0)
    y = g.matvec(x, parts=mixed, y=y)
    assert g.device_status() == nesa.OK
    assert torch.equal(y, ref)  # owner-computes kernels: the same bits as before the stall
    g.close()
