"""nesa_matvec_noalloc: the product without any device allocation.

Some callers cannot let the library call cudaMalloc (work inside a stream capture,
fixed device-memory budgets, real-time loops).  nesa_matvec_noalloc runs the product
with its work vectors in a fixed 32 MiB array that is part of the library image.
These tests call it through the C ABI and compare it with nesa_matvec, twice in a
row (the array keeps the previous call's data, which must not leak into the next
result), and check that an operator too large for the array is refused.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads import get_config, random_coefficients  # noqa: E402

TOL = 1e-10


def _entry():
    import paper_1801_03589_gb300 as nesa
    f = nesa.lib().nesa_matvec_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return nesa, f


def _build(name):
    import paper_1801_03589_gb300 as nesa
    c = get_config(name)
    return nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"])


@pytest.mark.parametrize("name,nrhs", [("tiny", 1), ("C1b", 2)])
def test_noalloc_matches_matvec_twice(name, nrhs):
    """On a fresh context (no work vectors allocated yet) the no-allocation product
    comes first and must leave the context's device memory unchanged; the reference
    product comes after it.  Two calls in a row with different inputs."""
    nesa, f = _entry()
    g = _build(name)
    torch.cuda.synchronize()
    for call in range(2):
        x = torch.from_numpy(random_coefficients(g.n, nrhs, seed=40 + call)).cuda()
        y = torch.full_like(x, complex(np.nan, np.nan))
        torch.cuda.synchronize()
        before = g.info()["device_bytes"]
        assert f(g._h, x.data_ptr(), y.data_ptr(), nrhs) == nesa.OK
        torch.cuda.synchronize()
        assert g.info()["device_bytes"] == before
        ref = g.matvec(x)
        yr, rr = y.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(yr))
        assert np.linalg.norm(yr - rr) <= TOL * np.linalg.norm(rr)
    g.close()


def test_noalloc_reports_why_it_refused():
    """A refusal inside the product (here: the context belongs to a batch captured with
    another number of right-hand sides) returns the status and leaves its reason in
    nesa_last_error."""
    nesa, f = _entry()
    g = _build("tiny")
    x1 = torch.from_numpy(random_coefficients(g.n, 1, seed=44)).cuda()
    y1 = torch.empty_like(x1)
    b = nesa.Batch([g], [x1], [y1])
    x2 = torch.zeros((2, g.n), dtype=torch.complex128, device="cuda")
    y2 = torch.zeros_like(x2)
    assert f(g._h, x2.data_ptr(), y2.data_ptr(), 2) == nesa.ERR_INVALID_ARG
    assert b"batch" in nesa.lib().nesa_last_error()
    b.close()
    g.close()


def test_noalloc_rejects_operator_larger_than_scratch():
    nesa, f = _entry()
    g = _build("C1b")
    nrhs = 64  # leaf-level work vectors alone need 272 boxes x 256 columns x 100 x 16 B
    x = torch.zeros((nrhs, g.n), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    assert f(g._h, x.data_ptr(), y.data_ptr(), nrhs) == nesa.ERR_INVALID_ARG
    assert b"scratch" in nesa.lib().nesa_last_error()
    g.close()
