"""GMRES on the device (nesa_solve) against the oracle's GMRES and the Mie series.

* With no restart inside the iteration budget, GMRES iterates are the unique
  minimisers of the residual over the same Krylov space, so the device and oracle
  iterates after a fixed number of steps agree up to rounding.
* A solve to 1e-6 is checked by recomputing its residual with the oracle's operator,
  and the sphere's RCS from the device solution is compared with the Mie series.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mie  # noqa: E402
from oracle.efie import ETA0  # noqa: E402
from oracle.gmres import gmres  # noqa: E402
from oracle.nesa import NesaOracle  # noqa: E402
from oracle.rhs import planewave_rhs  # noqa: E402
from workloads import get_config, plane_wave_directions  # noqa: E402

_cache = {}


def pair(name):
    if name not in _cache:
        import paper_1801_03589_gb300 as nesa
        c = get_config(name)
        o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
        g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"])
        _cache[name] = (c, o, g)
    return _cache[name]


def _b(c, o, khat=((0.0, 0.0, 1.0),), pol=((1.0, 0.0, 0.0),)):
    return planewave_rhs(c["vertices"], c["triangles"], o.rwg, c["k"], np.array(khat), np.array(pol))


def test_fixed_steps_match_oracle_gmres():
    c, o, g = pair("tiny")
    b = _b(c, o)[0]
    steps = 25
    xo, its, ok, _ = gmres(o.matvec, b, tol=1e-30, restart=steps, maxiter=steps)
    assert its == steps
    x, info = g.solve(torch.from_numpy(b).cuda().view(1, -1), tol=1e-30, restart=steps, max_iters=steps,
                      check=False)
    assert info["iterations"] == steps
    x = x.cpu().numpy()[0]
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-9


def test_solve_to_tolerance_and_true_residual():
    c, o, g = pair("C1")
    b = _b(c, o)[0]
    x, info = g.solve(torch.from_numpy(b).cuda().view(1, -1), tol=1e-6, restart=50)
    x = x.cpu().numpy()[0]
    r = np.linalg.norm(b - o.matvec(x)) / np.linalg.norm(b)
    assert r <= 1e-6 * (1 + 1e-6)
    assert abs(r - info["rel_residual"][0]) < 1e-9


def test_iteration_count_matches_oracle():
    c, o, g = pair("tiny")
    b = _b(c, o)[0]
    x, info = g.solve(torch.from_numpy(b).cuda().view(1, -1), tol=1e-5, restart=20)
    xo, its, ok, _ = gmres(o.matvec, b, tol=1e-5, restart=20)
    assert ok and abs(its - info["iterations"]) <= 1


def test_solution_rcs_matches_mie():
    c, o, g = pair("C1")
    b = _b(c, o)[0]
    x, _ = g.solve(torch.from_numpy(b).cuda().view(1, -1), tol=1e-6)
    j = x.cpu().numpy()[0]
    k = c["k"]
    th = np.linspace(0.0, math.pi, 19)
    rE = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    sE = mie.rcs_from_currents(c["vertices"], c["triangles"], o.rwg, j, k, ETA0, rE)
    mE, _ = mie.bistatic_rcs(k, 0.5, th)
    rms = math.sqrt(np.mean((10 * np.log10(sE / mE)) ** 2))
    assert rms < 0.5, rms


def test_multi_rhs_solve_matches_single():
    c, o, g = pair("C1b")
    kh, pol = plane_wave_directions(3, seed=21)
    B = g.rhs_planewave(kh, pol)
    X, info = g.solve(B, tol=1e-5, restart=40)
    assert info["converged"] == 3
    for r in range(3):
        x1, i1 = g.solve(B[r:r + 1].contiguous(), tol=1e-5, restart=40)
        assert i1["iterations"] <= info["iterations"]
        d = (X[r] - x1[0]).abs().pow(2).sum().sqrt() / x1[0].abs().pow(2).sum().sqrt()
        assert float(d) < 1e-4


def test_not_converged_status():
    import paper_1801_03589_gb300 as nesa
    c, o, g = pair("tiny")
    b = torch.from_numpy(_b(c, o)).cuda()
    x, info = g.solve(b, tol=1e-12, restart=5, max_iters=7, check=False)
    assert info["status"] == nesa.ERR_NOT_CONVERGED
    assert info["iterations"] == 7 and info["converged"] == 0
    assert np.isfinite(info["rel_residual"][0]) and info["rel_residual"][0] < 1.0
