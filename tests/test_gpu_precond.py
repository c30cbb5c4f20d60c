"""Preconditioners on the GPU against the oracle (oracle/learned.py), and what they
gain in GMRES iterations.

* features and block-Jacobi: element by element against the oracle;
* loss and gradient of the network (FP32 kernels) against the oracle's FP64 backward
  pass (which is itself pinned by finite differences), tolerance 2e-4 relative;
* training lowers the loss and the trained network needs fewer GMRES iterations than
  block-Jacobi on a right-hand side it was not trained on.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.learned import NPARAM, Preconditioner, initial_theta  # noqa: E402
from oracle.nesa import NesaOracle  # noqa: E402
from workloads import get_config, plane_wave_directions, random_coefficients  # noqa: E402

_cache = {}


def pair(name):
    import paper_1801_03589_gb300 as nesa
    if name not in _cache:
        c = get_config(name)
        g = nesa.Nesa(c["vertices"], c["triangles"], c["k"], leaf_size=c["leaf_size"], n_levels=c["n_levels"])
        o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
        _cache[name] = (c, g, Preconditioner(o))
    return _cache[name]


def test_features_match_oracle():
    c, g, p = pair("tiny")
    f = g.precond_features()
    assert np.abs(f - p.features).max() <= 2e-6 * np.abs(p.features).max()


def test_block_jacobi_matches_oracle():
    import paper_1801_03589_gb300 as nesa
    c, g, p = pair("C1")
    x = random_coefficients(g.n, 2, seed=71)
    z = g.precond_apply(torch.from_numpy(x).cuda(), nesa.PRECOND_BLOCK_JACOBI).cpu().numpy()
    ref = p.bj(x.T).T
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)


def test_loss_and_gradient_match_oracle():
    c, g, p = pair("tiny")
    rng = np.random.default_rng(72)
    theta = (initial_theta() + 0.05 * rng.standard_normal(NPARAM)).astype(np.float32)
    g.precond_params(theta)
    U = random_coefficients(g.n, 5, seed=73)
    V = random_coefficients(g.n, 5, seed=74)
    loss, grad = g.precond_loss_grad(torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda())
    L, G = p.loss_grad(theta.astype(np.float64), U.T, V.T)
    print("loss gpu %.8e oracle %.8e; grad rel err %.2e" % (loss, L, np.linalg.norm(grad - G) / np.linalg.norm(G)))
    assert abs(loss - L) <= 1e-5 * abs(L)
    assert np.linalg.norm(grad - G) <= 2e-4 * np.linalg.norm(G)


def test_learned_apply_matches_oracle():
    import paper_1801_03589_gb300 as nesa
    c, g, p = pair("tiny")
    rng = np.random.default_rng(75)
    theta = (initial_theta() + 0.05 * rng.standard_normal(NPARAM)).astype(np.float32)
    g.precond_params(theta)
    x = random_coefficients(g.n, 2, seed=76)
    z = g.precond_apply(torch.from_numpy(x).cuda(), nesa.PRECOND_LEARNED).cpu().numpy()
    # inference uses FP16 weights: compare with the oracle at the FP16-rounded weights
    th16 = theta.astype(np.float16).astype(np.float64)
    ref = p.apply(th16, x.T).T
    assert np.linalg.norm(z - ref) <= 1e-5 * np.linalg.norm(ref)


def test_overlapping_block_jacobi_matches_oracle():
    import paper_1801_03589_gb300 as nesa
    c, g, p = pair("C1")
    x = random_coefficients(g.n, 2, seed=79)
    z = g.precond_apply(torch.from_numpy(x).cuda(), nesa.PRECOND_OVERLAP).cpu().numpy()
    ref = p.ras(x.T).T
    # complex64 factorisation and product
    assert np.linalg.norm(z - ref) <= 1e-4 * np.linalg.norm(ref)


def test_preconditioner_iterations():
    import paper_1801_03589_gb300 as nesa
    c, g, p = pair("C1")
    kh, pol = plane_wave_directions(1, seed=77)
    b = g.rhs_planewave(kh, pol)
    its = {}
    for name, kind in (("none", nesa.PRECOND_NONE), ("block-Jacobi", nesa.PRECOND_BLOCK_JACOBI),
                       ("overlapping block-Jacobi", nesa.PRECOND_OVERLAP)):
        x, info = g.solve(b, tol=1e-5, restart=60, max_iters=3000, precond=kind)
        assert info["rel_residual"][0] <= 1e-5
        its[name] = info["iterations"]
    print("C1 iterations to 1e-5:", its)
    assert its["overlapping block-Jacobi"] < its["none"]


def test_trained_network_gain_on_held_out_rhs():
    import paper_1801_03589_gb300 as nesa
    c, g, p = pair("C1b")
    kh, pol = plane_wave_directions(3, seed=78)
    B = g.rhs_planewave(kh, pol)
    held = B[2:3].contiguous()
    _, inone = g.solve(held, tol=1e-5, restart=60, max_iters=3000)
    _, iov = g.solve(held, tol=1e-5, restart=60, max_iters=3000, precond=nesa.PRECOND_OVERLAP)
    info = g.precond_train(B[:2].contiguous(), samples=48, steps=300)
    print("training: loss %.4f -> %.4f (%d pairs, %.2f s); validation after %d steps: trained %.2e, "
          "initial %.2e, fallback %d" % (info["loss_initial"], info["loss_final"], info["samples"], info["seconds"],
                                         info["val_iters"], info["val_res_learned"], info["val_res_base"],
                                         info["fallback"]))
    assert info["loss_final"] < info["loss_initial"]
    # on this sphere the trained weights win the validation (no fallback to S)
    assert info["fallback"] == 0 and info["val_res_learned"] < info["val_res_base"]
    x, ilr = g.solve(held, tol=1e-5, restart=60, max_iters=3000, precond=nesa.PRECOND_LEARNED)
    print("C1b held-out RHS iterations to 1e-5: none %d, overlapping block-Jacobi %d, learned %d "
          "(true residual %.2e)" % (inone["iterations"], iov["iterations"], ilr["iterations"],
                                     ilr["rel_residual"][0]))
    assert ilr["rel_residual"][0] <= 1e-5
    r = held - g.matvec(x)
    assert float(r.abs().pow(2).sum().sqrt() / held.abs().pow(2).sum().sqrt()) <= 1e-5
    assert ilr["iterations"] < inone["iterations"]
    assert ilr["iterations"] <= iov["iterations"]
