"""Pins of the oracle's preconditioners (CPU): block-Jacobi inverts the diagonal
near-field blocks, the initial network is exactly block-Jacobi, and the hand-written
backward pass matches finite differences."""
import numpy as np
import pytest

from oracle.learned import NPARAM, Preconditioner, initial_theta
from oracle.nesa import NesaOracle
from workloads import get_config, random_coefficients


@pytest.fixture(scope="module")
def pre():
    c = get_config("tiny")
    o = NesaOracle(c["vertices"], c["triangles"], c["k"], c["leaf_size"], c["n_levels"])
    return Preconditioner(o)


def test_groups_partition_the_functions(pre):
    allm = np.sort(np.concatenate(pre.groups))
    assert np.array_equal(allm, np.arange(pre.o.n))


def test_block_jacobi_inverts_diagonal_blocks(pre):
    x = random_coefficients(pre.o.n, 1, seed=61)[0]
    # block-diagonal part of N applied to x, then BJ, gives x back
    y = np.zeros_like(x)
    for g in pre.groups:
        y[g] = pre.N[np.ix_(g, g)] @ x[g]
    assert np.linalg.norm(pre.bj(y) - x) <= 1e-10 * np.linalg.norm(x)


def test_initial_network_is_overlapping_block_jacobi(pre):
    U = random_coefficients(pre.o.n, 3, seed=62).T
    assert np.linalg.norm(pre.apply(initial_theta(), U) - pre.ras(U)) <= 1e-14 * np.linalg.norm(pre.ras(U))


def test_backward_matches_finite_differences(pre):
    rng = np.random.default_rng(63)
    theta = initial_theta() + 0.05 * rng.standard_normal(NPARAM)
    U = random_coefficients(pre.o.n, 4, seed=64).T
    V = random_coefficients(pre.o.n, 4, seed=65).T
    L, g = pre.loss_grad(theta, U, V)
    idx = rng.choice(NPARAM, size=40, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (pre.loss_grad(tp, U, V)[0] - pre.loss_grad(tm, U, V)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
