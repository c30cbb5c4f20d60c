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


# ------------------------------------------------------------ overlapping block-Jacobi
# Pins of the restricted additive Schwarz preconditioner S (ras_blocks / ras_apply)
# against what its definition fixes independently of the code: with one group spanning
# every function S is the inverse of N; on a block-diagonal N it is block-Jacobi; and
# S e_m is supported exactly on the functions whose home leaf touches the home of m.
from oracle import learned  # noqa: E402


def _homes(pre):
    o = pre.o
    return o.tree.point_leaf_ijk.reshape(-1, 7, 3)[o.rwg["tri"][:, 0], 0]


def _one_group_error(pre):
    u = random_coefficients(pre.o.n, 2, seed=66).T
    blocks = learned.ras_blocks(pre.N, np.zeros((pre.o.n, 3), int))
    z = learned.ras_apply(blocks, pre.N @ u)
    return np.linalg.norm(z - u) / np.linalg.norm(u)


def _block_diagonal_error(pre):
    nbd = np.zeros_like(pre.N)
    for g in pre.groups:
        nbd[np.ix_(g, g)] = pre.N[np.ix_(g, g)]
    u = random_coefficients(pre.o.n, 2, seed=67).T
    z = learned.ras_apply(learned.ras_blocks(nbd, _homes(pre)), u)
    ref = pre.bj(u)
    return np.linalg.norm(z - ref) / np.linalg.norm(ref)


def _support_mismatches(pre, cols=(0, 7, 101, 333)):
    home = _homes(pre)
    blocks = learned.ras_blocks(pre.N, home)
    bad = 0
    for m in cols:
        e = np.zeros(pre.o.n, complex)
        e[m] = 1.0
        z = learned.ras_apply(blocks, e)
        got = np.abs(z) > 1e-12 * np.abs(z).max()
        want = np.abs(home - home[m]).max(1) <= 1
        bad += int(np.sum(got != want))
    return bad


def test_overlapping_block_jacobi_with_one_group_is_the_inverse(pre):
    assert _one_group_error(pre) <= 1e-10


def test_overlapping_block_jacobi_on_block_diagonal_is_block_jacobi(pre):
    assert _block_diagonal_error(pre) <= 1e-12


def test_overlapping_block_jacobi_support_is_the_touching_homes(pre):
    assert _support_mismatches(pre) == 0


class _RowsOfTheWrongFunctions:
    """numpy, except that searchsorted picks the first rows of the inverse instead of
    the group's own rows (a planted mistake)."""

    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def searchsorted(E, g):
        return np.arange(len(g))


def test_planted_row_mistake_fails_the_block_diagonal_pin(pre, monkeypatch):
    monkeypatch.setattr(learned, "np", _RowsOfTheWrongFunctions())
    assert _block_diagonal_error(pre) > 1e-3


def test_planted_overlap_mistake_fails_the_support_pin(pre, monkeypatch):
    monkeypatch.setattr(learned, "touching", lambda a, b: max(abs(x - y) for x, y in zip(a, b)) <= 2)
    assert _support_mismatches(pre) > 0
