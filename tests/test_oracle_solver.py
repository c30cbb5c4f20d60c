"""Pins of the oracle's solver pieces: Mie series, GMRES, and the whole EFIE solve of a
PEC sphere against the Mie series.  CPU only."""
import math

import numpy as np
import pytest

from oracle import mie
from oracle.efie import ETA0, efie_rows
from oracle.gmres import gmres
from oracle.rhs import planewave_rhs
from oracle.rwg import build_rwg
from workloads import get_config


def test_mie_rayleigh_limit():
    # small PEC sphere: monostatic RCS -> 9 pi a^2 (ka)^4
    k, a = 2 * math.pi, 0.005
    sE, _ = mie.bistatic_rcs(k, a, np.array([math.pi]))
    assert abs(sE[0] / (9 * math.pi * a * a * (k * a) ** 4) - 1.0) < 1e-3


def test_mie_large_sphere_backscatter_tends_to_geometric():
    k, a = 2 * math.pi, 20.0
    sE, sH = mie.bistatic_rcs(k, a, np.array([math.pi]))
    assert abs(sE[0] / (math.pi * a * a) - 1.0) < 0.05
    assert abs(sE[0] - sH[0]) < 1e-9 * sE[0]


@pytest.mark.parametrize("ka", [0.7, math.pi, 6.0])
def test_mie_energy_balance(ka):
    # lossless sphere: extinction (optical theorem) = scattering (series) = integral of
    # the bistatic cross sections over all directions
    k = 2 * math.pi
    a = ka / k
    csca = mie.scattering_cross_section(k, a)
    cext = mie.extinction_cross_section(k, a)
    assert abs(csca - cext) < 1e-10 * csca
    th, wt = np.polynomial.legendre.leggauss(200)
    theta = np.arccos(th)
    sE, sH = mie.bistatic_rcs(k, a, theta)
    # dsigma/dOmega = (|S2|^2 cos^2 phi + |S1|^2 sin^2 phi)/k^2 = (sE cos^2 + sH sin^2)/(4 pi)
    integral = np.sum(wt * (sE + sH) / 2.0) * 2 * math.pi / (4 * math.pi)
    assert abs(integral - csca) < 1e-8 * csca


def test_gmres_against_direct_solve():
    rng = np.random.default_rng(0)
    n = 120
    A = np.eye(n) * 4 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, its, ok, hist = gmres(lambda v: A @ v, b, tol=1e-10, restart=15)
    assert ok
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) < 1e-8 * np.linalg.norm(xd)
    # the residual recomputed at a restart carries the rounding of b - A x
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-6) for i in range(len(hist) - 1))
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)


@pytest.fixture(scope="module")
def c1_solution():
    c = get_config("C1")
    v, t, k = c["vertices"], c["triangles"], c["k"]
    r = build_rwg(v, t)
    Z = efie_rows(v, t, r, k)
    b = planewave_rhs(v, t, r, k, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))[0]
    return c, r, Z, b, np.linalg.solve(Z, b)


@pytest.mark.slow
def test_sphere_rcs_matches_mie(c1_solution):
    c, r, Z, b, j = c1_solution
    k = c["k"]
    th = np.linspace(0.0, math.pi, 37)
    rE = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    rH = np.stack([0 * th, np.sin(th), np.cos(th)], 1)
    sE = mie.rcs_from_currents(c["vertices"], c["triangles"], r, j, k, ETA0, rE)
    sH = mie.rcs_from_currents(c["vertices"], c["triangles"], r, j, k, ETA0, rH)
    mE, mH = mie.bistatic_rcs(k, 0.5, th)
    rms = math.sqrt(np.mean(np.concatenate([10 * np.log10(sE / mE), 10 * np.log10(sH / mH)]) ** 2))
    assert rms < 0.5, rms


@pytest.mark.slow
def test_excitation_sign_by_optical_theorem(c1_solution):
    # with b_m = -int E^i.phi_m the current radiates a forward field that removes power
    # from the incident wave: C_ext = -(4 pi / k) Im(p . F(khat)) must be positive and
    # equal to the Mie value (time convention exp(+i w t)); the opposite sign of b
    # gives a negative extinction
    c, r, Z, b, j = c1_solution
    k = c["k"]
    F = mie.far_field(c["vertices"], c["triangles"], r, j, k, ETA0, np.array([[0.0, 0.0, 1.0]]))[0]
    cext = -4 * math.pi / k * np.imag(F[0])
    ref = mie.extinction_cross_section(k, 0.5)
    assert abs(cext / ref - 1.0) < 0.03, (cext, ref)


@pytest.mark.slow
def test_gmres_on_efie(c1_solution):
    c, r, Z, b, j = c1_solution
    x, its, ok, _ = gmres(lambda v: Z @ v, b, tol=1e-6, restart=50)
    assert ok
    assert np.linalg.norm(b - Z @ x) <= 1e-6 * np.linalg.norm(b)
