"""Mie series for a PEC sphere and the radar cross section from surface currents.

Not in the paper; used only to pin the whole solve (scattering of a plane wave by a
perfectly conducting sphere).  Coefficients for a sphere of radius a, x = k a
(Bohren & Huffman 1983, conducting limit; Harrington 1961):
    a_n = [x j_n(x)]' / [x h_n(x)]',   b_n = j_n(x) / h_n(x),   h_n = j_n + i y_n
    S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),  S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n)
with the angular functions pi_n, tau_n of cos(theta).  Series truncated at
n_max = x + 4 x^(1/3) + 2 (Wiscombe 1980).  For an x-polarised wave travelling along +z:
    sigma_E(theta) = 4 pi |S2|^2 / k^2   (phi = 0 plane),
    sigma_H(theta) = 4 pi |S1|^2 / k^2   (phi = 90 deg plane).
"""
import math

import numpy as np
from scipy.special import spherical_jn, spherical_yn

from .quadrature import WEIGHTS, triangle_points


def _nmax(x):
    return int(math.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0))


def mie_coefficients(x):
    n = np.arange(1, _nmax(x) + 1)
    j = spherical_jn(n, x)
    y = spherical_yn(n, x)
    jd = spherical_jn(n, x, derivative=True)
    yd = spherical_yn(n, x, derivative=True)
    h = j + 1j * y
    hd = jd + 1j * yd
    a = (j + x * jd) / (h + x * hd)
    b = j / h
    return n, a, b


def _pi_tau(nmax, mu):
    mu = np.atleast_1d(mu)
    pi = np.zeros((nmax + 1, len(mu)))
    tau = np.zeros((nmax + 1, len(mu)))
    pi[1] = 1.0
    for n in range(2, nmax + 1):
        pi[n] = (2 * n - 1) / (n - 1) * mu * pi[n - 1] - n / (n - 1) * pi[n - 2]
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def amplitudes(x, theta):
    n, a, b = mie_coefficients(x)
    pi, tau = _pi_tau(len(n), np.cos(theta))
    f = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(f * (a[:, None] * pi + b[:, None] * tau), 0)
    S2 = np.sum(f * (a[:, None] * tau + b[:, None] * pi), 0)
    return S1, S2


def bistatic_rcs(k, radius, theta):
    """(sigma_E, sigma_H) in the E and H planes at polar angles theta (from +z)."""
    S1, S2 = amplitudes(k * radius, np.asarray(theta, np.float64))
    return 4 * math.pi * np.abs(S2) ** 2 / k ** 2, 4 * math.pi * np.abs(S1) ** 2 / k ** 2


def scattering_cross_section(k, radius):
    n, a, b = mie_coefficients(k * radius)
    return 2 * math.pi / k ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))


def extinction_cross_section(k, radius):
    S1, S2 = amplitudes(k * radius, np.array([0.0]))
    return 4 * math.pi / k ** 2 * S1[0].real


def far_field(vertices, triangles, rwg, j, k, eta, rhat):
    """Far-field pattern F(rhat) with E_s ~ F exp(-i k r)/r (time convention exp(+i w t)):
    F = -i eta k/(4 pi) (I - rhat rhat) N,  N = sum_n j_n int phi_n(r') exp(i k rhat.r') dr'."""
    rhat = np.atleast_2d(rhat)
    q = triangle_points(vertices, triangles)
    tris = np.asarray(triangles)
    out = np.zeros((len(rhat), 3), np.complex128)
    for i, u in enumerate(rhat):
        ph = np.exp(1j * k * np.einsum("tpx,x->tp", q, u))
        N = np.zeros(3, np.complex128)
        for m in range(rwg["n"]):
            for side in range(2):
                t = rwg["tri"][m, side]
                c = rwg["free"][m, side]
                s = 1.0 if side == 0 else -1.0
                f = s * rwg["length"][m] / 2.0 * (q[t] - vertices[tris[t, c]])
                N += j[m] * np.sum((WEIGHTS * ph[t])[:, None] * f, 0)
        out[i] = -1j * eta * k / (4 * math.pi) * (N - u * np.dot(u, N))
    return out


def rcs_from_currents(vertices, triangles, rwg, j, k, eta, rhat):
    """sigma(rhat) = 4 pi |F(rhat)|^2 (unit incident amplitude)."""
    F = far_field(vertices, triangles, rwg, j, k, eta, rhat)
    return 4 * math.pi * np.real(np.einsum("ix,ix->i", F.conj(), F))
