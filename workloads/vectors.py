"""Seeded random vectors (no method arithmetic)."""
import numpy as np


def random_coefficients(n, nrhs=1, seed=0):
    """Complex128 ``[nrhs, n]`` (one row per right-hand side), entries with
    independent standard normal real and imaginary parts."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))).astype(np.complex128)


def plane_wave_directions(nrhs, seed=180103589):
    """``nrhs`` incidence directions uniform on the unit sphere (normalised Gaussian
    triples) and one polarisation per direction: theta-hat of the direction (phi-hat
    at the poles).  Returns ``(khat [nrhs,3], pol [nrhs,3] complex128)``."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((nrhs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pol = np.empty((nrhs, 3))
    for i, (x, y, z) in enumerate(d):
        st = np.hypot(x, y)
        if st < 1e-12:
            pol[i] = (0.0, 1.0, 0.0)
        else:
            ct = z
            cp, sp = x / st, y / st
            pol[i] = (ct * cp, ct * sp, -st)
    return d, pol.astype(np.complex128)
