"""Plane-wave excitation (paper Sec. 2, Eq. 2 and Eq. 3).

The two passages differ by a sign (Eq. 2 puts -int e^i.phi_m on the right of Z j, the
definition of e^i_m in Eq. 3 combined with [Z][j] = -[e^i] gives +).  Reading used:
the physical null-field condition of Eq. 2,  b_m = -int E^i(r).phi_m(r) dr,
with E^i = p exp(-i k khat.r) (time convention exp(+i w t), matching g of Eq. 1).
7-point rule per triangle.
"""
import numpy as np

from .quadrature import WEIGHTS, triangle_points


def planewave_rhs(vertices, triangles, rwg, k, khat, pol):
    """b [nrhs, N] for directions khat [nrhs,3] and complex polarisations pol [nrhs,3]."""
    khat = np.atleast_2d(khat)
    pol = np.atleast_2d(pol).astype(np.complex128)
    q = triangle_points(vertices, triangles)  # [nt,7,3]
    tris = np.asarray(triangles)
    b = np.zeros((len(khat), rwg["n"]), np.complex128)
    for r in range(len(khat)):
        ph = np.exp(-1j * k * np.einsum("tpx,x->tp", q, khat[r]))  # [nt,7]
        for m in range(rwg["n"]):
            acc = 0.0 + 0.0j
            for side in range(2):
                t = rwg["tri"][m, side]
                c = rwg["free"][m, side]
                s = 1.0 if side == 0 else -1.0
                v = vertices[tris[t, c]]
                # phi_m = s l/(2A) (r - v); integral = A sum_p w_p (...)
                f = s * rwg["length"][m] / 2.0 * (q[t] - v)  # [7,3] (area cancels)
                acc += np.sum(WEIGHTS * ph[t] * (f @ pol[r]))
            b[r, m] = -acc
    return b
