"""Triangle geometry and the 7-point degree-5 triangle rule.

The rule is Radon's 7-point formula (Stroud T2:5-1, tabulated by Dunavant 1985):
the centroid with weight 9/40 and two orbits of three points with barycentric
coordinates (a, b, b), a = (9 -+ 2 sqrt 15)/21, b = (6 +- sqrt 15)/21 and weights
(155 +- sqrt 15)/1200.  Weights sum to one (integral = area * sum w f).
It integrates every polynomial of total degree <= 5 exactly.
"""
import math

import numpy as np

_S15 = math.sqrt(15.0)
_A1, _B1 = (9.0 - 2.0 * _S15) / 21.0, (6.0 + _S15) / 21.0
_A2, _B2 = (9.0 + 2.0 * _S15) / 21.0, (6.0 - _S15) / 21.0
_W1, _W2 = (155.0 + _S15) / 1200.0, (155.0 - _S15) / 1200.0

BARY = np.array([[1 / 3, 1 / 3, 1 / 3],
                 [_A1, _B1, _B1], [_B1, _A1, _B1], [_B1, _B1, _A1],
                 [_A2, _B2, _B2], [_B2, _A2, _B2], [_B2, _B2, _A2]])
WEIGHTS = np.array([9.0 / 40.0, _W1, _W1, _W1, _W2, _W2, _W2])


def triangle_points(vertices, triangles):
    """Quadrature nodes ``[nt, 7, 3]`` of every triangle, evaluated as
    (l0 v0 + l1 v1) + l2 v2 with separately rounded products and sums, so that a node
    lying exactly on a box face is reproducible."""
    v = np.asarray(vertices, np.float64)[np.asarray(triangles)]  # [nt, 3, 3]
    B = BARY[None, :, :, None]
    return (B[:, :, 0] * v[:, None, 0, :] + B[:, :, 1] * v[:, None, 1, :]) + B[:, :, 2] * v[:, None, 2, :]


def triangle_areas(vertices, triangles):
    v = vertices[triangles]
    return 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1)
