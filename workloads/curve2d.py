"""Seeded charges on a curve in the plane, for the 2D model problem (Sec. 3).

The paper's source curve is shown only in a figure that is not available, so a
seeded smooth closed curve stands in: a circle of radius 1 whose radius is perturbed
by a few low Fourier modes, sampled at equal arc-length steps.  Geometry and random
numbers only.
"""
import numpy as np


def curve_points(n, seed=0, modes=6, amplitude=0.25):
    """n points (float64, [n][2]) at equal arc-length steps on a closed curve
    r(theta) = 1 + sum_k a_k cos(k theta + p_k), k = 2..modes+1, sum |a_k| <= amplitude."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, modes)
    a *= amplitude / np.abs(a).sum()
    ph = rng.uniform(0.0, 2.0 * np.pi, modes)
    k = np.arange(2, modes + 2)
    m = max(16 * n, 4096)  # fine polygon for the arc length
    th = np.linspace(0.0, 2.0 * np.pi, m + 1)
    r = 1.0 + (a[:, None] * np.cos(k[:, None] * th[None, :] + ph[:, None])).sum(0)
    xy = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    seg = np.linalg.norm(np.diff(xy, axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    t = (np.arange(n) + 0.5) * s[-1] / n
    return np.stack([np.interp(t, s, xy[:, 0]), np.interp(t, s, xy[:, 1])], 1)


def charges(n, seed=0):
    """n charges (float64), uniform in [-1, 1)."""
    return np.random.default_rng(seed + 7919).uniform(-1.0, 1.0, n)
