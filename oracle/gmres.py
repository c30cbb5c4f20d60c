"""Restarted GMRES(m) (Saad & Schultz 1986), the iterative solver named in Sec. 2.

Reading: x0 = 0; Arnoldi with modified Gram-Schmidt; Givens rotations on the
Hessenberg matrix; stop when the relative residual ||b - A x|| / ||b|| <= tol, using
the Givens estimate inside a cycle and the explicitly recomputed residual at each
restart.  Plain numpy, one right-hand side.
"""
import numpy as np


def gmres(apply_a, b, tol=1e-6, restart=50, maxiter=1000):
    """Returns (x, iterations, converged, history of relative residual estimates)."""
    b = np.asarray(b, np.complex128)
    n = len(b)
    x = np.zeros(n, np.complex128)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return x, 0, True, hist
    its = 0
    r = b.copy()
    beta = bnorm
    while True:
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            return x, its, True, hist
        if its >= maxiter:
            return x, its, False, hist
        m = restart
        V = np.zeros((m + 1, n), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m, np.complex128)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        V[0] = r / beta
        g[0] = beta
        j = 0
        while j < m and its < maxiter:
            w = apply_a(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = abs(a) / den if den else 1.0
            sn[j] = (a / abs(a)) * np.conj(c) / den if abs(a) else 1.0
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j += 1
            est = abs(g[j]) / bnorm
            if est <= tol:
                break
            hist.append(est)
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
        x = x + V[:j].T @ y
        r = b - apply_a(x)
        beta = np.linalg.norm(r)
