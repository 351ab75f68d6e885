"""Orthonormal Dubiner modal basis on the unit tetrahedron (oracle; test
infrastructure only).

The method expands each conservative variable in Dubiner's orthogonal
polynomials (Sec. 2.2, Eq. "modal dg space"); L = (N+1)(N+2)(N+3)/6 modes.
Reference element: vertices (0,0,0), (1,0,0), (0,1,0), (0,0,1) (reading R9).

phi_ijk = c_ijk * A_i * B_ij * C_ijk with
  A_i   = u^i P_i^{(0,0)}((2 xi - u)/u),            u = 1 - eta - zeta
  B_ij  = w^j P_j^{(2i+1,0)}((2 eta - w)/w),        w = 1 - zeta
  C_ijk = P_k^{(2i+2j+2,0)}(2 zeta - 1)
  c_ijk = sqrt((2i+1)(2i+2j+2)(2i+2j+2k+3))  (so that int phi^2 = 1)
The products y^n P_n(x/y) are evaluated by the scaled three-term recurrence,
which has no division and stays regular on edges and vertices.
Mode order: total degree i+j+k ascending, then (i,j,k) lexicographic.
"""
from __future__ import annotations

import numpy as np


def n_modes(N: int) -> int:
    return (N + 1) * (N + 2) * (N + 3) // 6


def mode_list(N: int):
    modes = []
    for d in range(N + 1):
        for i in range(d + 1):
            for j in range(d - i + 1):
                modes.append((i, j, d - i - j))
    return modes


def _scaled_jacobi(nmax, a, x, y):
    """Q_n(x,y) = y^n P_n^{(a,0)}(x/y) and its partials, n = 0..nmax."""
    b = 0.0
    Q = [np.ones_like(x)]
    Qx = [np.zeros_like(x)]
    Qy = [np.zeros_like(x)]
    if nmax >= 1:
        Q.append(0.5 * ((a + b + 2.0) * x + (a - b) * y))
        Qx.append(0.5 * (a + b + 2.0) * np.ones_like(x))
        Qy.append(0.5 * (a - b) * np.ones_like(x))
    for n in range(1, nmax):
        s = 2.0 * n + a + b
        d = 2.0 * (n + 1) * (n + a + b + 1) * s
        An = (s + 1) * (s + 2) * s / d
        Bn = (s + 1) * (a * a - b * b) / d
        Cn = 2.0 * (n + a) * (n + b) * (s + 2) / d
        lin = An * x + Bn * y
        Q.append(lin * Q[n] - Cn * y * y * Q[n - 1])
        Qx.append(An * Q[n] + lin * Qx[n] - Cn * y * y * Qx[n - 1])
        Qy.append(Bn * Q[n] + lin * Qy[n] - 2.0 * Cn * y * Q[n - 1] - Cn * y * y * Qy[n - 1])
    return Q, Qx, Qy


def eval_basis(N: int, pts: np.ndarray, grad: bool = False):
    """Values [P,L] (and gradients [P,L,3] w.r.t. (xi,eta,zeta)) at points [P,3]."""
    pts = np.asarray(pts, dtype=np.float64)
    xi, eta, zeta = pts[:, 0], pts[:, 1], pts[:, 2]
    u = 1.0 - eta - zeta
    w = 1.0 - zeta
    x1, y1 = 2.0 * xi - u, u
    x2, y2 = 2.0 * eta - w, w
    x3 = 2.0 * zeta - 1.0
    one = np.ones_like(xi)
    dx1, dy1 = np.array([2.0, 1.0, 1.0]), np.array([0.0, -1.0, -1.0])
    dx2, dy2 = np.array([0.0, 2.0, 1.0]), np.array([0.0, 0.0, -1.0])
    dx3 = np.array([0.0, 0.0, 2.0])

    QA, QAx, QAy = _scaled_jacobi(N, 0.0, x1, y1)
    modes = mode_list(N)
    L = len(modes)
    V = np.empty((pts.shape[0], L))
    G = np.empty((pts.shape[0], L, 3)) if grad else None
    cacheB, cacheC = {}, {}
    for m, (i, j, k) in enumerate(modes):
        if i not in cacheB:
            cacheB[i] = _scaled_jacobi(N, 2.0 * i + 1.0, x2, y2)
        QB, QBx, QBy = cacheB[i]
        key = 2 * i + 2 * j + 2
        if key not in cacheC:
            cacheC[key] = _scaled_jacobi(N, float(key), x3, one)
        QC, QCx, _ = cacheC[key]
        c = np.sqrt((2 * i + 1.0) * (2 * i + 2 * j + 2.0) * (2 * i + 2 * j + 2 * k + 3.0))
        A, B, C = QA[i], QB[j], QC[k]
        V[:, m] = c * A * B * C
        if grad:
            dA = QAx[i][:, None] * dx1 + QAy[i][:, None] * dy1
            dB = QBx[j][:, None] * dx2 + QBy[j][:, None] * dy2
            dC = QCx[k][:, None] * dx3
            G[:, m, :] = c * (dA * (B * C)[:, None] + dB * (A * C)[:, None] + dC * (A * B)[:, None])
    return (V, G) if grad else V
