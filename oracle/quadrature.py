"""Quadrature rules of the FP64 oracle (test infrastructure only).

Rules (reading R5 of the method's unstated quadrature; Appendix A, Eqs. "2nd
term", "3rd term", "rhs term" only name weights beta_i, gamma_z):
  * time: N+1-point Gauss-Legendre on [0, dt];
  * volume: (N+1)^3-point collapsed (Stroud) Gauss-Jacobi rule on the unit
    tetrahedron, exact to total degree 2N+1;
  * face: (N+1)^2-point collapsed Gauss-Jacobi rule on the unit triangle.
1-D Gauss-Jacobi nodes come from the Golub-Welsch eigenvalue method (the
symmetric Jacobi matrix of the three-term recurrence, diagonalised by
numpy.linalg.eigh).
"""
from __future__ import annotations

import math

import numpy as np


def gauss_jacobi(n: int, alpha: float, beta: float = 0.0):
    """n-point Gauss rule for int_{-1}^{1} (1-x)^alpha (1+x)^beta f(x) dx."""
    a, b = float(alpha), float(beta)
    k = np.arange(n, dtype=np.float64)
    s = 2.0 * k + a + b
    diag = np.empty(n)
    with np.errstate(invalid="ignore", divide="ignore"):
        diag[:] = (b * b - a * a) / (s * (s + 2.0))
    if n > 0 and abs(a + b) < 1e-14:
        diag[0] = (b - a) / (a + b + 2.0)
    kk = np.arange(1, n, dtype=np.float64)
    ss = 2.0 * kk + a + b
    off = np.sqrt(4.0 * kk * (kk + a) * (kk + b) * (kk + a + b)
                  / (ss * ss * (ss + 1.0) * (ss - 1.0)))
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(T)
    mu0 = 2.0 ** (a + b + 1.0) * math.gamma(a + 1.0) * math.gamma(b + 1.0) / math.gamma(a + b + 2.0)
    w = mu0 * V[0, :] ** 2
    return x, w


def gauss_legendre_01(n: int):
    """n-point Gauss-Legendre rule on [0,1]."""
    x, w = gauss_jacobi(n, 0.0, 0.0)
    return 0.5 * (x + 1.0), 0.5 * w


def tet_rule(n: int):
    """Collapsed rule with n points per direction on the unit tetrahedron
    {xi,eta,zeta >= 0, xi+eta+zeta <= 1}.  Returns points [n^3,3] and weights
    summing to the volume 1/6."""
    a, wa = gauss_jacobi(n, 0.0)
    b, wb = gauss_jacobi(n, 1.0)
    c, wc = gauss_jacobi(n, 2.0)
    A, B, C = np.meshgrid(a, b, c, indexing="ij")
    WA, WB, WC = np.meshgrid(wa, wb, wc, indexing="ij")
    xi = (1 + A) * (1 - B) * (1 - C) / 8.0
    eta = (1 + B) * (1 - C) / 4.0
    zeta = (1 + C) / 2.0
    pts = np.stack([xi.ravel(), eta.ravel(), zeta.ravel()], axis=1)
    w = (WA * WB * WC).ravel() / 64.0
    return pts, w


def tri_rule(n: int):
    """Collapsed rule with n points per direction on the unit triangle
    {s,t >= 0, s+t <= 1}.  Returns points [n^2,2] and weights summing to 1
    (i.e. normalised by the triangle area 1/2)."""
    a, wa = gauss_jacobi(n, 0.0)
    b, wb = gauss_jacobi(n, 1.0)
    A, B = np.meshgrid(a, b, indexing="ij")
    WA, WB = np.meshgrid(wa, wb, indexing="ij")
    s = (1 + A) * (1 - B) / 4.0
    t = (1 + B) / 2.0
    pts = np.stack([s.ravel(), t.ravel()], axis=1)
    w = (WA * WB).ravel() / 8.0 * 2.0
    return pts, w
