"""Boundary-face fluxes of the oracle: absorbing and free surface (Appendix A,
"Free surface and absorbing boundary conditions"; test infrastructure only).

Both fluxes use the effective isotropic Jacobian B^{1,eff} of the face-aligned
frame (x' = outward normal n, y' = s, z' = t), Eqs. "matrix_Beff_1..3" under
readings T1/T2, and its eigen-decomposition B^{1,eff} = R Lambda R^{-1}
(Eq. "matrix-R", reading T3: the second printed speed is c_s).

  absorbing   (Eq. "absorbing-flux"):     F = T R Lambda^+ R^{-1} T^{-1} u^-
  free surface (Eqs. "q_b", "matrix-C",  u^b = T^{-1} u^- + sum_k omega_k r^k with
               "freeSurface-flux"):       omega solving sigma_nn = sigma_ns = sigma_nt = 0
                                          for the face-aligned stress C u^b,
                                          F = T B^{1,eff} u^b

Face-aligned state ordering: (eps_nn, eps_ss, eps_tt, eps_ns, eps_st, eps_tn,
v_n, v_s, v_t, alpha), the global ordering with x, y, z replaced by n, s, t.

Both fluxes are linear in u^- for given (lambda_eff, mu_eff, rho), so each is
returned as a 10 x 10 matrix acting on the global state.  The effective Lame
parameters are those of the cell mean of the element the face belongs to
(reading R16: the paper does not say where B^{d,eff} is evaluated on a
boundary; the cell mean is also where the predictor evaluates it).
"""
from __future__ import annotations

import numpy as np

from .rheology import jacobian_eff

# Voigt pairs of the strain entries, in state order
PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))


def face_frame(n):
    """An orthonormal frame (n, s, t) with n the given unit normal: s is the
    normalised part of the coordinate axis least aligned with n that is
    orthogonal to n, t = n x s.  The fluxes do not depend on this choice."""
    n = np.asarray(n, dtype=np.float64)
    k = int(np.argmin(np.abs(n)))
    a = np.zeros(3)
    a[k] = 1.0
    s = a - (a @ n) * n
    s /= np.linalg.norm(s)
    t = np.cross(n, s)
    return n, s, t


def rotation_T(n, s, t):
    """T of Eq. "matrix-T": maps a face-aligned state to global coordinates.
    With Q = [n s t] (columns), the strain tensor transforms as Q eps' Q^T
    (tensor shear entries, so an off-diagonal face entry enters twice), the
    velocity as Q v', and alpha is unchanged."""
    Q = np.stack([np.asarray(n, float), np.asarray(s, float), np.asarray(t, float)], axis=1)
    T = np.zeros((10, 10))
    for p, (i, j) in enumerate(PAIRS):
        for q, (a, b) in enumerate(PAIRS):
            T[p, q] = Q[i, a] * Q[j, b]
            if a != b:
                T[p, q] += Q[i, b] * Q[j, a]
    T[6:9, 6:9] = Q
    T[9, 9] = 1.0
    return T


def speeds(lam, mu, rho):
    """c_p^eff and c_s^eff of the effective isotropic medium (reading T3)."""
    return np.sqrt((lam + 2.0 * mu) / rho), np.sqrt(mu / rho)


def eigen_R(lam, mu, rho):
    """Right eigenvectors of B^{1,eff} (Eq. "matrix-R") and the eigenvalues
    Lambda = diag(-c_p, -c_s, -c_s, 0, 0, 0, c_s, c_s, c_p, 0)."""
    cp, cs = speeds(lam, mu, rho)
    k = lam / (lam + 2.0 * mu)
    R = np.zeros((10, 10))
    R[0, 0], R[6, 0] = 1.0, cp                 # -c_p: (eps_nn, v_n)
    R[3, 1], R[7, 1] = 0.5, cs                 # -c_s: (eps_ns, v_s)
    R[5, 2], R[8, 2] = 0.5, cs                 # -c_s: (eps_tn, v_t)
    R[0, 3], R[2, 3] = -k, 1.0                 # 0: eps_tt with the compensating eps_nn
    R[4, 4] = 1.0                              # 0: eps_st
    R[0, 5], R[1, 5] = -k, 1.0                 # 0: eps_ss with the compensating eps_nn
    R[5, 6], R[8, 6] = -0.5, cs                # +c_s
    R[3, 7], R[7, 7] = -0.5, cs                # +c_s
    R[0, 8], R[6, 8] = -1.0, cp                # +c_p
    R[9, 9] = 1.0                              # 0: alpha
    lam_diag = np.array([-cp, -cs, -cs, 0.0, 0.0, 0.0, cs, cs, cp, 0.0])
    return R, lam_diag


def hooke_C(lam, mu):
    """C of Eq. "matrix-C" under reading T3: isotropic Hooke law with the
    effective Lame parameters on the strain entries (tensor shear, so the shear
    rows carry 2 mu), identity on velocity and alpha."""
    C = np.zeros((10, 10))
    for p in range(3):
        for q in range(3):
            C[p, q] = lam
        C[p, p] += 2.0 * mu
    for p in range(3, 6):
        C[p, p] = 2.0 * mu
    for p in range(6, 10):
        C[p, p] = 1.0
    return C


def absorbing_matrix(n, lam, mu, rho):
    """10 x 10 matrix of Eq. "absorbing-flux": T R Lambda^+ R^{-1} T^{-1}."""
    T = rotation_T(*face_frame(n))
    R, lam_diag = eigen_R(lam, mu, rho)
    lam_plus = np.diag(np.maximum(lam_diag, 0.0))
    return T @ R @ lam_plus @ np.linalg.inv(R) @ np.linalg.inv(T)


def _free_surface_parts(n, lam, mu, rho):
    """T and the face-aligned map u^n -> u^b of Eq. "q_b": u^b = u^n +
    omega_1 r^1 + omega_2 r^2 + omega_3 r^3 (the columns of R with speeds
    -c_p, -c_s, -c_s), omega from sigma_nn = sigma_ns = sigma_nt = 0 of the
    face-aligned stress C u^b (Eq. "matrix-C").  omega is linear in u^n, so
    u^b = (I + R_3 W) u^n with W the 3 x 10 solution operator."""
    T = rotation_T(*face_frame(n))
    R, _ = eigen_R(lam, mu, rho)
    C = hooke_C(lam, mu)
    rows = [0, 3, 5]                           # sigma_nn, sigma_ns, sigma_tn
    R3 = R[:, 0:3]
    A = (C @ R3)[rows, :]                      # d sigma_rows / d omega
    W = -np.linalg.solve(A, C[rows, :])        # omega = W u^n
    return T, np.eye(10) + R3 @ W


def free_surface_state(n, lam, mu, rho):
    """10 x 10 map from the own trace u^- to the boundary state u^b, both in
    global coordinates: T (I + R_3 W) T^{-1}."""
    T, Ub = _free_surface_parts(n, lam, mu, rho)
    return T @ Ub @ np.linalg.inv(T)


def free_surface_matrix(n, lam, mu, rho):
    """10 x 10 matrix of Eq. "freeSurface-flux": F = T B^{1,eff} u^b with
    u^b = (I + R_3 W) T^{-1} u^-."""
    T, Ub = _free_surface_parts(n, lam, mu, rho)
    B1 = jacobian_eff(np.array(lam), np.array(mu), np.array(rho))[0]
    return T @ B1 @ Ub @ np.linalg.inv(T)


def boundary_matrix(bc, n, lam, mu, rho):
    """Flux matrix of a boundary face: bc = 1 free surface, 2 absorbing."""
    if bc == 1:
        return free_surface_matrix(n, lam, mu, rho)
    if bc == 2:
        return absorbing_matrix(n, lam, mu, rho)
    raise ValueError(f"unknown boundary tag {bc}")
