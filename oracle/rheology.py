"""Pointwise CDM (Lyakhovsky continuum damage) law of the oracle (test
infrastructure only).  All arrays carry the 10 conservative variables in the
last axis: (eps_xx, eps_yy, eps_zz, eps_xy, eps_yz, eps_zx, v_x, v_y, v_z, alpha)
(Eq. "nonlinear hyper pdes"), tensor shear strains.

Material arrays `mat` have last axis (rho, lambda0, mu0, gamma_r, xi0, C_d) for
the CDM, (rho, lambda0, mu0, gamma_b, tau_b, unused) for the IVM
(Eq. "ivm-model", Murnaghan coefficients l0 = m0 = n0 = 0 as the paper sets
them) and (rho, lambda0, mu0, beta, unused, unused) for the nonlinear shear law
of the 1-D Riemann verification (Sec. 3.1, Eq. "1d Riemann eqs").  The
law-generic entry points take law = "cdm" (default), "ivm" or "nlshear".
"""
from __future__ import annotations

import numpy as np

I2_FLOOR = 1e-30   # reading R7: below this I2 counts as zero strain (xi = 0)

# (i, j) component -> index of the strain entry in u
SYM = np.array([[0, 3, 5],
                [3, 1, 4],
                [5, 4, 2]])


def strain_tensor(u):
    """3x3 strain tensor from u[..., 0:6]."""
    return u[..., SYM]


def invariants(u):
    """I1 = eps_kk, I2 = eps_ij eps_ij (sum over all 9 entries), sqrt(I2), xi
    (Sec. 2.1, text after Eq. "ivm-model" and Eq. "cdb-model"); xi = 0 where
    I2 is below the floor (reading R7)."""
    e = strain_tensor(u)
    I1 = e[..., 0, 0] + e[..., 1, 1] + e[..., 2, 2]
    I2 = np.einsum("...ij,...ij->...", e, e)
    zero = I2 <= I2_FLOOR
    s = np.where(zero, 0.0, np.sqrt(np.where(zero, 1.0, I2)))
    xi = np.where(zero, 0.0, I1 / np.where(zero, 1.0, s))
    return I1, I2, s, xi


def cdm_stress(u, mat):
    """Stress tensor [...,3,3] of Eq. "cdb-model":
    sigma = lambda0 I1 delta - alpha gamma_r sqrt(I2) delta
            + [2 (mu0 + alpha xi0 gamma_r) - alpha gamma_r xi] eps."""
    lam0, mu0, gr, xi0 = mat[..., 1], mat[..., 2], mat[..., 3], mat[..., 4]
    alpha = u[..., 9]
    e = strain_tensor(u)
    I1, I2, s, xi = invariants(u)
    iso = lam0 * I1 - alpha * gr * s
    shear = 2.0 * (mu0 + alpha * xi0 * gr) - alpha * gr * xi
    return iso[..., None, None] * np.eye(3) + shear[..., None, None] * e


def cdm_damage_rate(u, mat):
    """r_alpha of Eq. "cdb-model": C_d gamma_r I2 (xi - xi0) where xi > xi0,
    else 0.  Written as C_d gamma_r max(0, I1 sqrt(I2) - xi0 I2), which equals
    it for I2 > 0 and needs no division (reading R7)."""
    gr, xi0, cd = mat[..., 3], mat[..., 4], mat[..., 5]
    I1, I2, s, xi = invariants(u)
    return cd * gr * np.maximum(0.0, I1 * s - xi0 * I2)


def cdm_energy(u, mat):
    """Elastic energy density W with sigma = dW/d eps (derived, not printed):
    W = lambda0/2 I1^2 + (mu0 + alpha xi0 gamma_r) I2 - alpha gamma_r I1 sqrt(I2)."""
    lam0, mu0, gr, xi0 = mat[..., 1], mat[..., 2], mat[..., 3], mat[..., 4]
    alpha = u[..., 9]
    I1, I2, s, xi = invariants(u)
    return 0.5 * lam0 * I1 * I1 + (mu0 + alpha * xi0 * gr) * I2 - alpha * gr * I1 * s


def effective_lame(u, mat):
    """Effective Lame parameters of the CDM (Eq. "effective-cdb") under readings
    R2/R7: lambda_eff = lambda0 - alpha gamma_r (I1/3)/sqrt(I2)
                      = lambda0 - alpha gamma_r xi / 3,
    mu_eff = mu0 + alpha xi0 gamma_r - alpha gamma_r xi / 2 (sign of the xi0 term
    taken from the stress law of Eq. "cdb-model")."""
    lam0, mu0, gr, xi0 = mat[..., 1], mat[..., 2], mat[..., 3], mat[..., 4]
    alpha = u[..., 9]
    _, _, _, xi = invariants(u)
    lam = lam0 - alpha * gr * xi / 3.0
    mu = mu0 + alpha * xi0 * gr - 0.5 * alpha * gr * xi
    return lam, mu


def ivm_stress(u, mat):
    """Stress tensor [...,3,3] of Eq. "ivm-model" with l0 = m0 = n0 = 0:
    sigma = (1 - alpha) (lambda0 I1 delta + 2 mu0 eps)."""
    lam0, mu0 = mat[..., 1], mat[..., 2]
    alpha = u[..., 9]
    e = strain_tensor(u)
    I1 = e[..., 0, 0] + e[..., 1, 1] + e[..., 2, 2]
    iso = (1.0 - alpha) * lam0 * I1
    sh = (1.0 - alpha) * 2.0 * mu0
    return iso[..., None, None] * np.eye(3) + sh[..., None, None] * e


def ivm_damage_rate(u, mat):
    """r_alpha of Eq. "ivm-model" with W^mur = 0:
    (lambda0 I1^2 / 2 + mu0 I2 - phi(alpha)) / (gamma_b tau_b),
    phi(alpha) = gamma_b (alpha / (1 - alpha))^2."""
    lam0, mu0, gb, tb = mat[..., 1], mat[..., 2], mat[..., 3], mat[..., 4]
    alpha = u[..., 9]
    I1, I2, _, _ = invariants(u)
    s = alpha / (1.0 - alpha)
    return (0.5 * lam0 * I1 * I1 + mu0 * I2 - gb * s * s) / (gb * tb)


def ivm_energy(u, mat):
    """Elastic energy density of the IVM, W = (1 - alpha)(lambda0 I1^2 / 2 + mu0 I2),
    whose strain gradient is the stress of Eq. "ivm-model" (derived, not printed)."""
    lam0, mu0 = mat[..., 1], mat[..., 2]
    alpha = u[..., 9]
    I1, I2, _, _ = invariants(u)
    return (1.0 - alpha) * (0.5 * lam0 * I1 * I1 + mu0 * I2)


def ivm_effective_lame(u, mat):
    """Effective Lame parameters of the IVM (Eq. "effective-ivm"):
    lambda_eff = (1 - alpha) lambda0, mu_eff = (1 - alpha) mu0."""
    alpha = u[..., 9]
    return (1.0 - alpha) * mat[..., 1], (1.0 - alpha) * mat[..., 2]


def shear_magnitude(u):
    """gamma = sqrt(I2 / 2): for a plane shear state (eps_xy = eps_yx the only
    nonzero strains) I2 = 2 eps_xy^2 and gamma = |eps_xy|."""
    _, I2, _, _ = invariants(u)
    return np.sqrt(0.5 * I2)


def nlshear_stress(u, mat):
    """Stress of the nonlinear shear law (reading R19):
    sigma = lambda0 I1 delta + 2 mu0 (1 - beta gamma) eps,  gamma = sqrt(I2 / 2).
    It is the isotropic law whose plane shear response is the relation of
    Eq. "1d Riemann eqs", sigma_xy = 2 mu (1 - beta eps_xy) eps_xy for eps_xy >= 0;
    alpha plays no part."""
    lam0, mu0, beta = mat[..., 1], mat[..., 2], mat[..., 3]
    e = strain_tensor(u)
    I1 = e[..., 0, 0] + e[..., 1, 1] + e[..., 2, 2]
    g = shear_magnitude(u)
    sh = 2.0 * mu0 * (1.0 - beta * g)
    return (lam0 * I1)[..., None, None] * np.eye(3) + sh[..., None, None] * e


def nlshear_damage_rate(u, mat):
    """No damage variable evolves under the nonlinear shear law: r_alpha = 0."""
    return np.zeros(u.shape[:-1])


def nlshear_energy(u, mat):
    """Energy density whose strain gradient is nlshear_stress (derived, not
    printed): W = lambda0/2 I1^2 + mu0 I2 - (sqrt(2)/3) mu0 beta I2^(3/2), since
    d I2^(3/2) / d eps = 3 sqrt(I2) eps and sqrt(2) sqrt(I2) = 2 gamma."""
    lam0, mu0, beta = mat[..., 1], mat[..., 2], mat[..., 3]
    I1, I2, _, _ = invariants(u)
    return 0.5 * lam0 * I1 * I1 + mu0 * I2 - (np.sqrt(2.0) / 3.0) * mu0 * beta * I2 ** 1.5


def nlshear_effective_lame(u, mat):
    """Secant moduli at the state (reading R19): lambda_eff = lambda0,
    mu_eff = mu0 (1 - beta gamma), so that sigma(u) = lambda_eff I1 delta + 2 mu_eff eps."""
    return mat[..., 1] + 0.0 * u[..., 0], mat[..., 2] * (1.0 - mat[..., 3] * shear_magnitude(u))


_LAWS = {
    "cdm": (cdm_stress, cdm_damage_rate, cdm_energy, effective_lame),
    "ivm": (ivm_stress, ivm_damage_rate, ivm_energy, ivm_effective_lame),
    "nlshear": (nlshear_stress, nlshear_damage_rate, nlshear_energy, nlshear_effective_lame),
}


def stress(u, mat, law="cdm"):
    return _LAWS[law][0](u, mat)


def damage_rate(u, mat, law="cdm"):
    return _LAWS[law][1](u, mat)


def energy(u, mat, law="cdm"):
    return _LAWS[law][2](u, mat)


def effective_lame_law(u, mat, law="cdm"):
    return _LAWS[law][3](u, mat)


def flux(u, mat, law="cdm"):
    """Physical flux F^d_p [...,3(d),10(p)] of Eq. "nonlinear hyper pdes" under the
    rheology (follows from Eq. "nonlinear damage models"):
      F^d_{eps_ij} = -(v_i delta_jd + v_j delta_id)/2,
      F^d_{v_i}    = -sigma_id / rho,
      F^d_alpha    = 0."""
    rho = mat[..., 0]
    v = u[..., 6:9]
    sig = stress(u, mat, law)
    F = np.zeros(u.shape[:-1] + (3, 10))
    for p, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))):
        # -(v_i delta_jd + v_j delta_id)/2: the d = j entry gets -v_i/2, the d = i entry -v_j/2
        F[..., j, p] += -0.5 * v[..., i]
        F[..., i, p] += -0.5 * v[..., j]
    F[..., :, 6:9] = -np.swapaxes(sig, -1, -2) / rho[..., None, None]   # F[d, v_i] = -sigma_{i d}/rho
    return F


def jacobian_eff(lam, mu, rho):
    """Effective isotropic flux Jacobians B^{d,eff} [...,3,10,10] (Appendix A,
    Eqs. "matrix_Beff_1..3") rebuilt from the linear isotropic flux
    (reading T1: the printed B^2/B^3 rows have misplaced entries) with a zero
    alpha row (reading T2: F_alpha = 0, Lambda's last eigenvalue is 0)."""
    shape = np.shape(lam)
    B = np.zeros(shape + (3, 10, 10))
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))
    for d in range(3):
        for p, (i, j) in enumerate(pairs):
            # dF^d_{eps_ij}/d v_m = -(delta_im delta_jd + delta_jm delta_id)/2
            for m in range(3):
                val = -0.5 * ((i == m) * (j == d) + (j == m) * (i == d))
                if val != 0.0:
                    B[..., d, p, 6 + m] += val
        for i in range(3):
            row = 6 + i
            # sigma_id = lam I1 delta_id + 2 mu eps_id ; F = -sigma_id/rho
            if i == d:
                for q in range(3):
                    B[..., d, row, q] += -lam / rho
            q = SYM[i, d]
            B[..., d, row, q] += -2.0 * mu / rho
    return B
