"""Pins of the oracle's pointwise CDM law (Eq. "cdb-model") against derived
closed forms: stress as the gradient of an energy, hand-derived damage rates
of special strain states, the uniaxial stress and the shear secant modulus."""
import math

import numpy as np
import pytest

from oracle import (cdm_damage_rate, cdm_energy, cdm_stress, effective_lame, flux,
                    invariants)

MAT = np.array([2700.0, 3.2e10, 3.2e10, 3.7e10, -0.8, 1e-4])   # rho lam0 mu0 gamma_r xi0 Cd


def _u(exx=0, eyy=0, ezz=0, exy=0, eyz=0, ezx=0, vx=0, vy=0, vz=0, alpha=0):
    return np.array([exx, eyy, ezz, exy, eyz, ezx, vx, vy, vz, alpha], dtype=float)


def test_stress_is_energy_gradient():
    """sigma_ij = dW/d eps_ij with W = lam0/2 I1^2 + (mu0+a xi0 g) I2 - a g I1 sqrt(I2):
    a dropped term, a wrong sign or a wrong factor in sigma breaks this."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        u = _u(*rng.normal(size=6) * 1e-3, alpha=rng.uniform(0, 0.6))
        sig = cdm_stress(u, MAT)
        h = 1e-9
        for p, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))):
            up, um = u.copy(), u.copy()
            up[p] += h
            um[p] -= h
            dW = (cdm_energy(up, MAT) - cdm_energy(um, MAT)) / (2 * h)
            # shear entries appear twice in I2 = eps_ij eps_ij: dW/d eps_xy = 2 sigma_xy
            want = sig[i, j] * (1.0 if i == j else 2.0)
            assert dW == pytest.approx(want, rel=1e-5, abs=1e-3)
    np.testing.assert_allclose(sig, sig.T)


def test_invariants_of_special_states():
    e = 1e-3
    I1, I2, s, xi = invariants(_u(exx=e))
    assert (I1, I2, xi) == pytest.approx((e, e * e, 1.0))
    I1, I2, s, xi = invariants(_u(exy=e))                 # tensor shear counted twice
    assert (I1, I2, xi) == pytest.approx((0.0, 2 * e * e, 0.0))
    I1, I2, s, xi = invariants(_u(exx=-e, eyy=-e, ezz=-e))
    assert xi == pytest.approx(-math.sqrt(3.0))
    I1, I2, s, xi = invariants(_u(exx=e, eyy=e, ezz=e))
    assert xi == pytest.approx(math.sqrt(3.0))
    assert invariants(_u())[3] == 0.0                     # reading R7


@pytest.mark.parametrize("case", ["uniaxial_ext", "uniaxial_comp", "pure_shear",
                                  "iso_comp", "iso_ext", "zero"])
def test_damage_rate_special_states(case):
    g, xi0, cd = MAT[3], MAT[4], MAT[5]
    e = 1e-3
    u, want = {
        # xi = 1 > xi0: rate Cd g e^2 (1 - xi0)
        "uniaxial_ext": (_u(exx=e), cd * g * e * e * (1 - xi0)),
        # xi = -1 < xi0 = -0.8: no growth
        "uniaxial_comp": (_u(exx=-e), 0.0),
        # xi = 0: rate Cd g (2 e^2)(0 - xi0)
        "pure_shear": (_u(exy=e), cd * g * 2 * e * e * (-xi0)),
        # xi = -sqrt3: none
        "iso_comp": (_u(exx=-e, eyy=-e, ezz=-e), 0.0),
        # xi = sqrt3: Cd g 3e^2 (sqrt3 - xi0)
        "iso_ext": (_u(exx=e, eyy=e, ezz=e), cd * g * 3 * e * e * (math.sqrt(3) - xi0)),
        "zero": (_u(), 0.0),
    }[case]
    assert cdm_damage_rate(u, MAT) == pytest.approx(want, rel=1e-12, abs=1e-30)


def test_damage_rate_tie_and_alpha_independence():
    # xi == xi0 exactly gives zero rate (Eq. "cdb-model", second case)
    mat = MAT.copy()
    mat[4] = 0.0
    assert cdm_damage_rate(_u(exy=1e-3), mat) == 0.0
    # the CDM rate does not depend on alpha
    assert cdm_damage_rate(_u(exx=1e-3, alpha=0.3), MAT) == cdm_damage_rate(_u(exx=1e-3), MAT)


@pytest.mark.parametrize("alpha", [0.0, 0.2, 0.5])
@pytest.mark.parametrize("e", [1e-3, -1e-3])
def test_uniaxial_stress_closed_form(alpha, e):
    lam0, mu0, g, xi0 = MAT[1], MAT[2], MAT[3], MAT[4]
    sig = cdm_stress(_u(exx=e, alpha=alpha), MAT)
    want_xx = lam0 * e - alpha * g * abs(e) + (2 * (mu0 + alpha * xi0 * g) - alpha * g * np.sign(e)) * e
    want_yy = lam0 * e - alpha * g * abs(e)
    assert sig[0, 0] == pytest.approx(want_xx, rel=1e-12)
    assert sig[1, 1] == pytest.approx(want_yy, rel=1e-12)
    assert abs(sig[0, 1]) < 1e-9


def test_effective_shear_modulus_is_stress_secant():
    """mu_eff (reading R2) is half the coefficient of eps_ij in sigma_ij (i != j),
    for any strain state: the printed '-alpha xi0 gamma_r' would fail."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        u = _u(*rng.normal(size=6) * 1e-3, alpha=rng.uniform(0, 0.5))
        sig = cdm_stress(u, MAT)
        lam, mu = effective_lame(u, MAT)
        assert sig[0, 1] / u[3] == pytest.approx(2 * mu, rel=1e-10)
        I1, I2, s, xi = invariants(u)
        assert lam == pytest.approx(MAT[1] - u[9] * MAT[3] * (I1 / 3.0) / s, rel=1e-12)


def test_flux_linear_elastic_limit():
    """Damage off: F^d is the flux of linear elasticity, F^d_p = B^d_pq u_q."""
    from oracle import jacobian_eff
    rng = np.random.default_rng(4)
    u = _u(*rng.normal(size=9) * 1e-3)
    F = flux(u, MAT)
    B = jacobian_eff(np.array(MAT[1]), np.array(MAT[2]), np.array(MAT[0]))
    np.testing.assert_allclose(F, np.einsum("dpq,q->dp", B, u), rtol=1e-12, atol=1e-20)
