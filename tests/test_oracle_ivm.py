"""Pins of the oracle's IVM law (Eq. "ivm-model" without Murnaghan terms, Eq.
"effective-ivm"): the stress is the strain gradient of the energy
W = (1 - alpha)(lambda0 I1^2 / 2 + mu0 I2), the effective Lame parameters are
its exact secant, the rate of hand-evaluated states, and uniform-strain damage
evolution through the whole solver against an accurate ODE solution (second
order in dt, the order of the source update of Eqs. "CKIter-ref-source" and
"time-integrated")."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import Oracle, ivm_damage_rate, ivm_effective_lame, ivm_energy, ivm_stress
from synthetic import periodic_cube_mesh

SYM = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))
LAM, MU, RHO, GB, TB = 32e9, 32e9, 2700.0, 1e4, 0.05


def _mat(shape=()):
    return np.broadcast_to(np.array([RHO, LAM, MU, GB, TB, 0.0]), shape + (6,)).copy()


def _random_states(rng, n):
    u = np.zeros((n, 10))
    u[:, :6] = rng.normal(size=(n, 6)) * 1e-4
    u[:, 6:9] = rng.normal(size=(n, 3))
    u[:, 9] = rng.uniform(0.0, 0.6, size=n)
    return u


def test_stress_is_the_energy_gradient():
    rng = np.random.default_rng(1)
    u = _random_states(rng, 20)
    mat = _mat((20,))
    sig = ivm_stress(u, mat)
    h = 1e-9
    for i, j in SYM:
        d = np.zeros(10)
        if i == j:
            d[SYM.index((i, j))] = 1.0
        else:
            d[SYM.index((i, j))] = 0.5           # eps_ij and eps_ji both move by h/2
        dW = (ivm_energy(u + h * d, mat) - ivm_energy(u - h * d, mat)) / (2 * h)
        np.testing.assert_allclose(dW, sig[:, i, j], rtol=1e-6, atol=1e-6 * np.abs(sig).max())


def test_effective_lame_is_the_exact_secant():
    """At any strain and damage, sigma = lambda_eff I1 delta + 2 mu_eff eps."""
    rng = np.random.default_rng(2)
    u = _random_states(rng, 20)
    mat = _mat((20,))
    lam, mu = ivm_effective_lame(u, mat)
    e = u[:, [0, 3, 5, 3, 1, 4, 5, 4, 2]].reshape(-1, 3, 3)
    I1 = np.trace(e, axis1=1, axis2=2)
    ref = lam[:, None, None] * I1[:, None, None] * np.eye(3) + 2 * mu[:, None, None] * e
    np.testing.assert_allclose(ivm_stress(u, mat), ref, rtol=1e-12, atol=1e-20)
    np.testing.assert_allclose(lam, (1 - u[:, 9]) * LAM)


def test_rate_of_hand_evaluated_states():
    """Uniaxial strain e at alpha = 0: (lambda0/2 + mu0) e^2 / (gamma_b tau_b); pure shear
    eps_xy = g: 2 mu0 g^2 / (gamma_b tau_b); the rate vanishes where
    alpha / (1 - alpha) = sqrt(W / gamma_b)."""
    mat = _mat()
    e = 2e-4
    u = np.zeros(10)
    u[0] = e
    assert ivm_damage_rate(u, mat) == pytest.approx((0.5 * LAM + MU) * e * e / (GB * TB), rel=1e-14)
    g = 3e-4
    u = np.zeros(10)
    u[3] = g
    assert ivm_damage_rate(u, mat) == pytest.approx(2 * MU * g * g / (GB * TB), rel=1e-14)
    u = np.zeros(10)
    u[0] = e
    s = math.sqrt((0.5 * LAM + MU) * e * e / GB)
    u[9] = s / (1 + s)
    assert abs(ivm_damage_rate(u, mat)) <= 1e-12 * (0.5 * LAM + MU) * e * e / (GB * TB)


def _uniform_run(dt, T, N=2):
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=3)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, _mat((mesh.n_elem,)), law="ivm")
    eps = np.array([1e-4, -3e-5, 2e-5, 4e-5, 0.0, -1e-5])

    def const(x):
        u = np.zeros(x.shape[:-1] + (10,))
        u[..., :6] = eps
        return u
    Q = o.project(const)
    n = int(round(T / dt))
    for _ in range(n):
        Q = o.step(Q, dt)
    return o, Q, eps


def test_uniform_strain_damage_matches_the_ode():
    """Uniform strain, v = 0: strain and velocity stay exactly constant and the
    damage follows d alpha/dt = (W0 - gamma_b (alpha/(1-alpha))^2) / (gamma_b tau_b);
    the solver's alpha converges to the ODE solution at second order in dt."""
    T = 0.2
    ref = None
    errs = []
    for dt in (0.02, 0.01, 0.005):
        o, Q, eps = _uniform_run(dt, T)
        u = o.evaluate(Q, np.array([[0.2, 0.2, 0.2]]))[:, 0, :]
        assert np.abs(u[:, :6] - eps).max() <= 1e-10 * np.abs(eps).max()
        assert np.abs(u[:, 6:9]).max() <= 1e-9          # (a wave of this strain moves at ~0.6 m/s)
        if ref is None:
            e = eps[[0, 3, 5, 3, 1, 4, 5, 4, 2]].reshape(3, 3)
            W0 = 0.5 * LAM * np.trace(e) ** 2 + MU * np.sum(e * e)
            sol = solve_ivp(lambda t, a: [(W0 - GB * (a[0] / (1 - a[0])) ** 2) / (GB * TB)], (0, T), [0.0],
                            rtol=1e-12, atol=1e-14)
            ref = sol.y[0, -1]
            assert ref > 0.05
        errs.append(np.abs(u[:, 9] - ref).max())
    assert errs[-1] < 1e-3 * ref
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
