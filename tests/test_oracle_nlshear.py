"""Pins of the nonlinear shear law (reading R19: the isotropic law whose plane
shear response is the relation of Eq. "1d Riemann eqs") and of the exact 1-D
Riemann solution of Sec. 3.1: the stress as the strain gradient of an energy,
the plane-shear reduction, the secant moduli, the linear limit, the
Rankine-Hugoniot and Lax conditions at shocks, the Riemann invariant across a
rarefaction, the closed-form integral against quadrature, and the oracle's DG
solution against the exact one."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import Oracle
from oracle.rheology import (damage_rate, effective_lame_law, energy, invariants, stress,
                             strain_tensor)
from oracle.riemann import ShearRiemann
from synthetic import workload_riemann

MAT = np.array([1.0, 1.0, 1.0, 10.0, 0.0, 0.0])     # rho, lambda0, mu0, beta


def _states(n, scale, seed):
    rng = np.random.default_rng(seed)
    u = np.zeros((n, 10))
    u[:, :6] = rng.uniform(-scale, scale, size=(n, 6))
    u[:, 6:9] = rng.normal(size=(n, 3))
    u[:, 9] = rng.uniform(0, 0.5, size=n)
    return u


def test_stress_is_energy_gradient():
    u = _states(50, 0.02, 1)
    mat = np.broadcast_to(MAT, (50, 6))
    sig = stress(u, mat, "nlshear")
    h = 1e-7
    for p, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))):
        up, um = u.copy(), u.copy()
        up[:, p] += h
        um[:, p] -= h
        dW = (energy(up, mat, "nlshear") - energy(um, mat, "nlshear")) / (2 * h)
        # an off-diagonal strain entry appears twice in eps_ij eps_ij: dW/d eps_p = 2 sigma_ij
        expect = sig[:, i, j] * (1.0 if i == j else 2.0)
        assert np.allclose(dW, expect, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("e", [0.0, 0.004, 0.01, 0.02, 0.045])
def test_plane_shear_reduction(e):
    u = np.zeros((1, 10))
    u[0, 3] = e
    u[0, 9] = 0.3                                         # alpha takes no part
    sig = stress(u, MAT[None], "nlshear")[0]
    mu, beta = MAT[2], MAT[3]
    assert sig[0, 1] == pytest.approx(2 * mu * (1 - beta * e) * e, rel=1e-14, abs=1e-18)
    assert sig[1, 0] == sig[0, 1]
    others = sig.copy()
    others[0, 1] = others[1, 0] = 0.0
    assert np.all(others == 0.0)


def test_secant_moduli_and_linear_limit():
    u = _states(40, 0.03, 2)
    mat = np.broadcast_to(MAT, (40, 6))
    lam, mu = effective_lame_law(u, mat, "nlshear")
    e = strain_tensor(u)
    I1 = e[:, 0, 0] + e[:, 1, 1] + e[:, 2, 2]
    rebuilt = (lam * I1)[:, None, None] * np.eye(3) + (2 * mu)[:, None, None] * e
    assert np.allclose(stress(u, mat, "nlshear"), rebuilt, rtol=1e-13, atol=1e-16)
    lin = mat.copy()
    lin[:, 3] = 0.0
    ref = (lin[:, 1] * I1)[:, None, None] * np.eye(3) + (2 * lin[:, 2])[:, None, None] * e
    assert np.allclose(stress(u, lin, "nlshear"), ref, rtol=1e-14, atol=1e-18)
    assert np.all(damage_rate(u, mat, "nlshear") == 0.0)
    _, I2, _, _ = invariants(u)
    assert np.allclose(mu, MAT[2] * (1 - MAT[3] * np.sqrt(I2 / 2)))


def test_riemann_linear_limit():
    """beta = 0: two linear waves of speed c = sqrt(mu / rho); the middle state
    eps_m = (eps_L + eps_R)/2 + (v_R - v_L)/(4c) follows from v - 2c eps
    constant across the left wave and v + 2c eps across the right one."""
    r = ShearRiemann((0.01, -0.2), (0.03, 0.5), rho=2.0, mu=3.0, beta=0.0)
    c = math.sqrt(3.0 / 2.0)
    em = 0.02 + 0.7 / (4 * c)
    assert r.em == pytest.approx(em, rel=1e-12)
    assert r.vm == pytest.approx(-0.2 + 2 * c * (em - 0.01), rel=1e-12)


@pytest.mark.parametrize("left,right", [((0.01, 0.0), (0.02, 0.0)),        # rarefaction | shock
                                        ((0.02, 0.0), (0.01, 0.0)),        # shock | rarefaction
                                        ((0.01, -0.05), (0.02, -0.1)),     # shock | shock
                                        ((0.02, -0.1), (0.01, -0.05))])    # rarefaction | rarefaction
def test_riemann_wave_conditions(left, right):
    r = ShearRiemann(left, right)
    (a1, b1), (a2, b2) = r.speeds()
    assert a1 <= b1 < 0 < a2 <= b2
    for fam, (ea, va, eb, vb, kind) in ((1, (r.eL, r.vL, r.em, r.vm, r.kind1)),
                                        (2, (r.em, r.vm, r.eR, r.vR, r.kind2))):
        lam = (lambda e: -r.c(e)) if fam == 1 else r.c
        if kind == "shock":
            s = a1 if fam == 1 else a2
            # Rankine-Hugoniot for eps_t - v_x/2 = 0, v_t - sigma_x/rho = 0
            assert s * (eb - ea) == pytest.approx(-(vb - va) / 2, rel=1e-9, abs=1e-14)
            assert s * (vb - va) == pytest.approx(-(r.sigma(eb) - r.sigma(ea)) / r.rho, rel=1e-9, abs=1e-14)
            assert lam(ea) > s > lam(eb)                      # Lax: characteristics run into the shock
        else:
            assert lam(ea) <= lam(eb)                         # speeds spread across the fan
    # Riemann invariants inside the fans and continuity at their edges
    t = 0.7
    for fam, (lo, hi) in ((1, (a1, b1)), (2, (a2, b2))):
        if hi - lo < 1e-12:
            continue
        z = np.linspace(lo, hi, 9)[1:-1]
        eps, v = r.sample(z * t, t)
        inv = v - np.array([r.G(r.eL, e) for e in eps]) if fam == 1 else v + np.array([r.G(r.eR, e) for e in eps])
        ref = r.vL if fam == 1 else r.vR
        assert np.allclose(inv, ref, rtol=0, atol=1e-13)
        e_in, v_in = r.sample(np.array([lo + 1e-9, hi - 1e-9]) * t, t)
        e_out, v_out = r.sample(np.array([lo - 1e-9, hi + 1e-9]) * t, t)
        assert np.allclose(e_in, e_out, atol=1e-6) and np.allclose(v_in, v_out, atol=1e-6)


def test_riemann_integral_against_quadrature():
    r = ShearRiemann((0.01, 0.0), (0.02, 0.0))
    for a, b in ((0.0, 0.02), (0.013, 0.031), (0.04, 0.001)):
        num, _ = quad(lambda s: 2 * r.c(s), a, b, epsabs=1e-14, epsrel=1e-13)
        assert r.G(a, b) == pytest.approx(num, rel=1e-11)


def test_riemann_paper_states_are_not_hyperbolic():
    """Reading R19: under sigma_xy = 2 mu (1 - beta eps) eps with beta = 10 the
    paper's initial states eps = 0.1 and 0.2 have sigma' = 2 mu (1 - 2 beta eps)
    < 0, so the system is not hyperbolic there."""
    with pytest.raises(ValueError):
        ShearRiemann((0.1, -0.5), (0.2, -1.0))


def _ic(left, right):
    def f(x):
        u = np.zeros(x.shape[:-1] + (10,))
        neg = x[..., 0] < 0
        u[..., 3] = np.where(neg, left[0], right[0])
        u[..., 7] = np.where(neg, left[1], right[1])
        return u
    return f


def window_errors(o, Q, w, t):
    """L1 errors per unit length of eps_xy and v_y in |x| < eval_half_width,
    over the cross-section, by the rule tet_rule(N + 2)."""
    from oracle import tet_rule
    pts, wq = tet_rule(o.N + 2)
    u = o.evaluate(Q, pts)
    x = o.xyz[:, 0, None, :] + np.einsum("edk,qk->eqd", o.J, pts, optimize=True)
    r = ShearRiemann(w["left"], w["right"], *w["material"][0, [0, 2, 3]])
    eps, v = r.sample(x[..., 0], t)
    inside = np.abs(x[..., 0]) < w["eval_half_width"]
    dv = o.detJ[:, None] * wq[None, :] * inside
    area = (3 * w["h"]) ** 2
    return (float(np.sum(dv * np.abs(u[..., 3] - eps))) / area,
            float(np.sum(dv * np.abs(u[..., 7] - v))) / area)


def test_oracle_dg_tracks_the_exact_solution():
    """The oracle's DG solution (N = 1, 16 cells) stays close to the exact wave
    fan: the L1 error over the window is a small fraction of the strain jump
    times the window length, and the step between the fans is resolved."""
    w = workload_riemann(16, order=1)
    m = w["mesh"]
    o = Oracle(m.elem_xyz, m.elem_vid, 1, w["material"], law="nlshear")
    Q0 = o.project(_ic(w["left"], w["right"]))
    n = int(np.ceil(w["t_end"] / o.cfl_dt()))
    Q = o.run(Q0, w["t_end"] / n, n)
    err_e, err_v = window_errors(o, Q, w, w["t_end"])
    jump = abs(w["right"][0] - w["left"][0])
    length = 2 * w["eval_half_width"]
    assert err_e < 0.1 * jump * length, err_e
    assert err_v < 0.1 * jump * length, err_v
