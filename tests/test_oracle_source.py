"""Pins of the oracle's kinematic point source and receivers (Sec. 4.1: moment-tensor
point sources with a prescribed moment-rate time function; receivers sample the
velocity).  The reading: the source adds the strain rate -C0^{-1}:M w(t) delta(x - x_s),
C0 the undamaged isotropic stiffness, w the moment-rate time function (a Ricker
wavelet of unit peak, or a Gaussian of unit integral), integrated exactly over each
step through the antiderivative of w.

Each check fixes a part of that reading against mathematics, not against the
oracle's own formulas:
  * the antiderivative, by central differences against the rate it integrates
    and by its limits;
  * the compliance, by applying the fourth-order isotropic stiffness tensor,
    built from its index definition, to the oracle's source strain;
  * the whole step, by the exact balance of the total strain integral on a
    periodic mesh (the Rusanov fluxes and the mode-0 volume term move no
    strain in or out of the mesh), against a numerically quadratured w;
  * the delta, by its sifting property on polynomials of degree <= N;
  * the receivers, by the exact value of a projected polynomial.
A sign, a factor, a dropped 1/|J| or a wrong antiderivative fails one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import Oracle, stf_integral
from oracle.basis import eval_basis
from synthetic import periodic_cube_mesh, rock_material

SIDE = 4000.0
VOIGT = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))


def ricker_rate(tau, f0):
    a = (math.pi * f0 * tau) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


def gaussian_rate(tau, sig):
    return math.exp(-0.5 * (tau / sig) ** 2) / (sig * math.sqrt(2.0 * math.pi))


def rate(src, t):
    tau = t - src["t0"]
    return ricker_rate(tau, src["f0"]) if src["stf"] == 0 else gaussian_rate(tau, src["sigma"])


def to_tensor(v6):
    T = np.zeros((3, 3))
    for p, (i, j) in enumerate(VOIGT):
        T[i, j] = T[j, i] = v6[p]
    return T


def stiffness_tensor(lam, mu):
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)."""
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


@pytest.mark.parametrize("src", [
    {"stf": 0, "f0": 2.0, "t0": 0.45},
    {"stf": 0, "f0": 0.7, "t0": 1.3},
    {"stf": 1, "sigma": 0.25, "t0": 0.8},
    {"stf": 1, "f0": 0.6, "t0": 2.0},      # the C-ABI passes the Gaussian's sigma as f0_or_sigma
])
def test_stf_integral_is_the_antiderivative_of_the_rate(src):
    if "sigma" not in src and src["stf"] == 1:
        src = dict(src, sigma=src["f0"])
    width = 1.0 / src["f0"] if src["stf"] == 0 else src["sigma"]
    h = 1e-5 * width
    peak = 1.0 if src["stf"] == 0 else 1.0 / src["sigma"]             # size of the rate
    for t in src["t0"] + width * np.linspace(-4.0, 4.0, 41):
        fd = (stf_integral(src, t + h) - stf_integral(src, t - h)) / (2.0 * h)
        assert abs(fd - rate(src, t)) <= 1e-7 * peak
    far = 12.0 * width
    assert abs(stf_integral(src, src["t0"] - far)) < 1e-12           # zero at -infinity
    total = 0.0 if src["stf"] == 0 else 1.0                           # Ricker: zero net moment; Gaussian: unit
    assert abs(stf_integral(src, src["t0"] + far) - total) < 1e-12


def _oracle(n, N, seed, material=None, cd=0.0):
    mesh = periodic_cube_mesh(n, SIDE, jitter=0.1, seed=seed)
    mat = rock_material(mesh.n_elem, cd=cd) if material is None else material(mesh.n_elem)
    return Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat)


def test_source_strain_is_the_compliance_of_the_moment_tensor():
    rng = np.random.default_rng(11)

    def mixed(E):
        m = rock_material(E)
        m[:, 2] = rng.uniform(5e9, 40e9, size=E)                        # mu0
        m[:, 1] = m[:, 2] * rng.uniform(-0.5, 2.0, size=E)              # lambda0 > -2 mu0 / 3
        return m

    o = _oracle(3, 2, seed=3, material=mixed)
    for _ in range(6):
        m6 = rng.normal(size=6) * 1e15
        x = rng.uniform(0.1, 0.9, size=3) * SIDE
        o.set_sources([{"x": x, "m": m6, "stf": 0, "f0": 2.0, "t0": 0.4}])
        s = o.sources[0]
        rho, lam, mu = o.mat[s["e"], :3]
        sigma = np.einsum("ijkl,kl->ij", stiffness_tensor(lam, mu), to_tensor(s["eps"]))
        np.testing.assert_allclose(sigma, to_tensor(m6), rtol=1e-12, atol=1e-12 * np.abs(m6).max())
        # the located element contains x and phi is the basis at its reference point
        xi = np.linalg.solve(o.J[s["e"]], x - o.xyz[s["e"], 0])
        assert xi.min() >= -1e-12 and xi.sum() <= 1.0 + 1e-12
        np.testing.assert_allclose(s["phi"], eval_basis(2, xi[None, :])[0], rtol=0, atol=1e-12)


def _total_strain(o, Q):
    """int eps dV over the mesh: only mode 0 has a nonzero mean, and phi_0 = sqrt(6) on the
    reference tetrahedron of volume 1/6, so int_e eps = |J_e| Q_e0 / sqrt(6)."""
    return np.einsum("e,ep->p", o.detJ, Q[:, 0, :6]) / math.sqrt(6.0)


@pytest.mark.parametrize("N,stf", [(2, 0), (3, 1)])
def test_step_changes_total_strain_by_exactly_the_injected_moment(N, stf):
    """Periodic jittered cube, damage off, a rough random state and one interior source:
    one step changes int eps dV by -C0^{-1}:M [W(t+dt) - W(t)] and nothing else.  The step
    is far above the CFL limit on purpose: the balance holds for any dt, and a long step
    separates the exact antiderivative from a midpoint or end-point rule."""
    rng = np.random.default_rng(100 + N)
    o = _oracle(3, N, seed=7, cd=0.0)
    lam, mu = 32e9, 32e9
    Q = np.zeros((o.E, o.L, 10))
    Q[..., :9] = 1e-6 * rng.normal(size=(o.E, o.L, 9))
    Q[..., 6:9] *= 3000.0                                         # velocities at strain x c
    m6 = rng.normal(size=6) * 4e14
    src = {"x": np.array([0.37, 0.52, 0.61]) * SIDE, "m": m6, "stf": stf, "t0": 0.45}
    if stf == 0:
        src["f0"] = 2.0
    else:
        src["sigma"] = 0.2
    o.set_sources([src])
    t, dt = 0.3, 0.05
    Q1 = o.step(Q, dt, t)
    W, err = integrate.quad(lambda s: rate(src, s), t, t + dt, epsabs=0, epsrel=1e-13)
    C6 = np.array([[lam + 2 * mu, lam, lam, 0, 0, 0],
                   [lam, lam + 2 * mu, lam, 0, 0, 0],
                   [lam, lam, lam + 2 * mu, 0, 0, 0],
                   [0, 0, 0, 2 * mu, 0, 0],
                   [0, 0, 0, 0, 2 * mu, 0],
                   [0, 0, 0, 0, 0, 2 * mu]])
    expect = -np.linalg.solve(C6, m6) * W
    got = _total_strain(o, Q1) - _total_strain(o, Q)
    assert np.linalg.norm(got - expect) <= 1e-11 * np.linalg.norm(expect)
    # without the source the same step conserves the total strain to rounding
    o.set_sources([])
    got0 = _total_strain(o, o.step(Q, dt, t)) - _total_strain(o, Q)
    assert np.linalg.norm(got0) <= 1e-11 * np.linalg.norm(expect)


def test_source_is_a_delta_on_polynomials_of_degree_N():
    """From rest, one step of a source alone adds the modal coefficients of
    -C0^{-1}:M [W(t+dt)-W(t)] delta(x - x_s).  For any polynomial g of degree <= N,
    int g * (that field) dV must equal g(x_s) times the injected strain."""
    N = 3
    o = _oracle(3, N, seed=5, cd=0.0)
    rng = np.random.default_rng(9)
    x_s = np.array([0.21, 0.66, 0.48]) * SIDE
    m6 = rng.normal(size=6) * 1e15
    src = {"x": x_s, "m": m6, "stf": 0, "f0": 2.0, "t0": 0.45}
    o.set_sources([src])
    dQ = o.step(np.zeros((o.E, o.L, 10)), 0.01, 0.4)
    inj = -o.sources[0]["eps"] * (stf_integral(src, 0.41) - stf_integral(src, 0.4))
    for _ in range(4):
        c = rng.normal(size=(4, 4, 4))
        deg = np.add.outer(np.add.outer(np.arange(4), np.arange(4)), np.arange(4))
        c[deg > N] = 0.0

        def g(x):
            y = x / SIDE
            return np.einsum("ijk,...i,...j,...k->...", c, *(np.stack([y[..., d] ** p for p in range(4)], -1)
                                                               for d in range(3)))
        G = o.project(lambda x: np.repeat(g(x)[..., None], 10, axis=-1))[..., 0]   # [E, L]
        lhs = np.einsum("e,el,elp->p", o.detJ, G, dQ[..., :6])
        np.testing.assert_allclose(lhs, g(x_s) * inj, rtol=1e-11, atol=1e-13 * np.abs(inj).max())
    assert np.all(dQ[..., 6:] == 0.0)


def test_receivers_read_the_velocity_at_their_point():
    N = 2
    o = _oracle(3, N, seed=2, cd=0.0)
    rng = np.random.default_rng(4)
    A = rng.normal(size=(3, 3))
    b = rng.normal(size=3)

    def field(x):
        u = np.zeros(x.shape[:-1] + (10,))
        y = x / SIDE
        u[..., 6:9] = (y @ A.T + b) * (1.0 + y[..., :1])    # degree 2 per component
        return u
    Q = o.project(field)
    pts = rng.uniform(0.05, 0.95, size=(7, 3)) * SIDE
    o.set_receivers(pts)
    np.testing.assert_allclose(o.sample_receivers(Q), field(pts)[:, 6:9], rtol=1e-11, atol=1e-12)
