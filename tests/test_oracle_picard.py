"""Pins of the oracle's discrete Picard predictor (reading R20, the extension
Sec. 5.1 proposes): for a linear flux the CK coefficients are its fixed point,
the iteration contracts on a nonlinear state, and the time fit reproduces the
Taylor coefficients of a polynomial exactly."""
import math

import numpy as np
import pytest

from oracle import Oracle, gauss_legendre_01, n_modes
from synthetic import periodic_cube_mesh


def _mesh():
    return periodic_cube_mesh(3, 1.0, jitter=0.1, seed=5)


def _state(E, N, seed, scale=1e-3):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(E, n_modes(N), 10)) * scale
    Q[..., 9] = 0.0
    return Q


@pytest.mark.parametrize("N", [1, 2, 3])
def test_linear_flux_fixed_point(N):
    """beta = 0: the shear law is linear, R(q(t)) is a polynomial of degree N in
    t, the fit is exact, and Picard iterations leave the CK coefficients as
    they are."""
    mesh = _mesh()
    mat = np.zeros((mesh.n_elem, 6))
    mat[:, :4] = (1.0, 1.0, 1.0, 0.0)
    Q0 = _state(mesh.n_elem, N, 1)
    ck = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, law="nlshear")
    pc = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, law="nlshear", picard_iterations=3)
    dt = 0.5 * ck.cfl_dt()
    Q1, Q2 = ck.run(Q0, dt, 2), pc.run(Q0, dt, 2)
    assert np.abs(Q1 - Q2).max() <= 1e-13 * np.abs(Q1).max()


def test_iteration_contracts_on_a_nonlinear_state():
    """beta = 10, strains of 1e-2: the predicted polynomials q(t_z) = sum_o
    t_z^o/o! D^o of successive iterates differ by a factor of about dt |dR/dq|
    less each time."""
    N = 3
    mesh = _mesh()
    mat = np.zeros((mesh.n_elem, 6))
    mat[:, :4] = (1.0, 1.0, 1.0, 10.0)
    Q0 = _state(mesh.n_elem, N, 2, scale=1e-2)
    Q0[:, 0, 3] = 0.02 / math.sqrt(6.0)                   # a shear strain of 0.02 at every cell mean
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, law="nlshear")
    dt = 0.5 * o.cfl_dt()
    rows = np.arange(mesh.n_elem)
    D, _, _ = o.predictor(Q0, rows)
    tz = o.qt_x * dt
    coef = np.array([[t ** i / math.factorial(i) for i in range(N + 1)] for t in tz])
    values = lambda D: np.einsum("zi,inlp->nzlp", coef, D[..., :9])
    prev = D
    diffs = []
    for _ in range(4):
        nxt = o.picard(prev, rows, dt, 1)
        diffs.append(np.abs(values(nxt) - values(prev)).max())
        prev = nxt
    assert diffs[0] > 0
    for a, b in zip(diffs, diffs[1:]):
        assert b < 0.5 * a, diffs


@pytest.mark.parametrize("N", [1, 2, 4])
def test_time_fit_reproduces_taylor_coefficients(N):
    """The fit through the N + 1 Gauss time nodes of a step recovers the Taylor
    coefficients of any polynomial of degree N in t (the step behind R^j)."""
    dt = 0.37
    tz = gauss_legendre_01(N + 1)[0] * dt
    V = np.array([[t ** j / math.factorial(j) for j in range(N + 1)] for t in tz])
    coef = np.random.default_rng(N).normal(size=N + 1)
    vals = np.array([sum(coef[j] * t ** j / math.factorial(j) for j in range(N + 1)) for t in tz])
    assert np.allclose(np.linalg.solve(V, vals), coef, rtol=1e-10, atol=1e-12)
