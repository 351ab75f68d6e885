"""Pins of the oracle's reference-element building blocks (quadrature, basis)
and of its effective Jacobians against what the paper prints."""
import math
import os

import numpy as np
import pytest

from oracle import (eval_basis, gauss_legendre_01, jacobian_eff, mode_list, n_modes,
                    tet_rule, tri_rule)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _monomial_tet(a, b, c):
    # int over the unit tetrahedron of xi^a eta^b zeta^c = a! b! c! / (a+b+c+3)!
    return math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)


def _monomial_tri(a, b):
    # int over the unit triangle of s^a t^b = a! b! / (a+b+2)!
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_tet_rule_exact_to_degree_2n_minus_1(n):
    pts, w = tet_rule(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            for c in range(2 * n - a - b):
                got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert got == pytest.approx(_monomial_tet(a, b, c), rel=1e-12, abs=1e-15)
    assert np.all(w > 0)
    # points inside the element
    assert np.all(pts >= 0) and np.all(pts.sum(axis=1) <= 1)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_tri_rule_exact_to_degree_2n_minus_1(n):
    pts, w = tri_rule(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            got = 0.5 * np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b)   # weights are area-normalised
            assert got == pytest.approx(_monomial_tri(a, b), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_legendre_matches_numpy(n):
    x, w = gauss_legendre_01(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(np.sort(x), np.sort(0.5 * (xr + 1)), atol=1e-14)
    np.testing.assert_allclose(np.sum(w), 1.0, atol=1e-14)
    for deg in range(2 * n):
        assert np.sum(w * x ** deg) == pytest.approx(1.0 / (deg + 1), rel=1e-13)


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4, 5])
def test_basis_orthonormal_and_graded(N):
    L = n_modes(N)
    assert L == (N + 1) * (N + 2) * (N + 3) // 6 == len(mode_list(N))
    pts, w = tet_rule(N + 2)
    V = eval_basis(N, pts)
    np.testing.assert_allclose(V.T @ (w[:, None] * V), np.eye(L), atol=1e-13)
    # modes are grouped by total degree
    degs = [sum(m) for m in mode_list(N)]
    assert degs == sorted(degs)
    # first mode is the constant sqrt(6)
    np.testing.assert_allclose(V[:, 0], math.sqrt(6.0), rtol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_basis_spans_polynomials_of_degree_N(N):
    """Every monomial of degree <= N is reproduced exactly by its projection,
    and degree-d modes are orthogonal to all monomials of degree < d."""
    pts, w = tet_rule(N + 2)
    V = eval_basis(N, pts)
    rng = np.random.default_rng(0)
    test_pts = rng.dirichlet(np.ones(4), size=20)[:, 1:]
    Vt = eval_basis(N, test_pts)
    degs = np.array([sum(m) for m in mode_list(N)])
    for a in range(N + 1):
        for b in range(N + 1 - a):
            for c in range(N + 1 - a - b):
                f = pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c
                coef = V.T @ (w * f)
                ft = test_pts[:, 0] ** a * test_pts[:, 1] ** b * test_pts[:, 2] ** c
                np.testing.assert_allclose(Vt @ coef, ft, atol=1e-12)
                # hierarchical: modes of degree > a+b+c have zero coefficient
                assert np.all(np.abs(coef[degs > a + b + c]) < 1e-12)


def test_basis_gradient_matches_finite_difference():
    N = 4
    rng = np.random.default_rng(1)
    pts = rng.dirichlet(np.ones(4), size=10)[:, 1:]
    _, G = eval_basis(N, pts, grad=True)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (eval_basis(N, pts + e) - eval_basis(N, pts - e)) / (2 * h)
        np.testing.assert_allclose(G[:, :, d], fd, atol=2e-7 * np.abs(G).max())


def _read_symbolic(name, env):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([eval(tok, {}, env) for tok in line.split(";")])
    return np.array(rows, dtype=float)


def test_B1_matches_printed_rows_and_eigendecomposition():
    lam, mu, rho = 3.1e10, 2.7e10, 2650.0
    cp, cs = math.sqrt((lam + 2 * mu) / rho), math.sqrt(mu / rho)
    env = {"lam": lam, "mu": mu, "rho": rho, "cp": cp, "cs": cs}
    B = jacobian_eff(np.array(lam), np.array(mu), np.array(rho))
    printed = _read_symbolic("matrix_B1_paper.txt", env)
    printed[9, 9] = 0.0          # reading T2: F_alpha = 0, eigenvalue 0 in Lambda
    np.testing.assert_allclose(B[0], printed, rtol=1e-14, atol=0)
    R = _read_symbolic("matrix_R_paper.txt", env)
    Lam = np.diag([-cp, -cs, -cs, 0, 0, 0, cs, cs, cp, 0])
    np.testing.assert_allclose(B[0] @ R, R @ Lam, rtol=1e-12, atol=1e-9 * cp)


def test_Bn_spectrum_is_isotropic():
    """For every unit direction n, sum_d n_d B^d has eigenvalues
    {+-cp, +-cs, +-cs, 0 x4} (hyperbolic, isotropic)."""
    lam, mu, rho = 2.0e10, 3.0e10, 2500.0
    cp, cs = math.sqrt((lam + 2 * mu) / rho), math.sqrt(mu / rho)
    B = jacobian_eff(np.array(lam), np.array(mu), np.array(rho))
    rng = np.random.default_rng(3)
    want = np.sort([-cp, -cs, -cs, 0, 0, 0, 0, cs, cs, cp])
    for _ in range(5):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        ev = np.linalg.eigvals(np.einsum("d,dpq->pq", n, B))
        np.testing.assert_allclose(np.sort(ev.real), want, atol=1e-6 * cp)
        assert np.abs(ev.imag).max() < 1e-6 * cp
