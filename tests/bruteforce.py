"""Brute-force re-derivation of one ADER-DG step with a monomial basis in
physical coordinates (used only to pin the oracle).

Independent of the oracle's basis, reference matrices, geometry tables and
neighbour search: every element carries a polynomial in the scaled monomials
((x - c)/h)^a, |a| <= N; mass matrices and exact integrals use a high-order
Legendre/Duffy rule from numpy; the Cauchy-Kovalevskaya derivatives are taken
by exact differentiation of the polynomials in physical space; neighbours are
found geometrically (face vertex sets equal up to a periodic box translation);
boundary faces use a closed-form characteristic flux in global coordinates
(boundary_flux_closed_form) rather than the face rotation and eigenvector
matrices the oracle builds.

Quadrature nodes follow the method's convention: each element's reference
map lists its vertices by increasing vertex id.  Only the pointwise law (stress, damage rate, effective Lame parameters,
B^{d,eff}), which is pinned separately, is shared.  Where the method evaluates
a nonlinear function, it does so at quadrature nodes; those nodes (collapsed
Gauss-Jacobi on the element in its vertex order, on each face in ascending
local vertex order, Gauss-Legendre in time) are rebuilt here from scipy.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.special import roots_jacobi

from oracle.rheology import cdm_damage_rate, effective_lame, flux, jacobian_eff


def exponents(N):
    return [a for d in range(N + 1) for a in itertools.product(range(d + 1), repeat=3) if sum(a) == d]


class Poly:
    def __init__(self, N, center, h):
        self.N, self.c, self.h = N, np.asarray(center), float(h)
        self.exps = np.array(exponents(N))

    def values(self, x):
        y = (np.asarray(x) - self.c) / self.h
        return np.prod(y[:, None, :] ** self.exps[None, :, :], axis=2)

    def grads(self, x):
        y = (np.asarray(x) - self.c) / self.h
        G = np.zeros((y.shape[0], len(self.exps), 3))
        for d in range(3):
            e = self.exps.copy()
            coef = e[:, d].astype(float)
            e[:, d] = np.maximum(e[:, d] - 1, 0)
            G[:, :, d] = coef[None, :] * np.prod(y[:, None, :] ** e[None, :, :], axis=2) / self.h
        return G

    def diff_matrix(self, d):
        """Coefficient map of d/dx_d within the monomial space."""
        idx = {tuple(a): i for i, a in enumerate(self.exps)}
        M = np.zeros((len(self.exps), len(self.exps)))
        for j, a in enumerate(self.exps):
            if a[d] == 0:
                continue
            b = list(a)
            b[d] -= 1
            M[idx[tuple(b)], j] = a[d] / self.h
        return M


def collapsed_tet_nodes(n):
    a, wa = roots_jacobi(n, 0, 0)
    b, wb = roots_jacobi(n, 1, 0)
    c, wc = roots_jacobi(n, 2, 0)
    P, W = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                P.append(((1 + a[i]) * (1 - b[j]) * (1 - c[k]) / 8, (1 + b[j]) * (1 - c[k]) / 4, (1 + c[k]) / 2))
                W.append(wa[i] * wb[j] * wc[k] / 64)
    return np.array(P), np.array(W)


def collapsed_tri_nodes(n):
    a, wa = roots_jacobi(n, 0, 0)
    b, wb = roots_jacobi(n, 1, 0)
    P, W = [], []
    for i in range(n):
        for j in range(n):
            P.append(((1 + a[i]) * (1 - b[j]) / 4, (1 + b[j]) / 2))
            W.append(wa[i] * wb[j] / 8)
    return np.array(P), np.array(W)        # weights sum to the area 1/2


def duffy_rule(n):
    """High-order rule on the unit tetrahedron from Gauss-Legendre on the cube."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1)
    w = 0.5 * w
    P, W = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                u, v, s = x[i], x[j], x[k]
                P.append((u * (1 - v) * (1 - s), v * (1 - s), s))
                W.append(w[i] * w[j] * w[k] * (1 - v) * (1 - s) ** 2)
    return np.array(P), np.array(W)


def boundary_flux_closed_form(bc, u, n, lam, mu, rho):
    """Normal flux on a boundary face in global coordinates, derived here from
    the characteristic decomposition of the effective isotropic Jacobian
    instead of the face rotation and eigenvector matrices.

    With tau = sigma n the traction (sigma from the effective Hooke law),
    a = -v.n + c_p sigma_nn / (lambda + 2 mu) and the tangential vector
    b = -v_tan / 2 + c_s (eps n)_tan:
      free surface: the boundary state has zero traction and the incoming
        characteristic amplitudes that achieve it, so the flux is the strain
        part a n n^T + n b^T + b n^T and zero velocity flux;
      absorbing: half of that strain part, and the velocity flux
        (-sigma_nn / rho + c_p v.n) n / 2 + (-tau_tan / rho + c_s v_tan) / 2
        (only the outgoing characteristics).
    alpha has no flux.  u: [..., 10]; returns [..., 10]."""
    u = np.asarray(u, float)
    n = np.asarray(n, float)
    cp, cs = math.sqrt((lam + 2 * mu) / rho), math.sqrt(mu / rho)
    Em = u[..., SYM_IDX]                                   # [...,3,3]
    v = u[..., 6:9]
    I1 = Em[..., 0, 0] + Em[..., 1, 1] + Em[..., 2, 2]
    En = Em @ n
    enn = En @ n
    snn = lam * I1 + 2 * mu * enn
    vn = v @ n
    vt = v - vn[..., None] * n
    et = En - enn[..., None] * n
    a = -vn + cp * snn / (lam + 2 * mu)
    b = -0.5 * vt + cs * et
    Fe = (a[..., None, None] * np.outer(n, n) + n[:, None] * b[..., None, :]
          + b[..., :, None] * n[None, :])
    F = np.zeros_like(u)
    for p, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))):
        F[..., p] = Fe[..., i, j]
    if bc == 1:
        return F
    if bc != 2:
        raise ValueError(bc)
    F[..., 0:6] *= 0.5
    F[..., 6:9] = (0.5 * (-snn / rho + cp * vn))[..., None] * n + 0.5 * (-2 * mu * et / rho + cs * vt)
    return F


SYM_IDX = np.array([[0, 3, 5], [3, 1, 4], [5, 4, 2]])


class BruteForce:
    def __init__(self, xyz, vid, N, mat, box, face_bc=None):
        # node placement convention of the method (reading R15): vertices by increasing id
        order = np.argsort(np.asarray(vid), axis=1, kind="stable")
        rows = np.arange(len(order))[:, None]
        self.xyz = np.asarray(xyz, float)[rows, order]
        self.E = self.xyz.shape[0]
        self.face_bc = (np.zeros((self.E, 4), dtype=np.int8) if face_bc is None
                        else np.asarray(face_bc)[rows, order])
        self.N = N
        self.mat = np.asarray(mat, float)
        self.box = np.asarray(box, float)
        self.polys = []
        self.M = []
        hp, hw = duffy_rule(2 * N + 4)
        self.hq = []
        for e in range(self.E):
            X = self.xyz[e]
            J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
            vol6 = abs(np.linalg.det(J))
            p = Poly(N, X.mean(axis=0), np.max(np.linalg.norm(X - X.mean(axis=0), axis=1)))
            xq = X[0] + hp @ J.T
            V = p.values(xq)
            W = hw * vol6
            self.polys.append(p)
            self.M.append(V.T @ (W[:, None] * V))
            self.hq.append((xq, W))
        self._neighbours()
        self.vn, self.vw = collapsed_tet_nodes(N + 1)
        self.fn, self.fw = collapsed_tri_nodes(N + 1)
        tx, tw = np.polynomial.legendre.leggauss(N + 1)
        self.tx, self.tw = 0.5 * (tx + 1), 0.5 * tw

    def _neighbours(self):
        self.nbr = np.full((self.E, 4), -1)
        self.shift = np.zeros((self.E, 4, 3))
        keyed = {}
        for e in range(self.E):
            for f in range(4):
                if self.face_bc[e, f] != 0:
                    continue
                vs = self.xyz[e, [v for v in range(4) if v != f]]
                wrapped = np.mod(vs + 1e-6 * self.box, self.box)
                key = tuple(sorted(tuple(np.round(w / self.box * 1e6).astype(int)) for w in wrapped))
                keyed.setdefault(key, []).append((e, f))
        for key, lst in keyed.items():
            assert len(lst) == 2, "non-conforming face"
            (e0, f0), (e1, f1) = lst
            c0 = self.xyz[e0, [v for v in range(4) if v != f0]].mean(axis=0)
            c1 = self.xyz[e1, [v for v in range(4) if v != f1]].mean(axis=0)
            self.nbr[e0, f0], self.nbr[e1, f1] = e1, e0
            self.shift[e0, f0], self.shift[e1, f1] = c1 - c0, c0 - c1

    def project(self, func):
        C = []
        for e in range(self.E):
            xq, W = self.hq[e]
            V = self.polys[e].values(xq)
            C.append(np.linalg.solve(self.M[e], V.T @ (W[:, None] * func(e, xq))))
        return np.array(C)

    def evaluate(self, C, e, x):
        return self.polys[e].values(x) @ C[e]

    def step(self, C, dt):
        N, E = self.N, self.E
        taylor = []
        cp = np.empty(E)
        lame = np.empty((E, 2))
        for e in range(E):
            p, mat = self.polys[e], self.mat[e]
            xq, W = self.hq[e]
            ubar = (W @ (p.values(xq) @ C[e])) / W.sum()
            lam, mu = effective_lame(ubar, mat)
            lame[e] = lam, mu
            cp[e] = math.sqrt((lam + 2 * mu) / mat[0])
            B = jacobian_eff(np.array(lam), np.array(mu), np.array(mat[0]))
            Dm = [p.diff_matrix(d) for d in range(3)]
            D = [C[e]]
            X = self.xyz[e]
            J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
            xv = X[0] + self.vn @ J.T
            Wv = self.vw * abs(np.linalg.det(J))
            Vv = p.values(xv)
            for i in range(1, N + 1):
                # d/dt u = -B^d d/dx_d u, exactly in the monomial space
                Di = -sum(Dm[d] @ D[i - 1] @ B[d].T for d in range(3))
                if i == 1:
                    r = cdm_damage_rate(Vv @ C[e], mat)
                    Di[:, 9] += np.linalg.solve(self.M[e], Vv.T @ (Wv * r))
                D.append(Di)
            taylor.append(D)

        def u_at(e, x, t):
            V = self.polys[e].values(x)
            return sum(t ** i / math.factorial(i) * (V @ taylor[e][i]) for i in range(N + 1))

        out = np.empty_like(C)
        for e in range(E):
            p, mat = self.polys[e], self.mat[e]
            X = self.xyz[e]
            J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
            xv = X[0] + self.vn @ J.T
            Wv = self.vw * abs(np.linalg.det(J))
            Vv, Gv = p.values(xv), p.grads(xv)
            rhs = np.zeros_like(C[e])
            for tz, gz in zip(self.tx * dt, self.tw * dt):
                u = u_at(e, xv, tz)
                F = flux(u, mat)                               # [q,3,10]
                rhs += gz * np.einsum("q,qkd,qdp->kp", Wv, Gv, F)
                s = np.zeros_like(u)
                s[:, 9] = cdm_damage_rate(u, mat)
                rhs += gz * np.einsum("q,qk,qp->kp", Wv, Vv, s)
            for f in range(4):
                a, b, c = [v for v in range(4) if v != f]
                xf = X[a] + np.outer(self.fn[:, 0], X[b] - X[a]) + np.outer(self.fn[:, 1], X[c] - X[a])
                cr = np.cross(X[b] - X[a], X[c] - X[a])
                area = 0.5 * np.linalg.norm(cr)
                n = cr / np.linalg.norm(cr)
                if n @ (X[f] - X[a]) > 0:
                    n = -n
                Wf = self.fw * 2 * area
                nb = self.nbr[e, f]
                Vf = p.values(xf)
                for tz, gz in zip(self.tx * dt, self.tw * dt):
                    um = u_at(e, xf, tz)
                    if nb < 0:
                        Fs = boundary_flux_closed_form(int(self.face_bc[e, f]), um, n, lame[e, 0], lame[e, 1], mat[0])
                        rhs -= gz * Vf.T @ (Wf[:, None] * Fs)
                        continue
                    up = u_at(nb, xf + self.shift[e, f], tz)
                    Fm = np.einsum("qdp,d->qp", flux(um, mat), n)
                    Fp = np.einsum("qdp,d->qp", flux(up, self.mat[nb]), n)
                    Fs = 0.5 * (Fm + Fp) + 0.5 * max(cp[e], cp[nb]) * (um - up)
                    Fs[:, 9] = 0.0
                    rhs -= gz * Vf.T @ (Wf[:, None] * Fs)
            out[e] = C[e] + np.linalg.solve(self.M[e], rhs)
        return out
