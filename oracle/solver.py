"""FP64 ADER-DG step for the CDM damage rheology on tetrahedra (oracle; test
infrastructure only).

One step from t_n to t_{n+1} = t_n + dt, in the order of Appendix A:
  1. cell mean u_bar of the state (mode 0);
  2. effective Lame parameters at u_bar (Eq. "effective-cdb", readings R1/R2/R7;
     Eq. "effective-ivm" with law="ivm");
  3. effective Jacobians B^{d,eff} (Eqs. "matrix_Beff_1..3", readings T1/T2);
  4. star matrices A*_e = Theta^{-1}_{ed} B^{d,eff};
  5. Cauchy-Kovalevskaya predictor D^i = -K^e D^{i-1} A*_e^T (Eq. "CKIter-ref-matrix",
     index reading R10), with the damage-rate source added at i = 1 only
     (Eq. "CKIter-ref-source", reading R11), projected with the volume rule (R4);
  6. Taylor expansion U(t) (Eq. "eq:taylor_expansion") at the time nodes;
  7. volume term int dphi_k/dx_d int F^d (Eq. "3rd term") and source term
     int phi_k int s (Eq. "rhs term") by space-time quadrature (reading R4);
  8. Rusanov flux (Eq. "rusanov-flux") at the face space-time nodes
     (Eq. "2nd term"), neighbour trace taken at the same physical point by
     inverting the neighbour's affine map, C = max of the two cells'
     effective P speeds (reading R3), no flux on alpha (reading R6); on
     boundary faces the absorbing or free-surface flux of Appendix A
     ("Free surface and absorbing boundary conditions", oracle/boundary.py);
  9. update of Eq. "time-integrated" with M = I (orthonormal basis).
Point sources enter step 9 as strain-rate deltas; receivers sample velocity.
The pointwise law is the CDM of Eq. "cdb-model" (law="cdm", default), the IVM
of Eq. "ivm-model" without Murnaghan terms (law="ivm") or the nonlinear shear
law of the 1-D Riemann verification (law="nlshear", Eq. "1d Riemann eqs",
reading R19), whose effective moduli in step 2 are its secant moduli.

State layout inside the oracle: Q[E, L, 10] (mode, field), modes of the
Dubiner basis mapped onto each element with its vertices in increasing vertex
id (reading R15).  The C-ABI layout [E, 10, L] is produced by to_abi()/from_abi().
"""
from __future__ import annotations

import math

import numpy as np

from .basis import eval_basis, mode_list, n_modes
from .boundary import boundary_matrix
from .quadrature import gauss_legendre_01, tet_rule, tri_rule
from .rheology import (damage_rate, effective_lame_law, energy, flux,
                       invariants, jacobian_eff)

REF_VERTS = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
PHI0 = math.sqrt(6.0)


class MeshError(ValueError):
    pass


def to_abi(Q):
    return np.ascontiguousarray(np.swapaxes(Q, 1, 2))


def from_abi(q):
    return np.ascontiguousarray(np.swapaxes(q, 1, 2))


def face_vertices(f):
    """Local vertices of face f (the face opposite vertex f), ascending."""
    return [v for v in range(4) if v != f]


def stf_integral(src, t):
    """Antiderivative of the moment-rate time function, zero at -infinity.
    stf 0: Ricker w(t) = (1 - 2 c tau^2) exp(-c tau^2), c = (pi f0)^2, tau = t - t0,
           antiderivative tau exp(-c tau^2);
    stf 1: Gaussian rate of standard deviation sigma (the "sigma" field, or "f0"
           as in the C-ABI's f0_or_sigma), unit integral."""
    tau = t - src["t0"]
    if src["stf"] == 0:
        c = (math.pi * src["f0"]) ** 2
        return tau * math.exp(-c * tau * tau)
    sig = src["sigma"] if "sigma" in src else src["f0"]
    return 0.5 * (1.0 + math.erf(tau / (sig * math.sqrt(2.0))))


class Oracle:
    def __init__(self, elem_xyz, elem_vid, order, material, face_bc=None, cfl=0.5, face_rows=None,
                 law="cdm", picard_iterations=0):
        """face_rows: elements whose face tables are built (default all); step()
        can only produce new states for those elements.  picard_iterations > 0
        refines the CK predictor by that many discrete Picard iterations
        (Sec. 5.1's proposed extension, reading R20); 0 keeps the CK predictor."""
        xyz = np.asarray(elem_xyz, dtype=np.float64)
        vid = np.asarray(elem_vid, dtype=np.int64)
        # Reading R15: each element's reference map lists its vertices by
        # increasing global vertex id, so the face nodes seen from the two
        # elements of a face are the same physical points.
        vorder = np.argsort(vid, axis=1, kind="stable")
        rows = np.arange(xyz.shape[0])[:, None]
        self.xyz = np.ascontiguousarray(xyz[rows, vorder])
        self.vid = np.ascontiguousarray(vid[rows, vorder])
        self.E = self.xyz.shape[0]
        self.N = int(order)
        self.L = n_modes(self.N)
        self.mat = np.asarray(material, dtype=np.float64).reshape(self.E, 6)
        self.face_bc = (np.zeros((self.E, 4), dtype=np.int8) if face_bc is None
                        else np.asarray(face_bc, dtype=np.int8)[rows, vorder])
        if np.any((self.face_bc < 0) | (self.face_bc > 2)):
            raise MeshError("face tags must be 0 (interior), 1 (free surface) or 2 (absorbing)")
        if law not in ("cdm", "ivm", "nlshear"):
            raise ValueError(f"unknown rheology {law}")
        self.law = law
        self.picard_iterations = int(picard_iterations)
        self.flag_nonhyperbolic = False
        self.cfl = cfl
        self._reference()
        self._geometry()
        self._match_faces()
        self.face_rows = np.arange(self.E) if face_rows is None else np.unique(np.asarray(face_rows))
        self._face_tables()
        self.sources = []
        self.receivers = None

    # ---------------- reference element ----------------
    def _reference(self):
        N = self.N
        self.qv_pts, self.qv_w = tet_rule(N + 1)
        self.Vv, Gv = eval_basis(N, self.qv_pts, grad=True)       # [Nq,L], [Nq,L,3]
        self.Gv = Gv
        # K^e_{kl} = int phi_k d phi_l / d xi_e  (stored as Kt[e, k, l])
        self.Kt = np.einsum("q,qk,qle->ekl", self.qv_w, self.Vv, Gv, optimize=True)
        self.qf_pts, self.qf_w = tri_rule(N + 1)                   # weights sum to 1
        self.qt_x, self.qt_w = gauss_legendre_01(N + 1)

    # ---------------- geometry ----------------
    def _geometry(self):
        X = self.xyz
        J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)  # x = X0 + J xi
        det = np.linalg.det(J)
        scale = np.max(np.abs(J), axis=(1, 2)) ** 3
        if np.any(np.abs(det) <= 1e-12 * scale):
            raise MeshError("degenerate tetrahedron")
        self.J = J
        self.detJ = np.abs(det)
        self.Jinv = np.linalg.inv(J)                 # Theta^{-1}[e, d] = d xi_e / d x_d
        self.normal = np.empty((self.E, 4, 3))
        self.area = np.empty((self.E, 4))
        for f in range(4):
            a, b, c = face_vertices(f)
            cr = np.cross(X[:, b] - X[:, a], X[:, c] - X[:, a])
            nrm = np.linalg.norm(cr, axis=1)
            n = cr / nrm[:, None]
            flip = np.einsum("ed,ed->e", n, X[:, f] - X[:, a]) > 0
            n[flip] *= -1
            self.normal[:, f] = n
            self.area[:, f] = 0.5 * nrm
        # inradius 3V / surface
        vol = self.detJ / 6.0
        self.r_in = 3.0 * vol / self.area.sum(axis=1)

    def cfl_dt(self):
        """dt = cfl * 2 r_in / ((2N+1) c_p), minimised over elements (the paper
        does not state its time-step rule)."""
        rho, lam, mu = self.mat[:, 0], self.mat[:, 1], self.mat[:, 2]
        cp = np.sqrt((lam + 2 * mu) / rho)
        return float(np.min(self.cfl * 2.0 * self.r_in / ((2 * self.N + 1) * cp)))

    def _match_faces(self):
        """Interior faces pair up by their vertex-id triple; a face tagged as a
        boundary (free surface or absorbing) must belong to one element only
        and keeps nbr = -1."""
        keys = {}
        for e in range(self.E):
            if len(set(self.vid[e].tolist())) != 4:
                raise MeshError("element with repeated vertex ids")
            for f in range(4):
                key = tuple(sorted(self.vid[e, face_vertices(f)].tolist()))
                keys.setdefault(key, []).append((e, f))
        self.nbr = -np.ones((self.E, 4), dtype=np.int64)
        self.nbr_face = -np.ones((self.E, 4), dtype=np.int64)
        self.shift = np.zeros((self.E, 4, 3))
        for key, lst in keys.items():
            tagged = [self.face_bc[e, f] != 0 for e, f in lst]
            if any(tagged):
                if len(lst) != 1:
                    raise MeshError(f"boundary face {key} is shared by {len(lst)} element faces")
                continue
            if len(lst) != 2 or lst[0][0] == lst[1][0]:
                raise MeshError(f"face {key} is shared by {len(lst)} element faces")
            (e0, f0), (e1, f1) = lst
            self.nbr[e0, f0], self.nbr_face[e0, f0] = e1, f1
            self.nbr[e1, f1], self.nbr_face[e1, f1] = e0, f0
            # periodic shift: coordinates of the shared vertices seen from each side
            v0 = {int(self.vid[e0, v]): self.xyz[e0, v] for v in face_vertices(f0)}
            v1 = {int(self.vid[e1, v]): self.xyz[e1, v] for v in face_vertices(f1)}
            d = np.mean([v1[k] - v0[k] for k in key], axis=0)
            self.shift[e0, f0] = d
            self.shift[e1, f1] = -d

    def _face_tables(self):
        """Own and neighbour basis values at the face nodes of every element face."""
        s, t = self.qf_pts[:, 0], self.qf_pts[:, 1]
        Nf = s.size
        self.Vf_own = np.empty((4, Nf, self.L))
        rows = self.face_rows
        self.row_of = -np.ones(self.E, dtype=np.int64)
        self.row_of[rows] = np.arange(rows.size)
        X = self.xyz[rows]
        self.face_x = np.empty((rows.size, 4, Nf, 3))
        for f in range(4):
            a, b, c = face_vertices(f)
            R = REF_VERTS
            xi = R[a] + s[:, None] * (R[b] - R[a]) + t[:, None] * (R[c] - R[a])
            self.Vf_own[f] = eval_basis(self.N, xi)
            self.face_x[:, f] = (X[:, a, None] + s[None, :, None] * (X[:, b] - X[:, a])[:, None]
                                 + t[None, :, None] * (X[:, c] - X[:, a])[:, None])
        self.Vf_nbr = np.zeros((rows.size, 4, Nf, self.L))
        for f in range(4):
            nb = self.nbr[rows, f]
            inner = nb >= 0                                               # boundary faces have no neighbour
            nbi = nb[inner]
            xp = self.face_x[inner, f] + self.shift[rows[inner], f, None, :]   # in the neighbour's frame
            xi_nb = np.einsum("ead,eqd->eqa", self.Jinv[nbi], xp - self.xyz[nbi, 0][:, None, :], optimize=True)
            self.Vf_nbr[inner, f] = eval_basis(self.N, xi_nb.reshape(-1, 3)).reshape(nbi.size, Nf, self.L)

    # ---------------- sources / receivers ----------------
    def locate(self, x, tol=1e-10):
        """First element (index order) whose closure contains x (unwrapped coordinates)."""
        x = np.asarray(x, dtype=np.float64)
        xi = np.einsum("ead,ed->ea", self.Jinv, x[None, :] - self.xyz[:, 0], optimize=True)
        bary = np.concatenate([1.0 - xi.sum(axis=1, keepdims=True), xi], axis=1)
        inside = np.all(bary >= -tol, axis=1)
        idx = np.nonzero(inside)[0]
        if idx.size == 0:
            raise MeshError("point outside the mesh")
        e = int(idx[0])
        return e, xi[e]

    def set_sources(self, sources):
        self.sources = []
        for src in sources:
            e, xi = self.locate(src["x"])
            phi = eval_basis(self.N, xi[None, :])[0]
            rho, lam, mu = self.mat[e, 0], self.mat[e, 1], self.mat[e, 2]
            m = np.asarray(src["m"], dtype=np.float64)
            tr = m[0] + m[1] + m[2]
            # strain of the moment tensor under the undamaged stiffness C0
            eps = m / (2.0 * mu)
            eps[:3] -= lam / (2.0 * mu * (3.0 * lam + 2.0 * mu)) * tr
            self.sources.append({"e": e, "phi": phi, "eps": eps, "src": src})

    def set_receivers(self, xyz):
        self.receivers = []
        for x in np.asarray(xyz, dtype=np.float64).reshape(-1, 3):
            e, xi = self.locate(x)
            self.receivers.append((e, eval_basis(self.N, xi[None, :])[0]))

    def sample_receivers(self, Q):
        if not self.receivers:
            return np.zeros((0, 3))
        return np.stack([phi @ Q[e, :, 6:9] for e, phi in self.receivers])

    # ---------------- the step ----------------
    def predictor(self, Q, rows):
        """Steps 1-5 for the elements in `rows`: Taylor coefficients D[i] of shape
        [len(rows), L, 10], i = 0..N, the effective P speed of each cell and its
        effective Lame parameters (lambda_eff, mu_eff)."""
        mat = self.mat[rows]
        Qr = Q[rows]
        ubar = Qr[:, 0, :] * PHI0                                         # 1. cell mean
        lam, mu = effective_lame_law(ubar, mat, self.law)                # 2.
        rho = mat[:, 0]
        self.flag_nonhyperbolic |= bool(np.any((mu <= 0) | (lam + 2 * mu <= 0)))
        cp = np.sqrt(np.maximum(lam + 2 * mu, 0.0) / rho)
        B = jacobian_eff(lam, mu, rho)                                   # 3. [n,3(d),10,10]
        Astar = np.einsum("ned,ndpq->nepq", self.Jinv[rows], B, optimize=True)          # 4.
        D = [Qr]
        for i in range(1, self.N + 1):                                   # 5.
            G = np.einsum("ekl,nlq->nekq", self.Kt, D[i - 1], optimize=True)
            Di = -np.einsum("nekq,nepq->nkp", G, Astar, optimize=True)
            if i == 1:
                uq = np.einsum("ql,nlp->nqp", self.Vv, Qr, optimize=True)
                r = damage_rate(uq, mat[:, None, :], self.law)
                Di[:, :, 9] += np.einsum("q,qk,nq->nk", self.qv_w, self.Vv, r, optimize=True)
            D.append(Di)
        return np.stack(D, axis=0), cp, (lam, mu)

    def picard(self, D, rows, dt, iterations):
        """Discrete Picard iteration on the element-local evolution (reading R20):
        with q(t) = sum_i t^i/i! D^i the predictor's polynomial, one iteration
        evaluates R(q) = -div F(q) + S(q) at the Gauss time nodes t_z of the step,
          R_kp(t_z) = -sum_e sum_l Kt[e,k,l] Fhat*_{l,e,p}(t_z) + Shat_kp(t_z),
        Fhat* the volume-rule projection of Theta^{-1}_{ed} F^d(q_h) and Shat that
        of the source (the damage rate), fits the interpolating polynomial
        sum_j t^j/j! R^j through the N + 1 values, and sets D^{j+1} = R^j.  Each
        D^o is then truncated as the CK's is (degree N - o for the wave fields,
        first order for alpha), so the output keeps the predictor's form.  For a
        linear flux the CK coefficients are a fixed point."""
        N, L = self.N, self.L
        mat = self.mat[rows]
        Jinv = self.Jinv[rows]
        tz = self.qt_x * dt
        V = np.array([[t ** j / math.factorial(j) for j in range(N + 1)] for t in tz])   # [z, j]
        Vinv = np.linalg.inv(V)
        deg = np.array([sum(m) for m in mode_list(N)])
        D = np.array(D, copy=True)
        for _ in range(iterations):
            U = np.einsum("zi,inlp->nzlp", V, D, optimize=True)
            u = np.einsum("ql,nzlp->nzqp", self.Vv, U, optimize=True)
            F = flux(u, mat[:, None, None, :], self.law)                       # [n,z,q,3(d),10]
            Fs = np.einsum("ned,nzqdp->nzqep", Jinv, F, optimize=True)
            Fh = np.einsum("q,ql,nzqep->nzlep", self.qv_w, self.Vv, Fs, optimize=True)
            R = -np.einsum("ekl,nzlep->nzkp", self.Kt, Fh, optimize=True)
            r = damage_rate(u, mat[:, None, None, :], self.law)                # [n,z,q]
            R[..., 9] += np.einsum("q,ql,nzq->nzl", self.qv_w, self.Vv, r, optimize=True)
            Rj = np.einsum("jz,nzkp->jnkp", Vinv, R, optimize=True)
            for o in range(1, N + 1):
                Do = Rj[o - 1].copy()
                Do[:, deg > N - o, :9] = 0.0
                if o > 1:
                    Do[..., 9] = 0.0
                D[o] = Do
        return D

    def step(self, Q, dt, t=0.0, rows=None):
        """Advance Q[E,L,10] by dt; returns the new state (all elements, or only
        `rows` when given, as an array [len(rows),L,10])."""
        self.flag_nonhyperbolic = False
        out_rows = np.arange(self.E) if rows is None else np.asarray(rows, dtype=np.int64)
        nbrs = self.nbr[out_rows].ravel()
        need = np.unique(np.concatenate([out_rows, nbrs[nbrs >= 0]]))
        pos = -np.ones(self.E, dtype=np.int64)
        pos[need] = np.arange(need.size)
        D, cp, (lam_eff, mu_eff) = self.predictor(Q, need)
        if self.picard_iterations > 0:
            D = self.picard(D, need, dt, self.picard_iterations)
        tz = self.qt_x * dt
        gz = self.qt_w * dt
        N = self.N
        # 6. U(t_z) = sum_i (t_z)^i / i! D^i  -> [n, Nt, L, 10]
        coef = np.array([[tz_ ** i / math.factorial(i) for i in range(N + 1)] for tz_ in tz])
        U = np.einsum("zi,inlp->nzlp", coef, D, optimize=True)
        new = np.empty((out_rows.size, self.L, 10))
        chunk = 256
        for c0 in range(0, out_rows.size, chunk):
            rr = out_rows[c0:c0 + chunk]
            pr = pos[rr]
            mat = self.mat[rr]
            # 7. volume and source terms (reference measure; |J| cancels)
            uq = np.einsum("ql,nzlp->nzqp", self.Vv, U[pr], optimize=True)
            F = flux(uq, mat[:, None, None, :], self.law)                    # [n,z,q,3,10]
            s = np.zeros_like(uq)
            s[..., 9] = damage_rate(uq, mat[:, None, None, :], self.law)
            gphys = np.einsum("qke,ned->nqkd", self.Gv, self.Jinv[rr], optimize=True)       # d phi_k / d x_d
            vol = np.einsum("z,q,nqkd,nzqdp->nkp", gz, self.qv_w, gphys, F, optimize=True)
            src = np.einsum("z,q,qk,nzqp->nkp", gz, self.qv_w, self.Vv, s, optimize=True)
            # 8. face terms
            face = np.zeros((rr.size, self.L, 10))
            for f in range(4):
                nb = self.nbr[rr, f]
                inner = nb >= 0
                nbs = np.where(inner, nb, rr)          # boundary rows: placeholder, replaced below
                n = self.normal[rr, f]
                um = np.einsum("il,nzlp->nzip", self.Vf_own[f], U[pr], optimize=True)
                fr = self.row_of[rr]
                if np.any(fr < 0):
                    raise ValueError("face tables were not built for some requested rows")
                up = np.einsum("nil,nzlp->nzip", self.Vf_nbr[fr, f], U[pos[nbs]], optimize=True)
                Fm = np.einsum("nzidp,nd->nzip", flux(um, mat[:, None, None, :], self.law), n, optimize=True)
                Fp = np.einsum("nzidp,nd->nzip", flux(up, self.mat[nbs][:, None, None, :], self.law), n,
                               optimize=True)
                C = np.maximum(cp[pr], cp[pos[nbs]])
                Fs = 0.5 * (Fp + Fm) + 0.5 * C[:, None, None, None] * (um - up)
                # boundary faces (Appendix A): flux matrix of the face applied to the own trace
                for k in np.nonzero(~inner)[0]:
                    e = rr[k]
                    Mb = boundary_matrix(int(self.face_bc[e, f]), self.normal[e, f], lam_eff[pr[k]],
                                         mu_eff[pr[k]], self.mat[e, 0])
                    Fs[k] = np.einsum("pq,ziq->zip", Mb, um[k])
                Fs[..., 9] = 0.0
                face += self.area[rr, f][:, None, None] * np.einsum(
                    "z,i,ik,nzip->nkp", gz, self.qf_w, self.Vf_own[f], Fs, optimize=True)
            # 9. update
            new[c0:c0 + chunk] = Q[rr] + vol + src - face / self.detJ[rr][:, None, None]
        # point sources: strain rate -C0^{-1}:M w(t) delta(x - x_s), time integrated
        for s_ in self.sources:
            e = s_["e"]
            k = np.nonzero(out_rows == e)[0]
            if k.size == 0:
                continue
            amp = stf_integral(s_["src"], t + dt) - stf_integral(s_["src"], t)
            new[k[0], :, 0:6] -= np.outer(s_["phi"], s_["eps"]) * amp / self.detJ[e]
        return new

    def run(self, Q, dt, n_steps, t0=0.0, record=False):
        t = t0
        traces = []
        for _ in range(n_steps):
            Q = self.step(Q, dt, t)
            t += dt
            if record:
                traces.append(self.sample_receivers(Q))
        return (Q, np.array(traces)) if record else Q

    # ---------------- diagnostics ----------------
    def project(self, func, rule_points=None):
        """L2 projection of func(x[...,3]) -> [...,10] onto the modes of each element."""
        n = self.N + 2 if rule_points is None else rule_points
        pts, w = tet_rule(n)
        V = eval_basis(self.N, pts)
        x = self.xyz[:, 0, None, :] + np.einsum("edk,qk->eqd", self.J, pts, optimize=True)
        vals = func(x)
        return np.einsum("q,qk,eqp->ekp", w, V, vals, optimize=True)

    def to_reference(self, e, x):
        """Reference coordinates in element e of physical points x[...,3]."""
        return (np.asarray(x) - self.xyz[e, 0]) @ self.Jinv[e].T

    def evaluate_at(self, Q, e, x):
        """Fields [...,10] of element e at physical points x[...,3]."""
        xi = self.to_reference(e, x).reshape(-1, 3)
        return (eval_basis(self.N, xi) @ Q[e]).reshape(np.shape(x)[:-1] + (10,))

    def evaluate(self, Q, pts_ref):
        V = eval_basis(self.N, pts_ref)
        return np.einsum("ql,elp->eqp", V, Q, optimize=True)

    def energy(self, Q):
        """int (rho |v|^2 / 2 + W(eps, alpha)) dV over the mesh."""
        pts, w = tet_rule(self.N + 2)
        u = self.evaluate(Q, pts)
        mat = self.mat[:, None, :]
        kin = 0.5 * mat[..., 0] * np.sum(u[..., 6:9] ** 2, axis=-1)
        W = energy(u, mat, self.law)
        return float(np.sum(self.detJ[:, None] * w[None, :] * (kin + W)))

    def damage_dissipation_rate(self, Q):
        """-int dW/dalpha * r_alpha dV  (>= 0): energy removed by damage growth."""
        pts, w = tet_rule(self.N + 2)
        u = self.evaluate(Q, pts)
        mat = self.mat[:, None, :]
        I1, I2, s, xi = invariants(u)
        if self.law == "nlshear":
            return 0.0
        if self.law == "ivm":
            dWda = -(0.5 * mat[..., 1] * I1 * I1 + mat[..., 2] * I2)
        else:
            dWda = mat[..., 4] * mat[..., 3] * I2 - mat[..., 3] * I1 * s
        r = damage_rate(u, mat, self.law)
        return float(-np.sum(self.detJ[:, None] * w[None, :] * dWda * r))
