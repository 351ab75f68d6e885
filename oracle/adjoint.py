"""Discrete adjoint of the oracle's CK step under the CDM law (test
infrastructure only).

The receiver misfit of a run of n steps from Q^0,
    J = 1/2 sum_{k=1..n} dt sum_r |v_r(Q^k) - v_r^ref(t_k)|^2,
is differentiated with respect to the per-element damage parameters xi0 and
C_d of Eq. "cdb-model" (and the initial state) by reverse accumulation through
the steps of Oracle.step, in the order of Appendix A:
    Q^{k+1} = Q^k + vol(U) + src(U) - face(U, U_nbr, C) / |J|,
U the Taylor expansion of the CK predictor (Eqs. "CKIter-ref-matrix",
"CKIter-ref-source") whose star matrices depend on the cell mean through the
effective Lame parameters (Eq. "effective-cdb"), C = max of the two cells'
effective P speeds (Eq. "rusanov-flux", reading R3).  Every product of the
forward step is transposed here as written, with the derivative of each
pointwise map (stress, damage rate, effective Lame parameters, P speed) taken
by hand.  Conventions at the non-smooth points (reading R21): the damage rate
C_d gamma_r max(0, I1 sqrt(I2) - xi0 I2) has derivative zero where its
argument is <= 0; xi and sqrt(I2) have derivative zero below I2 = 1e-30; at a
tie of the two P speeds the derivative of the max is split in halves, which is
what a central difference sees.

Pins (tests/test_oracle_adjoint.py): each pointwise derivative against central
differences of the forward law, the step adjoint against central differences
of Oracle.step along random directions (the dot-product test), and the misfit
gradient against central differences of whole runs, element by element.
Boundary faces (free surface, absorbing) are covered: their flux is linear in
the own trace with a matrix of the own cell's effective Lame parameters, whose
derivative in those parameters is taken by a central difference of relative
step 1e-6 (error ~1e-10 of the term).  The Picard predictor and the other laws
are not covered.
"""
from __future__ import annotations

import math

import numpy as np

from .rheology import I2_FLOOR, invariants, jacobian_eff, strain_tensor
from .boundary import boundary_matrix
from .solver import PHI0

_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))


def _dI(u):
    """dI1/du_p and dI2/du_p (p < 6) of the strain entries u[..., :6]: I2 counts
    each shear entry twice."""
    d1 = np.zeros(u.shape[:-1] + (6,))
    d1[..., :3] = 1.0
    d2 = np.concatenate([2.0 * u[..., :3], 4.0 * u[..., 3:6]], axis=-1)
    return d1, d2


def _ds_dxi(u):
    """s = sqrt(I2), xi = I1 / s and their derivatives in u[..., :6] (zero below
    the I2 floor)."""
    I1, I2, s, xi = invariants(u)
    d1, d2 = _dI(u)
    live = I2 > I2_FLOOR
    sg = np.where(live, s, 1.0)
    ds = np.where(live[..., None], d2 / (2.0 * sg[..., None]), 0.0)
    dxi = np.where(live[..., None], d1 / sg[..., None] - (I1 / (sg * sg))[..., None] * ds, 0.0)
    return I1, I2, s, xi, ds, dxi


def stress_vjp(u, mat, lam_sig):
    """Gradient of sum_ij lam_sig_ij sigma_ij(u) (CDM stress of Eq. "cdb-model",
    lam_sig [..., 3, 3]) with respect to u[..., :10] and xi0."""
    lam0, gr, xi0 = mat[..., 1], mat[..., 3], mat[..., 4]
    alpha = u[..., 9]
    mu0 = mat[..., 2]
    I1, I2, s, xi, ds, dxi = _ds_dxi(u)
    e = strain_tensor(u)
    tr = lam_sig[..., 0, 0] + lam_sig[..., 1, 1] + lam_sig[..., 2, 2]
    le = np.einsum("...ij,...ij->...", lam_sig, e)
    ag = alpha * gr
    sh = 2.0 * (mu0 + ag * xi0) - ag * xi
    out = np.zeros(u.shape)
    d1, _ = _dI(u)
    diso = lam0[..., None] * d1 - ag[..., None] * ds
    dsh = -ag[..., None] * dxi
    out[..., :6] = tr[..., None] * diso + le[..., None] * dsh
    for p, (i, j) in enumerate(_PAIRS):
        direct = lam_sig[..., i, j] + (lam_sig[..., j, i] if i != j else 0.0)
        out[..., p] += sh * direct
    out[..., 9] = tr * (-gr * s) + le * (2.0 * gr * xi0 - gr * xi)
    g_xi0 = le * 2.0 * ag
    return out, g_xi0


def rate_vjp(u, mat, lam_r):
    """Gradient of lam_r * r(u) (CDM damage rate) with respect to u[..., :10],
    xi0 and C_d."""
    gr, xi0, cd = mat[..., 3], mat[..., 4], mat[..., 5]
    I1, I2, s, xi, ds, dxi = _ds_dxi(u)
    d1, d2 = _dI(u)
    arg = I1 * s - xi0 * I2
    on = arg > 0.0
    k = np.where(on, lam_r * cd * gr, 0.0)
    out = np.zeros(u.shape)
    out[..., :6] = k[..., None] * (d1 * s[..., None] + I1[..., None] * ds - xi0[..., None] * d2)
    g_xi0 = -k * I2
    g_cd = lam_r * gr * np.maximum(0.0, arg)
    return out, g_xi0, g_cd


def lame_vjp(ubar, mat, a_lam, a_mu):
    """Gradient of a_lam lambda_eff + a_mu mu_eff (Eq. "effective-cdb") with
    respect to the cell mean ubar[..., :10] and xi0."""
    gr, xi0 = mat[..., 3], mat[..., 4]
    alpha = ubar[..., 9]
    _, _, _, xi, _, dxi = _ds_dxi(ubar)
    w = a_lam / 3.0 + 0.5 * a_mu
    out = np.zeros(ubar.shape)
    out[..., :6] = -(alpha * gr * w)[..., None] * dxi
    out[..., 9] = -gr * xi * w + a_mu * xi0 * gr
    return out, a_mu * alpha * gr


def flux_vjp(u, mat, lam_F):
    """Gradient of sum_{d,p} lam_F[..., d, p] F^d_p(u) (flux of Eq. "nonlinear hyper
    pdes", lam_F [..., 3, 10]) with respect to u[..., :10] and xi0."""
    rho = mat[..., 0]
    out = np.zeros(u.shape)
    for p, (i, j) in enumerate(_PAIRS):
        out[..., 6 + i] += -0.5 * lam_F[..., j, p]
        out[..., 6 + j] += -0.5 * lam_F[..., i, p]
    # F[d, 6+i] = -sigma_{i d} / rho
    lam_sig = -np.swapaxes(lam_F[..., :, 6:9], -1, -2) / rho[..., None, None]
    su, g = stress_vjp(u, mat, lam_sig)
    return out + su, g


def _lame_partials(rho):
    """dB/dlambda and dB/dmu of the effective Jacobians (they are affine in
    lambda and mu)."""
    z = np.zeros_like(rho)
    o = np.ones_like(rho)
    B0 = jacobian_eff(z, z, rho)
    return jacobian_eff(o, z, rho) - B0, jacobian_eff(z, o, rho) - B0


def step_vjp(o, Q, dt, lam):
    """lam [E, L, 10] = dJ/dQ^{k+1}; returns (dJ/dQ^k, dJ/dxi0, dJ/dC_d) of
    Q^{k+1} = Oracle.step(Q^k) (all elements, CK predictor, CDM law; interior,
    free-surface and absorbing faces).  Point sources add a state-independent term
    and drop out."""
    if o.law != "cdm" or o.picard_iterations:
        raise ValueError("the oracle adjoint covers the CDM law with the CK predictor")
    E, L, N = o.E, o.L, o.N
    mat = o.mat
    rows = np.arange(E)
    D, cp, (lam_eff, mu_eff) = o.predictor(Q, rows)          # D [N+1, E, L, 10]
    tz, gz = o.qt_x * dt, o.qt_w * dt
    coef = np.array([[t ** i / math.factorial(i) for i in range(N + 1)] for t in tz])   # [z, i]
    U = np.einsum("zi,inlp->nzlp", coef, D, optimize=True)
    g_xi0 = np.zeros(E)
    g_cd = np.zeros(E)
    lamU = np.zeros_like(U)
    mz = mat[:, None, None, :]

    # 7. volume term vol_kp = sum_z gz sum_q w_q dphi_k/dx_d F^d_p(u_zq)
    uq = np.einsum("ql,nzlp->nzqp", o.Vv, U, optimize=True)
    gphys = np.einsum("qke,ned->nqkd", o.Gv, o.Jinv, optimize=True)
    lamF = np.einsum("z,q,nqkd,nkp->nzqdp", gz, o.qv_w, gphys, lam, optimize=True)
    lu, gx = flux_vjp(uq, mz, lamF)
    g_xi0 += gx.sum(axis=(1, 2))
    #    source term src_k9 = sum_z gz sum_q w_q phi_k r(u_zq)
    lam_r = np.einsum("z,q,qk,nk->nzq", gz, o.qv_w, o.Vv, lam[:, :, 9], optimize=True)
    lr, gx, gc = rate_vjp(uq, mz, lam_r)
    g_xi0 += gx.sum(axis=(1, 2))
    g_cd += gc.sum(axis=(1, 2))
    lamU += np.einsum("ql,nzqp->nzlp", o.Vv, lu + lr, optimize=True)

    # 8. face terms: new -= area/|J| sum_z gz sum_i w_i phi_k(x_i) Fs_zip
    lam_cp = np.zeros(E)
    a_lam_b = np.zeros(E)            # boundary faces: d/d lambda_eff, d/d mu_eff of the own cell
    a_mu_b = np.zeros(E)
    for f in range(4):
        nb_all = o.nbr[:, f]
        inner = nb_all >= 0
        um_all = np.einsum("il,nzlp->nzip", o.Vf_own[f], U, optimize=True)
        lamFs_all = -np.einsum("n,z,i,ik,nkp->nzip", o.area[:, f] / o.detJ, gz, o.qf_w, o.Vf_own[f], lam,
                               optimize=True)
        lamFs_all[..., 9] = 0.0
        # interior faces: Fs = (F(u-).n + F(u+).n)/2 + C/2 (u- - u+)
        rr = np.nonzero(inner)[0]
        if rr.size:
            nb = nb_all[rr]
            n = o.normal[rr, f]
            um = um_all[rr]
            lamFs = lamFs_all[rr]
            up = np.einsum("nil,nzlp->nzip", o.Vf_nbr[o.row_of[rr], f], U[nb], optimize=True)
            # d(F(u).n) / du: lam_F[d, p] = lamFs_p n_d
            lFn = np.einsum("nzip,nd->nzidp", lamFs, n, optimize=True)
            lm, gm = flux_vjp(um, mat[rr][:, None, None, :], lFn)
            lp, gp = flux_vjp(up, mat[nb][:, None, None, :], lFn)
            C = np.maximum(cp[rr], cp[nb])
            lam_um = 0.5 * lm + 0.5 * C[:, None, None, None] * lamFs
            lam_up = 0.5 * lp - 0.5 * C[:, None, None, None] * lamFs
            lC = 0.5 * np.einsum("nzip,nzip->n", lamFs, um - up, optimize=True)
            own = np.where(cp[rr] > cp[nb], 1.0, np.where(cp[rr] < cp[nb], 0.0, 0.5))
            np.add.at(lam_cp, rr, own * lC)
            np.add.at(lam_cp, nb, (1.0 - own) * lC)
            np.add.at(g_xi0, rr, 0.5 * gm.sum(axis=(1, 2)))
            np.add.at(g_xi0, nb, 0.5 * gp.sum(axis=(1, 2)))
            np.add.at(lamU, rr, np.einsum("il,nzip->nzlp", o.Vf_own[f], lam_um, optimize=True))
            np.add.at(lamU, nb, np.einsum("nil,nzip->nzlp", o.Vf_nbr[o.row_of[rr], f], lam_up, optimize=True))
        # boundary faces (Appendix A): Fs = M(lambda_eff, mu_eff) u-, M the face's flux matrix; its
        # derivative in the effective Lame parameters by a central difference of relative step 1e-6
        for k in np.nonzero(~inner)[0]:
            bc, n = int(o.face_bc[k, f]), o.normal[k, f]
            le, me, rho_k = lam_eff[k], mu_eff[k], mat[k, 0]
            Mb = boundary_matrix(bc, n, le, me, rho_k)
            lFs, uk = lamFs_all[k], um_all[k]
            lamU[k] += np.einsum("il,zip,pq->zlq", o.Vf_own[f], lFs, Mb, optimize=True)
            hl, hm = 1e-6 * abs(le) + 1e-300, 1e-6 * abs(me) + 1e-300
            dMl = (boundary_matrix(bc, n, le + hl, me, rho_k) - boundary_matrix(bc, n, le - hl, me, rho_k)) / (2 * hl)
            dMm = (boundary_matrix(bc, n, le, me + hm, rho_k) - boundary_matrix(bc, n, le, me - hm, rho_k)) / (2 * hm)
            a_lam_b[k] += np.einsum("zip,pq,ziq->", lFs, dMl, uk, optimize=True)
            a_mu_b[k] += np.einsum("zip,pq,ziq->", lFs, dMm, uk, optimize=True)

    # 6. Taylor expansion U(t_z) = sum_i t_z^i / i! D^i
    lamD = np.einsum("zi,nzlp->inlp", coef, lamU, optimize=True)

    # 5. Cauchy-Kovalevskaya D^i_kp = -sum_e Kt^e_kl D^{i-1}_lq A*^e_pq, transposed from i = N down
    rho = mat[:, 0]
    B = jacobian_eff(lam_eff, mu_eff, rho)
    Astar = np.einsum("ned,ndpq->nepq", o.Jinv, B, optimize=True)
    lamA = np.zeros_like(Astar)
    for i in range(N, 0, -1):
        G = np.einsum("ekl,nlq->nekq", o.Kt, D[i - 1], optimize=True)
        lamG = -np.einsum("nkp,nepq->nekq", lamD[i], Astar, optimize=True)
        lamD[i - 1] += np.einsum("ekl,nekq->nlq", o.Kt, lamG, optimize=True)
        lamA += -np.einsum("nekq,nkp->nepq", G, lamD[i], optimize=True)
        if i == 1:
            # damage-rate source of D^1 from the state at t_n
            uq0 = np.einsum("ql,nlp->nqp", o.Vv, Q, optimize=True)
            lr0 = np.einsum("q,qk,nk->nq", o.qv_w, o.Vv, lamD[1][:, :, 9], optimize=True)
            l0, gx, gc = rate_vjp(uq0, mat[:, None, :], lr0)
            g_xi0 += gx.sum(axis=1)
            g_cd += gc.sum(axis=1)
            lamD[0] += np.einsum("ql,nqp->nlp", o.Vv, l0, optimize=True)

    # 4./3. star matrices -> effective Lame parameters; the P speed of the Rusanov C
    lamB = np.einsum("ned,nepq->ndpq", o.Jinv, lamA, optimize=True)
    dBl, dBm = _lame_partials(rho)
    a_lam = np.einsum("ndpq,ndpq->n", lamB, dBl, optimize=True)
    a_mu = np.einsum("ndpq,ndpq->n", lamB, dBm, optimize=True)
    m2 = lam_eff + 2.0 * mu_eff
    live = m2 > 0.0
    dc = np.where(live, lam_cp / (2.0 * rho * np.where(live, cp, 1.0)), 0.0)
    a_lam += dc + a_lam_b
    a_mu += 2.0 * dc + a_mu_b
    # 2./1. effective Lame parameters at the cell mean ubar = phi_0 Q_0
    ubar = Q[:, 0, :] * PHI0
    lb, gx = lame_vjp(ubar, mat, a_lam, a_mu)
    g_xi0 += gx
    lamD[0][:, 0, :] += PHI0 * lb
    return lam + lamD[0], g_xi0, g_cd


def misfit(o, Q0, dt, n_steps, ref, t0=0.0):
    """J of a run and the receiver residuals r[k-1] = v_r(Q^k) - ref[k-1]."""
    Q, t = Q0, t0
    res = []
    for _ in range(n_steps):
        Q = o.step(Q, dt, t)
        t += dt
        res.append(o.sample_receivers(Q) - ref[len(res)])
    res = np.array(res)
    return 0.5 * dt * float(np.sum(res * res)), res


def misfit_gradient(o, Q0, dt, n_steps, ref, t0=0.0):
    """(J, dJ/dxi0 [E], dJ/dC_d [E], dJ/dQ^0 [E, L, 10]) of the receiver misfit
    against ref [n_steps, R, 3], every state of the run kept in memory."""
    states = [Q0]
    Q, t = Q0, t0
    res = []
    for k in range(n_steps):
        Q = o.step(Q, dt, t)
        t += dt
        states.append(Q)
        res.append(o.sample_receivers(Q) - ref[k])
    res = np.array(res)
    J = 0.5 * dt * float(np.sum(res * res))

    def seed(lam, k):
        for r, (e, phi) in enumerate(o.receivers):
            lam[e, :, 6:9] += dt * np.outer(phi, res[k - 1, r])

    lam = np.zeros_like(Q0)
    seed(lam, n_steps)
    gx = np.zeros(o.E)
    gc = np.zeros(o.E)
    for k in range(n_steps - 1, -1, -1):
        lam, a, b = step_vjp(o, states[k], dt, lam)
        gx += a
        gc += b
        if k >= 1:
            seed(lam, k)
    return J, gx, gc, lam
