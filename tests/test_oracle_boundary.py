"""Pins of the oracle's boundary faces (Appendix A, "Free surface and absorbing
boundary conditions"): the eigen-decomposition and rotation matrices against
the flux Jacobians, the characteristic structure of both fluxes, a closed form
derived independently, zero traction on the free surface, and step-level
checks (rigid translation of a free body, a P pulse leaving through absorbing
faces, energy decay, an independent monomial-basis brute force)."""
import math

import numpy as np
import pytest

from oracle import MeshError, Oracle
from oracle.boundary import (absorbing_matrix, eigen_R, face_frame, free_surface_matrix,
                             free_surface_state, rotation_T)
from oracle.rheology import cdm_stress, jacobian_eff
from synthetic import rock_material
from synthetic.mesh import FACE_BC_ABSORBING, FACE_BC_FREE_SURFACE, kuhn_box_mesh

from bruteforce import BruteForce, boundary_flux_closed_form

RHO, LAM, MU = 2700.0, 32e9, 32e9
CP = math.sqrt((LAM + 2 * MU) / RHO)


def _random_media(rng, k=6):
    out = []
    for _ in range(k):
        rho = rng.uniform(1500.0, 3000.0)
        mu = rng.uniform(1e9, 4e10)
        lam = rng.uniform(-0.5 * mu, 3 * mu)          # lambda + 2 mu > 0, lambda may be negative
        out.append((lam, mu, rho))
    return out


def _random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _random_state(rng, scale_v=1.0):
    u = rng.normal(size=10) * np.array([1e-4] * 6 + [scale_v] * 3 + [0.3])
    return u


def test_R_diagonalises_B1():
    """B^{1,eff} R = R Lambda with R invertible: every printed eigenvector column
    (with the c_s reading of the second printed speed) is an eigenvector."""
    rng = np.random.default_rng(1)
    for lam, mu, rho in _random_media(rng):
        B1 = jacobian_eff(np.array(lam), np.array(mu), np.array(rho))[0]
        R, L = eigen_R(lam, mu, rho)
        scale = np.abs(B1 @ R).max()
        assert np.abs(B1 @ R - R * L[None, :]).max() <= 1e-13 * scale
        assert abs(np.linalg.det(R)) > 1e-6


def test_T_rotates_strain_and_velocity():
    """T maps a face-aligned state to the global one as Q eps' Q^T and Q v', and
    the frame of the transposed rotation inverts it."""
    rng = np.random.default_rng(2)
    sym = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))
    for _ in range(5):
        n, s, t = face_frame(_random_unit(rng))
        Q = np.stack([n, s, t], axis=1)
        assert np.allclose(Q.T @ Q, np.eye(3), atol=1e-14)
        up = rng.normal(size=10)
        Ep = np.array([[up[0], up[3], up[5]], [up[3], up[1], up[4]], [up[5], up[4], up[2]]])
        Eg = Q @ Ep @ Q.T
        ug = rotation_T(n, s, t) @ up
        for p, (i, j) in enumerate(sym):
            assert ug[p] == pytest.approx(Eg[i, j], abs=1e-13)
        assert np.allclose(ug[6:9], Q @ up[6:9], atol=1e-14)
        assert ug[9] == up[9]
        Tinv = rotation_T(Q[0], Q[1], Q[2])
        assert np.allclose(Tinv @ rotation_T(n, s, t), np.eye(10), atol=1e-13)


def test_rotated_jacobian_is_the_normal_jacobian():
    """Rotational invariance of the isotropic flux: T B^1 T^{-1} = sum_d n_d B^d
    for any outward normal (ties T to the Jacobians built from the flux)."""
    rng = np.random.default_rng(3)
    for lam, mu, rho in _random_media(rng, 3):
        B = jacobian_eff(np.array(lam), np.array(mu), np.array(rho))
        for _ in range(4):
            n = _random_unit(rng)
            T = rotation_T(*face_frame(n))
            lhs = T @ B[0] @ np.linalg.inv(T)
            rhs = np.einsum("d,dpq->pq", n, B)
            assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


def test_absorbing_keeps_only_outgoing_characteristics():
    """For a state along one characteristic: the absorbing flux is the full
    normal flux c u on an outgoing (c > 0) one and zero otherwise; and it does
    not depend on the choice of tangent vectors."""
    rng = np.random.default_rng(4)
    for lam, mu, rho in _random_media(rng, 3):
        B = jacobian_eff(np.array(lam), np.array(mu), np.array(rho))
        R, L = eigen_R(lam, mu, rho)
        n = _random_unit(rng)
        T = rotation_T(*face_frame(n))
        Mabs = absorbing_matrix(n, lam, mu, rho)
        Bn = np.einsum("d,dpq->pq", n, B)
        for k in range(10):
            u = T @ R[:, k]
            F = Mabs @ u
            if L[k] > 0:
                assert np.allclose(F, Bn @ u, rtol=1e-12, atol=1e-12 * np.abs(Bn @ u).max())
                assert np.allclose(F, L[k] * u, rtol=1e-12, atol=1e-12 * L[k] * np.abs(u).max())
            else:
                assert np.abs(F).max() <= 1e-12 * np.abs(Bn).max() * np.abs(u).max()
        # another tangent pair (rotated about n) gives the same matrix
        _, s, t = face_frame(n)
        th = rng.uniform(0, 2 * np.pi)
        s2, t2 = math.cos(th) * s + math.sin(th) * t, -math.sin(th) * s + math.cos(th) * t
        T2 = rotation_T(n, s2, t2)
        lp = np.diag(np.maximum(L, 0.0))
        M2 = T2 @ R @ lp @ np.linalg.inv(R) @ np.linalg.inv(T2)
        assert np.abs(M2 - Mabs).max() <= 1e-12 * np.abs(Mabs).max()


def test_free_surface_state_is_traction_free():
    """The free-surface boundary state has zero traction sigma(u^b) n (stress from
    the effective Hooke law, evaluated in global coordinates), differs from u^-
    only along the three incoming characteristics, leaves a traction-free state
    unchanged, and the flux is the physical normal flux of u^b, with no velocity
    component."""
    rng = np.random.default_rng(5)
    for lam, mu, rho in _random_media(rng, 4):
        B = jacobian_eff(np.array(lam), np.array(mu), np.array(rho))
        R, L = eigen_R(lam, mu, rho)
        for _ in range(3):
            n = _random_unit(rng)
            S = free_surface_state(n, lam, mu, rho)
            M = free_surface_matrix(n, lam, mu, rho)
            T = rotation_T(*face_frame(n))
            u = _random_state(rng)
            ub = S @ u
            # effective Hooke law (no damage term): material with alpha = 0 and the effective moduli
            mat = np.array([rho, lam, mu, 0.0, 0.0, 0.0])
            sig = cdm_stress(ub, mat)
            tr = sig @ n
            assert np.abs(tr).max() <= 1e-12 * np.abs(cdm_stress(u, mat)).max()
            amp = np.linalg.solve(R, np.linalg.inv(T) @ (ub - u))
            assert np.abs(amp[3:]).max() <= 1e-12 * np.abs(amp).max()
            assert np.all(L[:3] < 0)
            F = M @ u
            Bn = np.einsum("d,dpq->pq", n, B)
            bound = 1e-12 * (np.abs(Bn) @ np.abs(ub) + np.abs(M) @ np.abs(u))   # per-entry rounding scale
            assert np.all(np.abs(F - Bn @ ub) <= bound)
            assert np.all(np.abs(F[6:9]) <= bound[6:9])
            # a traction-free state is its own boundary state
            assert np.allclose(S @ ub, ub, rtol=1e-12, atol=1e-12 * np.abs(ub).max())


@pytest.mark.parametrize("bc", [FACE_BC_FREE_SURFACE, FACE_BC_ABSORBING])
def test_boundary_matrix_matches_closed_form(bc):
    """The oracle's literal T R Lambda^+ R^{-1} T^{-1} / omega-solve matrices
    agree with the closed-form characteristic flux derived in global
    coordinates (tests/bruteforce.py) for random states, normals and media."""
    rng = np.random.default_rng(6 + bc)
    for lam, mu, rho in _random_media(rng, 4):
        for _ in range(3):
            n = _random_unit(rng)
            M = (free_surface_matrix if bc == FACE_BC_FREE_SURFACE else absorbing_matrix)(n, lam, mu, rho)
            u = _random_state(rng, scale_v=math.sqrt(mu / rho) * 1e-4)
            ref = boundary_flux_closed_form(bc, u, n, lam, mu, rho)
            assert np.abs(ref).max() > 0
            # rounding scale per entry: the size of the terms of the physical normal flux
            Bn = np.einsum("d,dpq->pq", n, jacobian_eff(np.array(lam), np.array(mu), np.array(rho)))
            assert np.all(np.abs(M @ u - ref) <= 1e-12 * (np.abs(Bn) @ np.abs(u)))


def _box(n=2, periodic=(False, False, False), top=FACE_BC_FREE_SURFACE, side=FACE_BC_ABSORBING,
         jitter=0.1, seed=3, lengths=(4000.0, 4000.0, 4000.0), cells=None):
    cells = cells or (n, n, n)
    grids = [np.linspace(0.0, Lx, c + 1) for Lx, c in zip(lengths, cells)]
    return kuhn_box_mesh(*grids, periodic=periodic, jitter=jitter, seed=seed, top_bc=top, side_bc=side)


def test_mesh_tags_and_matching():
    """Every boundary face of a closed box is tagged and unmatched, every
    interior face is matched once; a tag on a shared face is an error."""
    mesh = _box()
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, 1, rock_material(mesh.n_elem), face_bc=mesh.face_bc)
    tagged = o.face_bc != 0
    assert np.all((o.nbr < 0) == tagged)
    assert tagged.sum() == 6 * 2 * mesh.cells[0] * mesh.cells[1]
    bad = mesh.face_bc.copy()
    e, f = np.argwhere(mesh.face_bc == 0)[0]
    bad[e, f] = FACE_BC_ABSORBING
    with pytest.raises(MeshError):
        Oracle(mesh.elem_xyz, mesh.elem_vid, 1, rock_material(mesh.n_elem), face_bc=bad)
    with pytest.raises(MeshError):
        Oracle(mesh.elem_xyz, mesh.elem_vid, 1, rock_material(mesh.n_elem))   # outer faces untagged


def test_rigid_translation_of_a_free_body():
    """A uniformly moving, unstrained body with free surfaces everywhere is an
    exact steady state (zero traction on every face); the step keeps it to
    rounding, damage on."""
    mesh = _box(top=FACE_BC_FREE_SURFACE, side=FACE_BC_FREE_SURFACE)
    mat = rock_material(mesh.n_elem, cd=1e-4)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, 2, mat, face_bc=mesh.face_bc)
    v = np.array([0.3, -0.2, 0.5])

    def const(x):
        u = np.zeros(x.shape[:-1] + (10,))
        u[..., 6:9] = v
        u[..., 9] = 0.1
        return u
    Q0 = o.project(const)
    Q = Q0
    dt = o.cfl_dt()
    for _ in range(3):
        Q = o.step(Q, dt)
    assert np.abs(Q - Q0).max() <= 1e-13 * np.abs(Q0).max()


def _pulse_run(bc_x):
    """Right-going Gaussian P pulse along x in a slab periodic in y and z, with
    faces normal to x tagged bc_x; returns (energy before, energy after the
    pulse would have left the slab)."""
    Lx = 4000.0
    mesh = _box(periodic=(False, True, True), side=bc_x, top=bc_x, cells=(8, 3, 3),
                lengths=(Lx, 1500.0, 1500.0), jitter=0.1, seed=7)
    mat = rock_material(mesh.n_elem, cd=0.0)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, 1, mat, face_bc=mesh.face_bc)
    A, x0, w = 1e-4, 1500.0, 400.0

    def pulse(x):
        g = A * np.exp(-((x[..., 0] - x0) / w) ** 2)
        u = np.zeros(x.shape[:-1] + (10,))
        u[..., 0] = g
        u[..., 6] = -CP * g
        return u
    Q = o.project(pulse)
    E0 = o.energy(Q)
    dt = o.cfl_dt()
    T = (Lx - x0 + 3 * w) / CP
    n = int(math.ceil(T / dt))
    for _ in range(n):
        Q = o.step(Q, T / n)
    return E0, o.energy(Q)


def test_absorbing_faces_let_a_pulse_leave():
    """A P pulse travelling along x leaves through absorbing faces: after the
    travel time almost no energy is left (reflections only at discretisation
    level), while free-surface faces keep the energy in the slab."""
    E0, E1 = _pulse_run(FACE_BC_ABSORBING)
    assert E1 < 1e-3 * E0, E1 / E0
    F0, F1 = _pulse_run(FACE_BC_FREE_SURFACE)
    assert F1 > 0.5 * F0, F1 / F0


def test_energy_does_not_grow_with_boundaries():
    """Damage off, free top and absorbing sides: the discrete energy is
    non-increasing from step to step (both boundary fluxes dissipate or
    conserve)."""
    mesh = _box(n=2)
    mat = rock_material(mesh.n_elem, cd=0.0)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, 2, mat, face_bc=mesh.face_bc)
    rng = np.random.default_rng(8)
    coef = rng.normal(size=(4, 10))

    def field(x):
        y = x / 4000.0
        mono = np.stack([np.ones_like(y[..., 0]), y[..., 0], y[..., 1], y[..., 2]], axis=-1)
        return mono @ coef * np.array([1e-4] * 6 + [1e-4 * CP] * 3 + [0.0])
    Q = o.project(field)
    dt = o.cfl_dt()
    E = [o.energy(Q)]
    for _ in range(6):
        Q = o.step(Q, dt)
        E.append(o.energy(Q))
    assert all(E[i + 1] <= E[i] * (1 + 1e-12) for i in range(len(E) - 1)), E


@pytest.mark.parametrize("N,damage", [(1, True), (2, False), (2, True)])
def test_bruteforce_step_with_boundaries(N, damage):
    """P4 with boundary faces: one oracle step on a closed box (free top,
    absorbing sides) equals the monomial-basis brute force, whose boundary flux
    is the closed form instead of the rotation/eigenvector matrices."""
    mesh = _box(n=2, jitter=0.1, seed=13)
    mat = rock_material(mesh.n_elem, cd=1e-4 if damage else 0.0)
    rng = np.random.default_rng(17)
    coef = rng.normal(size=(mesh.n_elem, 4, 10))
    centers = mesh.elem_xyz.mean(axis=1)
    scale = np.array([1e-4] * 6 + [1e-4 * CP] * 3 + [0.2 if damage else 0.0])

    def one(e, x):
        y = (x - centers[e]) / 2000.0
        mono = np.stack([np.ones_like(y[:, 0]), y[:, 0], y[:, 1], y[:, 2]], axis=-1)
        u = (mono @ coef[e]) * scale
        u[:, 9] = 0.5 * scale[9] + 0.25 * u[:, 9]
        return u

    def every(x):
        return np.stack([one(e, x[e]) for e in range(mesh.n_elem)])
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, face_bc=mesh.face_bc)
    box = np.where(np.array(mesh.periodic), mesh.extent, 1e3 * mesh.extent)
    bf = BruteForce(mesh.elem_xyz, mesh.elem_vid, N, mat, box, face_bc=mesh.face_bc)
    Q0, C0 = o.project(every), bf.project(one)
    dt = 0.8 * o.cfl_dt()
    Q1, C1 = o.step(Q0, dt), bf.step(C0, dt)
    pts = np.random.default_rng(9)
    errs, norms = [], []
    for e in range(mesh.n_elem):
        x = pts.dirichlet(np.ones(4), size=4) @ mesh.elem_xyz[e]
        errs.append(np.abs(o.evaluate_at(Q1, e, x) - bf.evaluate(C1, e, x)).max(axis=0))
        norms.append(np.abs(bf.evaluate(C1, e, x) - bf.evaluate(C0, e, x)).max(axis=0))
    errs, norms = np.max(errs, axis=0), np.max(norms, axis=0)
    for p in range(10):
        if norms[p] > 0:
            assert errs[p] <= 1e-9 * norms[p] + 1e-15, (p, errs[p], norms[p])
