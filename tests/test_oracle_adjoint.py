"""Pins of the oracle's discrete adjoint (oracle/adjoint.py, reading R21): the
derivative of each pointwise map against central differences of the forward
law, the adjoint of one step against central differences of Oracle.step along
random state and parameter directions (the dot-product test), the split
derivative of the Rusanov speed at a tie, and the gradient of the receiver
misfit against central differences of whole runs on the 384-tet cube,
element by element for xi0 and C_d."""
import numpy as np
import pytest

from oracle import Oracle, mode_list
from oracle.adjoint import flux_vjp, lame_vjp, misfit, misfit_gradient, rate_vjp, step_vjp, stress_vjp
from oracle.rheology import cdm_damage_rate, cdm_stress, effective_lame, flux
from synthetic import periodic_cube_mesh, workload_adjoint


def _points(n, seed):
    rng = np.random.default_rng(seed)
    mat = np.zeros((n, 6))
    mat[:] = (2700.0, 32e9, 32e9, 3.7e10, -0.8, 1e-5)
    mat[:, 4] = rng.uniform(-1.0, -0.6, n)
    u = np.zeros((n, 10))
    u[:, :6] = rng.normal(size=(n, 6)) * 1e-3
    u[:, 6:9] = rng.normal(size=(n, 3))
    u[:, 9] = rng.uniform(0.0, 0.3, n)
    return u, mat, rng


def _fd(f, u, p, h):
    up, um = u.copy(), u.copy()
    up[:, p] += h
    um[:, p] -= h
    return (f(up) - f(um)) / (2.0 * h)


def _close(a, b, rtol):
    assert np.abs(a - b).max() <= rtol * np.abs(b).max(), (np.abs(a - b).max(), np.abs(b).max())


def test_pointwise_derivatives():
    u, mat, rng = _points(40, 1)
    # stress: sum_ij Lambda_ij sigma_ij
    Ls = rng.normal(size=(40, 3, 3))
    g, gx = stress_vjp(u, mat, Ls)
    J = lambda uu, mm=mat: np.einsum("nij,nij->n", Ls, cdm_stress(uu, mm))
    for p in list(range(6)) + [9]:
        _close(g[:, p], _fd(J, u, p, 1e-9 if p < 6 else 1e-6), 1e-6)
    _close(gx, _fd(lambda m: J(u, m), mat, 4, 1e-6), 1e-6)
    # damage rate (no state of this sample sits within 1e-6 of the kink)
    lr = rng.normal(size=40)
    g, gx, gc = rate_vjp(u, mat, lr)
    R = lambda uu, mm=mat: lr * cdm_damage_rate(uu, mm)
    for p in range(6):
        _close(g[:, p], _fd(R, u, p, 1e-9), 1e-6)
    assert np.all(g[:, 6:] == 0.0)
    _close(gx, _fd(lambda m: R(u, m), mat, 4, 1e-6), 1e-6)
    _close(gc, _fd(lambda m: R(u, m), mat, 5, 1e-9), 1e-6)
    # effective Lame parameters at a cell mean
    al, am = rng.normal(size=40), rng.normal(size=40)
    g, gx = lame_vjp(u, mat, al, am)

    def lf(uu, mm=mat):
        lam, mu = effective_lame(uu, mm)
        return al * lam + am * mu
    for p in list(range(6)) + [9]:
        _close(g[:, p], _fd(lf, u, p, 1e-9 if p < 6 else 1e-6), 1e-6)
    _close(gx, _fd(lambda m: lf(u, m), mat, 4, 1e-6), 1e-6)
    # flux F^d_p
    LF = rng.normal(size=(40, 3, 10))
    g, gx = flux_vjp(u, mat, LF)
    Fl = lambda uu, mm=mat: np.einsum("ndp,ndp->n", LF, flux(uu, mm))
    for p in range(10):
        _close(g[:, p], _fd(Fl, u, p, 1e-9 if p < 6 else 1e-6), 1e-5)
    _close(gx, _fd(lambda m: Fl(u, m), mat, 4, 1e-6), 1e-6)


def _step_setup(N, seed, alpha_spread=True):
    rng = np.random.default_rng(seed)
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=3)
    E = mesh.n_elem
    mat = np.zeros((E, 6))
    mat[:] = (2700.0, 32e9, 32e9, 3.7e10, -0.8, 1e-5)
    if alpha_spread:
        mat[:, 1] *= rng.uniform(0.9, 1.1, E)
        mat[:, 4] = rng.uniform(-1.0, -0.6, E)
        mat[:, 5] = 10 ** rng.uniform(-6, -4, E)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat)
    deg = np.array([sum(m) for m in mode_list(N)])
    Q = rng.normal(size=(E, o.L, 10)) * (0.5 ** deg)[None, :, None]
    Q[..., :6] *= 1e-3
    Q[..., 6:9] *= 3.0
    Q[..., 9] *= 0.02 if alpha_spread else 0.0
    Q[:, 0, 9] = (0.05 + 0.05 * rng.uniform(size=E)) if alpha_spread else 0.0
    return mesh, mat, o, Q, 0.5 * o.cfl_dt(), rng


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_step_dot_product(N):
    """<lam, dQ^{k+1}> by central differences of Oracle.step equals
    <step_vjp(lam), dQ^k> along random state directions, and likewise for
    random xi0 and C_d directions."""
    mesh, mat, o, Q, dt, rng = _step_setup(N, 10 + N)
    lam = rng.normal(size=Q.shape)
    lQ, gx, gc = step_vjp(o, Q, dt, lam)
    for _ in range(2):
        d = rng.normal(size=Q.shape) * np.abs(Q).mean(axis=0, keepdims=True)
        h = 1e-6
        fd = np.sum(lam * (o.step(Q + h * d, dt) - o.step(Q - h * d, dt))) / (2 * h)
        assert abs(fd - np.sum(lQ * d)) <= 1e-7 * abs(fd), (fd, np.sum(lQ * d))
    for col, g, h in ((4, gx, 1e-6), (5, gc, 1e-12)):
        d = rng.normal(size=mesh.n_elem)
        step = np.outer(d, np.eye(6)[col]) * h
        o1 = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat + step)
        o2 = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat - step)
        fd = np.sum(lam * (o1.step(Q, dt) - o2.step(Q, dt))) / (2 * h)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd), (col, fd, np.sum(g * d))


def test_tied_speeds_split_the_derivative():
    """Homogeneous rock at alpha = 0: every cell has the same P speed, so C =
    max(cp-, cp+) sits on a tie at every face.  Splitting its derivative in
    halves reproduces the central difference along a direction that moves the
    cell-mean damage (and hence cp) of every cell."""
    mesh, mat, o, Q, dt, rng = _step_setup(2, 7, alpha_spread=False)
    lam = rng.normal(size=Q.shape)
    lQ, _, _ = step_vjp(o, Q, dt, lam)
    d = np.zeros_like(Q)
    d[:, 0, 9] = rng.uniform(0.5, 1.5, size=mesh.n_elem) * 0.01
    d[:, :, :6] = rng.normal(size=(mesh.n_elem, o.L, 6)) * 1e-4
    h = 1e-6
    fd = np.sum(lam * (o.step(Q + h * d, dt) - o.step(Q - h * d, dt))) / (2 * h)
    assert abs(fd - np.sum(lQ * d)) <= 1e-7 * abs(fd), (fd, np.sum(lQ * d))


def test_misfit_gradient_against_finite_differences():
    """The 384-tet jittered cube at N = 2 with damage on: the gradient of the
    misfit of 32 receivers over 3 steps, against a run with perturbed
    parameters, matches central differences of whole oracle runs for xi0 and
    C_d on 16 random elements and along a random initial-state direction."""
    w = workload_adjoint(n=4, order=2, steps=3)
    m = w["mesh"]
    N, ns = 2, 3
    mat, mref = w["material"], w["material_ref"]
    o = Oracle(m.elem_xyz, m.elem_vid, N, mat)
    oref = Oracle(m.elem_xyz, m.elem_vid, N, mref)
    rng = np.random.default_rng(21)
    deg = np.array([sum(mm) for mm in mode_list(N)])
    Q0 = rng.normal(size=(m.n_elem, o.L, 10)) * (0.5 ** deg)[None, :, None]
    Q0[..., :6] *= 2e-4
    Q0[..., 6:9] *= 0.6
    Q0[..., 9] = 0.0
    for oo in (o, oref):
        oo.set_receivers(w["receivers"])
    dt = 0.5 * o.cfl_dt()
    _, ref = oref.run(Q0, dt, ns, record=True)
    J, gx, gc, lq = misfit_gradient(o, Q0, dt, ns, ref)
    assert J > 0
    assert J == pytest.approx(misfit(o, Q0, dt, ns, ref)[0], rel=1e-14)
    els = rng.choice(m.n_elem, 16, replace=False)
    for col, g, rel_h in ((4, gx, 1e-5), (5, gc, 1e-3)):
        fd = []
        for e in els:
            h = rel_h * abs(mat[e, col])
            runs = []
            for sgn in (1.0, -1.0):
                mm = mat.copy()
                mm[e, col] += sgn * h
                oo = Oracle(m.elem_xyz, m.elem_vid, N, mm)
                oo.set_receivers(w["receivers"])
                runs.append(misfit(oo, Q0, dt, ns, ref)[0])
            fd.append((runs[0] - runs[1]) / (2 * h))
        fd = np.array(fd)
        assert np.count_nonzero(fd) >= 8
        assert np.abs(fd - g[els]).max() <= 1e-6 * np.abs(fd).max(), (col, fd, g[els])
    d = rng.normal(size=Q0.shape) * np.abs(Q0).mean(axis=0, keepdims=True)
    h = 1e-5
    fd = (misfit(o, Q0 + h * d, dt, ns, ref)[0] - misfit(o, Q0 - h * d, dt, ns, ref)[0]) / (2 * h)
    assert abs(fd - np.sum(lq * d)) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("N", [1, 2])
def test_step_dot_product_with_boundary_faces(N):
    """A closed jittered box with a free-surface top and absorbing sides: the
    step transpose, including the boundary fluxes' dependence on the effective
    Lame parameters of the cell mean, passes the dot-product test along random
    state, xi0 and C_d directions."""
    from synthetic.mesh import kuhn_box_mesh
    rng = np.random.default_rng(40 + N)
    g = np.linspace(0.0, 4000.0, 4)
    mesh = kuhn_box_mesh(g, g, g, periodic=(False, False, False), jitter=0.1, seed=3)
    E = mesh.n_elem
    mat = np.zeros((E, 6))
    mat[:] = (2700.0, 32e9, 32e9, 3.7e10, -0.8, 1e-5)
    mat[:, 1] *= rng.uniform(0.9, 1.1, E)
    mat[:, 4] = rng.uniform(-1.0, -0.6, E)
    mat[:, 5] = 10 ** rng.uniform(-6, -4, E)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, face_bc=mesh.face_bc)
    assert np.any(o.nbr < 0)
    deg = np.array([sum(m) for m in mode_list(N)])
    Q = rng.normal(size=(E, o.L, 10)) * (0.5 ** deg)[None, :, None]
    Q[..., :6] *= 1e-3
    Q[..., 6:9] *= 3.0
    Q[..., 9] *= 0.02
    Q[:, 0, 9] = 0.05 + 0.05 * rng.uniform(size=E)
    dt = 0.5 * o.cfl_dt()
    lam = rng.normal(size=Q.shape)
    lQ, gx, gc = step_vjp(o, Q, dt, lam)
    d = rng.normal(size=Q.shape) * np.abs(Q).mean(axis=0, keepdims=True)
    h = 1e-6
    fd = np.sum(lam * (o.step(Q + h * d, dt) - o.step(Q - h * d, dt))) / (2 * h)
    assert abs(fd - np.sum(lQ * d)) <= 1e-7 * abs(fd), (fd, np.sum(lQ * d))
    # the alpha cell means alone: the boundary matrices' dependence on lambda_eff, mu_eff
    d = np.zeros_like(Q)
    d[:, 0, 9] = rng.uniform(0.5, 1.5, size=E) * 0.01
    fd = np.sum(lam * (o.step(Q + h * d, dt) - o.step(Q - h * d, dt))) / (2 * h)
    assert abs(fd - np.sum(lQ * d)) <= 1e-6 * abs(fd), (fd, np.sum(lQ * d))
    for col, gg, hh in ((4, gx, 1e-6), (5, gc, 1e-12)):
        dd = rng.normal(size=E)
        step = np.outer(dd, np.eye(6)[col]) * hh
        o1 = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat + step, face_bc=mesh.face_bc)
        o2 = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat - step, face_bc=mesh.face_bc)
        fd = np.sum(lam * (o1.step(Q, dt) - o2.step(Q, dt))) / (2 * hh)
        assert abs(fd - np.sum(gg * dd)) <= 1e-6 * abs(fd), (col, fd, np.sum(gg * dd))


def test_misfit_gradient_with_boundary_faces():
    """The closed 162-tet box at N = 1 over 3 steps: the misfit gradient matches
    central differences of whole oracle runs on 8 random elements, for xi0 and
    C_d."""
    from synthetic.mesh import kuhn_box_mesh
    rng = np.random.default_rng(61)
    g = np.linspace(0.0, 4000.0, 4)
    mesh = kuhn_box_mesh(g, g, g, periodic=(False, False, False), jitter=0.1, seed=3)
    E, N, ns = mesh.n_elem, 1, 3
    w = workload_adjoint(n=3, order=N, steps=ns)
    mat, mref = w["material"].copy(), w["material_ref"].copy()
    rec = rng.uniform(400.0, 3600.0, size=(16, 3))
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, face_bc=mesh.face_bc)
    oref = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mref, face_bc=mesh.face_bc)
    for oo in (o, oref):
        oo.set_receivers(rec)
    deg = np.array([sum(mm) for mm in mode_list(N)])
    Q0 = rng.normal(size=(E, o.L, 10)) * (0.5 ** deg)[None, :, None]
    Q0[..., :6] *= 2e-4
    Q0[..., 6:9] *= 0.6
    Q0[..., 9] = 0.0
    Q0[:, 0, 9] = 0.05
    dt = 0.5 * o.cfl_dt()
    _, ref = oref.run(Q0, dt, ns, record=True)
    J, gx, gc, _ = misfit_gradient(o, Q0, dt, ns, ref)
    assert J > 0
    els = rng.choice(E, 8, replace=False)
    for col, gg, rel_h in ((4, gx, 1e-5), (5, gc, 1e-3)):
        fd = []
        for e in els:
            h = rel_h * abs(mat[e, col])
            runs = []
            for sgn in (1.0, -1.0):
                mm = mat.copy()
                mm[e, col] += sgn * h
                oo = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mm, face_bc=mesh.face_bc)
                oo.set_receivers(rec)
                runs.append(misfit(oo, Q0, dt, ns, ref)[0])
            fd.append((runs[0] - runs[1]) / (2 * h))
        fd = np.array(fd)
        assert np.count_nonzero(fd) >= 4
        assert np.abs(fd - gg[els]).max() <= 1e-6 * np.abs(fd).max(), (col, fd, gg[els])


def test_misfit_gradient_with_a_point_source():
    """Point sources add a state-independent term to each step and drop out of
    the adjoint: with the adjoint workload's dip-slip source active (its Ricker
    peak inside the 3 steps), the gradient still matches central differences of
    whole runs for xi0 and C_d on 8 random elements."""
    w = workload_adjoint(n=4, order=2, steps=3)
    m = w["mesh"]
    N, ns, t0 = 2, 3, 0.44
    mat, mref = w["material"], w["material_ref"]
    rng = np.random.default_rng(71)
    # two receivers beside the source: within 3 steps its effect spreads two face-hops only
    rec = np.vstack([w["receivers"][:16], [[2100.0, 2100.0, 2100.0], [1900.0, 2050.0, 2000.0]]])
    o = Oracle(m.elem_xyz, m.elem_vid, N, mat)
    oref = Oracle(m.elem_xyz, m.elem_vid, N, mref)
    for oo in (o, oref):
        oo.set_receivers(rec)
        oo.set_sources(w["sources"])
    deg = np.array([sum(mm) for mm in mode_list(N)])
    Q0 = rng.normal(size=(m.n_elem, o.L, 10)) * (0.5 ** deg)[None, :, None]
    Q0[..., :6] *= 2e-4
    Q0[..., 6:9] *= 0.6
    Q0[..., 9] = 0.0
    dt = 0.5 * o.cfl_dt()
    _, ref = oref.run(Q0, dt, ns, t0=t0, record=True)
    J, gx, gc, _ = misfit_gradient(o, Q0, dt, ns, ref, t0=t0)
    # the source changes the run: the misfit differs from the sourceless one
    o_free = Oracle(m.elem_xyz, m.elem_vid, N, mat)
    o_free.set_receivers(rec)
    assert abs(misfit(o_free, Q0, dt, ns, ref, t0=t0)[0] - J) > 1e-4 * J
    els = rng.choice(m.n_elem, 8, replace=False)
    for col, gg, rel_h in ((4, gx, 1e-5), (5, gc, 1e-3)):
        fd = []
        for e in els:
            h = rel_h * abs(mat[e, col])
            runs = []
            for sgn in (1.0, -1.0):
                mm = mat.copy()
                mm[e, col] += sgn * h
                oo = Oracle(m.elem_xyz, m.elem_vid, N, mm)
                oo.set_receivers(rec)
                oo.set_sources(w["sources"])
                runs.append(misfit(oo, Q0, dt, ns, ref, t0=t0)[0])
            fd.append((runs[0] - runs[1]) / (2 * h))
        fd = np.array(fd)
        assert np.count_nonzero(fd) >= 4
        assert np.abs(fd - gg[els]).max() <= 1e-6 * np.abs(fd).max(), (col, fd, gg[els])
