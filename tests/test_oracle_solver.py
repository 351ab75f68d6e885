"""Step-level pins of the FP64 oracle (P1-P5, P7): design-order convergence on
the elastic plane wave, the closed-form uniform-strain damage growth, energy
decay, agreement with an independent monomial-basis brute force, invariance
under relabelling / vertex order / rotation / translation, monotone damage."""
import math

import numpy as np
import pytest

from oracle import MeshError, Oracle
from synthetic import periodic_cube_mesh, rock_material
from synthetic.mesh import Mesh

from bruteforce import BruteForce

RHO, LAM, MU = 2700.0, 32e9, 32e9
CP = math.sqrt((LAM + 2 * MU) / RHO)
CS = math.sqrt(MU / RHO)


def plane_wave(kind, kvec, A):
    """Exact travelling plane wave of linear elasticity: u(x,t) = A r sin(k.x - c|k| t)."""
    kvec = np.asarray(kvec, float)
    kn = np.linalg.norm(kvec)
    n = kvec / kn
    if kind == "P":
        c, pol = CP, n
    else:
        c = CS
        pol = np.cross(n, [0.0, 0.0, 1.0])
        pol /= np.linalg.norm(pol)
    eps = 0.5 * (np.outer(n, pol) + np.outer(pol, n))

    def f(x, t):
        ph = np.sin(x @ kvec - c * kn * t)
        u = np.zeros(x.shape[:-1] + (10,))
        for p, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))):
            u[..., p] = A * eps[i, j] * ph
        u[..., 6:9] = -c * A * ph[..., None] * pol
        return u
    return f


def _rel_err(o, Q, Qex):
    w = o.detJ[:, None, None]
    return math.sqrt(np.sum(w * (Q - Qex) ** 2) / np.sum(w * Qex ** 2))


def _plane_wave_error(n, N, kind, kvec, T=0.12):
    mesh = periodic_cube_mesh(n, 4000.0)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, rock_material(mesh.n_elem, cd=0.0))
    f = plane_wave(kind, kvec, 1e-4)
    Q = o.project(lambda x: f(x, 0.0))
    ns = int(math.ceil(T / o.cfl_dt()))
    Q = o.run(Q, T / ns, ns)
    return _rel_err(o, Q, o.project(lambda x: f(x, T)))


@pytest.mark.parametrize("N,kind,kvec", [
    (1, "P", (2 * math.pi / 4000, 0, 0)),
    (2, "P", (2 * math.pi / 4000, 0, 0)),
    (2, "S", (2 * math.pi / 4000, 0, 0)),
    (1, "P", (2 * math.pi / 4000, 2 * math.pi / 4000, 0)),
])
def test_P1_plane_wave_design_order(N, kind, kvec):
    """P1: damage off, the error against the exact plane wave falls at order
    >= N+1-0.3 from 3^3 to 6^3 cells (design order of linear ADER-DG)."""
    e3 = _plane_wave_error(3, N, kind, kvec)
    e6 = _plane_wave_error(6, N, kind, kvec)
    order = math.log(e3 / e6) / math.log(2.0)
    assert order >= N + 1 - 0.3, (e3, e6, order)
    assert e6 < 0.1


@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("state", ["uniaxial_ext", "uniaxial_comp", "pure_shear", "iso_comp", "mixed"])
def test_P2_uniform_strain_damage_is_linear_in_time(N, state):
    """P2: a uniform strain with v = 0 is a steady state of the fluxes; alpha
    grows exactly linearly at the pointwise rate, whatever the mesh jitter."""
    e = 1e-3
    eps = {"uniaxial_ext": (e, 0, 0, 0, 0, 0), "uniaxial_comp": (-e, 0, 0, 0, 0, 0),
           "pure_shear": (0, 0, 0, e, 0, 0), "iso_comp": (-e, -e, -e, 0, 0, 0),
           "mixed": (e, -0.3 * e, 0.2 * e, 0.4 * e, -0.1 * e, 0.25 * e)}[state]
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=7)
    mat = rock_material(mesh.n_elem)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat)
    alpha0 = 0.05
    u0 = np.array(list(eps) + [0, 0, 0, alpha0])
    Q = o.project(lambda x: np.broadcast_to(u0, x.shape[:-1] + (10,)).copy())
    dt, n = 2e-3, 6
    Q = o.run(Q, dt, n)
    # hand-derived rate: Cd gamma_r max(0, I1 sqrt(I2) - xi0 I2)
    exx, eyy, ezz, exy, eyz, ezx = eps
    I1 = exx + eyy + ezz
    I2 = exx ** 2 + eyy ** 2 + ezz ** 2 + 2 * (exy ** 2 + eyz ** 2 + ezx ** 2)
    rate = 1e-4 * 3.7e10 * max(0.0, I1 * math.sqrt(I2) + 0.8 * I2)
    mean = Q[:, 0, :] * math.sqrt(6.0)
    np.testing.assert_allclose(mean[:, 9], alpha0 + rate * dt * n, rtol=1e-12)
    np.testing.assert_allclose(mean[:, :6], np.broadcast_to(eps, (mesh.n_elem, 6)), rtol=1e-11, atol=1e-17)
    assert np.abs(mean[:, 6:9]).max() < 1e-14
    assert np.abs(Q[:, 1:, :]).max() < 1e-12 * max(1.0, rate)


def test_P3_energy_decays_without_damage():
    """P3: the Rusanov flux is dissipative; with damage off the discrete energy
    never grows, and the loss shrinks under refinement."""
    losses = []
    for n in (3, 6):
        mesh = periodic_cube_mesh(n, 4000.0, jitter=0.1, seed=3)
        o = Oracle(mesh.elem_xyz, mesh.elem_vid, 2, rock_material(mesh.n_elem, cd=0.0))
        f = plane_wave("P", (2 * math.pi / 4000, 2 * math.pi / 4000, 0), 1e-4)
        Q = o.project(lambda x: f(x, 0.0))
        dt = o.cfl_dt()
        E = [o.energy(Q)]
        for _ in range(int(0.06 / dt) + 1):
            Q = o.step(Q, dt)
            E.append(o.energy(Q))
        E = np.array(E)
        assert np.all(np.diff(E) <= 1e-12 * E[0])
        losses.append((E[0] - E[-1]) / E[0])
    assert losses[1] < 0.25 * losses[0]


def _random_poly_state(mesh, N, seed, alpha_scale=0.2):
    """Per-element random polynomials of degree N (discontinuous across faces).
    Returns (all_elements(x[E,q,3]) -> [E,q,10], one_element(e, x[q,3]) -> [q,10])."""
    rng = np.random.default_rng(seed)
    exps = [(a, b, d - a - b) for d in range(N + 1) for a in range(d + 1) for b in range(d + 1 - a)]
    coef = rng.normal(size=(mesh.n_elem, len(exps), 10))
    scale = np.array([1e-4] * 6 + [1e-4 * CP] * 3 + [alpha_scale])
    centers = mesh.elem_xyz.mean(axis=1)
    h = 4000.0 / mesh.cells[0]

    def one(e, x):
        y = (x - centers[e]) / h
        mono = np.stack([y[:, 0] ** a * y[:, 1] ** b * y[:, 2] ** c for a, b, c in exps], axis=-1)
        u = (mono @ coef[e]) * scale
        u[:, 9] = 0.5 * alpha_scale + 0.25 * u[:, 9]
        return u

    def every(x):
        return np.stack([one(e, x[e]) for e in range(mesh.n_elem)])
    return every, one


@pytest.mark.parametrize("N,damage", [(1, False), (1, True), (2, True)])
def test_P4_bruteforce_monomial_step(N, damage):
    """P4: one step of the oracle equals one step re-derived with a monomial
    basis in physical coordinates, exact integrals and geometric neighbour
    search, to ~1e-11 relative (same space-time nodes for nonlinear terms)."""
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=11)
    mat = rock_material(mesh.n_elem, cd=1e-4 if damage else 0.0)
    every, one = _random_poly_state(mesh, N, seed=5, alpha_scale=0.2 if damage else 0.0)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat)
    Q0 = o.project(every)
    bf = BruteForce(mesh.elem_xyz, mesh.elem_vid, N, mat, mesh.extent)
    C0 = bf.project(one)
    dt = 0.8 * o.cfl_dt()
    Q1 = o.step(Q0, dt)
    C1 = bf.step(C0, dt)
    rng = np.random.default_rng(9)
    errs, norms = [], []
    for e in range(0, mesh.n_elem, 7):
        bary = rng.dirichlet(np.ones(4), size=6)
        x = bary @ mesh.elem_xyz[e]
        uo = o.evaluate_at(Q1, e, x)
        ub = bf.evaluate(C1, e, x)
        u0 = bf.evaluate(C0, e, x)
        errs.append(np.abs(uo - ub).max(axis=0))
        norms.append(np.abs(ub - u0).max(axis=0))
    errs, norms = np.max(errs, axis=0), np.max(norms, axis=0)
    # the change over the step is matched to 1e-9 of its size in every field
    for p in range(10):
        if norms[p] > 0:
            assert errs[p] <= 1e-9 * norms[p] + 1e-15, (p, errs[p], norms[p])


def test_P5_relabelling_and_vertex_order_invariance():
    """P5: relabelling elements and reordering each element's input vertices
    gives the same fields at the same physical points, with damage off and on
    (the reference map follows the vertex ids, reading R15)."""
    base = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=21)
    rng = np.random.default_rng(1)
    perm = rng.permutation(base.n_elem)
    vperm = np.array([rng.permutation(4) for _ in range(base.n_elem)])
    coef = np.random.default_rng(2).normal(size=(10, 10))

    def poly(x):
        # a global quadratic field (projected exactly by any rule of degree >= 4)
        y = x / 4000.0
        mono = np.stack([np.ones_like(y[..., 0]), y[..., 0], y[..., 1], y[..., 2], y[..., 0] ** 2,
                         y[..., 1] ** 2, y[..., 2] ** 2, y[..., 0] * y[..., 1], y[..., 1] * y[..., 2],
                         y[..., 2] * y[..., 0]], axis=-1)
        return mono @ coef * np.array([1e-4] * 6 + [1e-4 * CP] * 3 + [0.0])
    for damage, vertex_too in ((False, True), (True, True)):
        mat = rock_material(base.n_elem, cd=1e-4 if damage else 0.0)
        pm = base.permuted(elem_perm=perm, vertex_perm=vperm if vertex_too else None)
        res = []
        for mesh, m in ((base, mat), (pm, mat[perm])):
            o = Oracle(mesh.elem_xyz, mesh.elem_vid, 2, m)

            def ic(x, damage=damage):
                u = poly(x)
                u[..., 9] = 0.1 if damage else 0.0     # alpha > 0 makes the law nonlinear
                return u
            Q = o.project(ic)
            dt = 2e-3
            Q = o.run(Q, dt, 3)
            res.append((o, mesh, Q))
        (o0, m0, Q0), (o1, m1, Q1) = res
        # same physical sample points: barycentric coords follow the vertex permutation
        rngs = np.random.default_rng(0)
        bary = rngs.dirichlet(np.ones(4), size=5)
        for new in range(0, base.n_elem, 5):
            old = perm[new]
            x = bary @ base.elem_xyz[old]
            a = o0.evaluate_at(Q0, old, x)
            b = o1.evaluate_at(Q1, new, x)
            np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-12 * np.abs(a).max())


def test_P5_rotation_and_translation_invariance():
    """P5: rotating mesh and initial state rotates the fields (isotropic law,
    damage on); translating by a lattice vector changes nothing."""
    base = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=22)
    mat = rock_material(base.n_elem)
    f = plane_wave("S", (2 * math.pi / 4000, 0, 0), 1e-4)

    def ic(x):
        u = f(x, 0.0) * 10.0
        u[..., 0] += 3e-4          # pre-strain drives damage
        u[..., 9] = 0.05
        return u
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, math.cos(0.4), -math.sin(0.4)], [0, math.sin(0.4), math.cos(0.4)]])
    sym = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))

    def rot_u(u):
        eps = np.zeros(u.shape[:-1] + (3, 3))
        for p, (i, j) in enumerate(sym):
            eps[..., i, j] = eps[..., j, i] = u[..., p]
        er = np.einsum("ab,...bc,dc->...ad", R, eps, R)
        out = u.copy()
        for p, (i, j) in enumerate(sym):
            out[..., p] = er[..., i, j]
        out[..., 6:9] = u[..., 6:9] @ R.T
        return out

    o0 = Oracle(base.elem_xyz, base.elem_vid, 2, mat)
    Q0 = o0.run(o0.project(ic), 2e-3, 3)
    rot = Mesh(base.elem_xyz @ R.T, base.elem_vid, base.face_bc, base.cells, base.periodic, base.extent)
    o1 = Oracle(rot.elem_xyz, rot.elem_vid, 2, mat)
    Q1 = o1.run(o1.project(lambda x: rot_u(ic(x @ R))), 2e-3, 3)
    shift = base.elem_xyz + np.array([4000.0, -8000.0, 4000.0])
    o2 = Oracle(shift, base.elem_vid, 2, mat)
    Q2 = o2.run(o2.project(lambda x: ic(x - np.array([4000.0, -8000.0, 4000.0]))), 2e-3, 3)
    pts = np.random.default_rng(3).dirichlet(np.ones(4), size=4)[:, 1:]
    a = o0.evaluate(Q0, pts)
    b = o1.evaluate(Q1, pts)
    c = o2.evaluate(Q2, pts)
    scale = np.abs(a).max(axis=(0, 1))
    ra = rot_u(a)
    for group in (slice(0, 6), slice(6, 9), slice(9, 10)):
        tol = 1e-10 * np.abs(ra[..., group]).max()
        np.testing.assert_allclose(b[..., group], ra[..., group], rtol=0, atol=tol)
    np.testing.assert_allclose(c, a, rtol=1e-10, atol=1e-14)


def test_P7_cell_mean_damage_is_monotone():
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=4)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, 2, rock_material(mesh.n_elem))
    f = plane_wave("P", (2 * math.pi / 4000, 0, 0), 1e-3)
    Q = o.project(lambda x: f(x, 0.0))
    prev = Q[:, 0, 9].copy()
    for _ in range(5):
        Q = o.step(Q, 3e-3)
        assert np.all(Q[:, 0, 9] >= prev - 1e-18)
        prev = Q[:, 0, 9].copy()
    assert prev.max() > 0


def test_mesh_errors_are_reported():
    mesh = periodic_cube_mesh(3, 4000.0)
    bad = mesh.elem_vid.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(MeshError):
        Oracle(mesh.elem_xyz, bad, 1, rock_material(mesh.n_elem))
    flat = mesh.elem_xyz.copy()
    flat[0, 3] = flat[0, 0] + 0.5 * (flat[0, 1] - flat[0, 0]) + 0.5 * (flat[0, 2] - flat[0, 0])
    with pytest.raises(MeshError):
        Oracle(flat, mesh.elem_vid, 1, rock_material(mesh.n_elem))
