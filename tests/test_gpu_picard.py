"""GPU checks of the Picard predictor (reading R20): parity with the oracle's
Picard predictor at degrees 1..4 under the CDM with damage and under the other
two laws, the linear fixed point, and the restored order on the smooth
nonlinear simple wave of the shear law, against the CK predictor's first order."""
import math

import numpy as np
import pytest

from oracle import Oracle, from_abi, mode_list, tet_rule, to_abi
from oracle.riemann import ShearSimpleWave
from synthetic import kuhn_box_mesh, periodic_cube_mesh

from parity_util import TOL_ALPHA, TOL_REL_L2, alpha_max_diff, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    dgpkg.load_library()


def _material(law, E, rng):
    mat = np.zeros((E, 6))
    mat[:, 0] = 2700.0 * rng.uniform(0.9, 1.1, size=E)
    mat[:, 1] = 30e9 * rng.uniform(0.9, 1.1, size=E)
    mat[:, 2] = 32e9 * rng.uniform(0.9, 1.1, size=E)
    if law == "cdm":
        mat[:, 3] = 3.7e10 * rng.uniform(0.9, 1.1, size=E)
        mat[:, 4] = -0.8
        # alpha grows by ~1e-2 over the run, so the cells stay hyperbolic
        mat[:, 5] = 2e-6 * rng.uniform(0.5, 1.5, size=E)
    elif law == "ivm":
        mat[:, 3] = 1e5 * rng.uniform(0.5, 2.0, size=E)
        mat[:, 4] = 1.0 * rng.uniform(0.5, 2.0, size=E)
    else:
        mat[:, 3] = 10.0 * rng.uniform(0.5, 1.5, size=E)
    return mat


def _rough_state(E, N, seed, strain=3e-4, alpha=0.1):
    rng = np.random.default_rng(seed)
    deg = np.array([sum(m) for m in mode_list(N)])
    Q = rng.normal(size=(E, len(deg), 10)) * (0.5 ** deg)[None, :, None]
    Q[..., :6] *= strain
    Q[..., 6:9] *= strain * 1800.0
    Q[..., 9] *= 0.2 * alpha
    Q[:, 0, 9] = alpha / math.sqrt(6.0) + np.abs(Q[:, 0, 9])
    return Q


@pytest.mark.parametrize("N,law", [(1, "cdm"), (2, "cdm"), (3, "cdm"), (4, "cdm"), (3, "ivm"), (3, "nlshear")])
def test_picard_parity(N, law):
    import paper_2502_09714_gb300 as dgpkg
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=44)
    rng = np.random.default_rng(30 + N)
    mesh = mesh.permuted(vertex_perm=np.array([rng.permutation(4) for _ in range(mesh.n_elem)]))
    mat = _material(law, mesh.n_elem, rng)
    Q0 = _rough_state(mesh.n_elem, N, seed=600 + N, strain=3e-3 if law == "nlshear" else 3e-4)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, law=law, picard_iterations=N)
    dt = 0.5 * o.cfl_dt()
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, law=law)
    s.set_material(mat)
    s.set_predictor("picard", N)
    s.set_state(to_abi(Q0))
    s.step(3, dt)
    q, _ = s.get_state()
    Q = o.run(Q0, dt, 3)
    errs = rel_l2(to_abi(from_abi(q) - Q0), Q - Q0, o.detJ)
    for name, e in errs.items():
        assert e <= TOL_REL_L2, (name, e)
    assert alpha_max_diff(q, Q, N) <= TOL_ALPHA


def test_picard_linear_fixed_point():
    """beta = 0: the CK coefficients are the fixed point, so the GPU's Picard
    run equals its CK run up to FP32 rounding."""
    import paper_2502_09714_gb300 as dgpkg
    N = 3
    mesh = periodic_cube_mesh(3, 1.0, jitter=0.1, seed=5)
    mat = np.zeros((mesh.n_elem, 6))
    mat[:, :4] = (1.0, 1.0, 1.0, 0.0)
    Q0 = _rough_state(mesh.n_elem, N, seed=7, strain=1e-3)
    Q0[..., 9] = 0.0
    dt = 0.5 * Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, law="nlshear").cfl_dt()
    out = []
    for kind in ("ck", "picard"):
        s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, law="nlshear")
        s.set_material(mat)
        s.set_predictor(kind, 3 if kind == "picard" else 0)
        s.set_state(to_abi(Q0))
        s.step(5, dt)
        out.append(from_abi(s.get_state()[0]))
    assert np.sqrt(np.sum((out[1] - out[0]) ** 2) / np.sum((out[0] - Q0) ** 2)) <= 1e-5


def _simple_wave_errors(nx, N, picard, amp=0.004, t_end=1.0):
    import paper_2502_09714_gb300 as dgpkg
    sw = ShearSimpleWave(amp=amp)
    h = 1.0 / nx
    xs = np.linspace(0.0, 1.0, nx + 1)
    yz = np.linspace(0.0, 3 * h, 4)
    m = kuhn_box_mesh(xs, yz, yz, periodic=(True, True, True), sort_by_vid=True)
    mat = np.zeros((m.n_elem, 6))
    mat[:, :4] = (1.0, 1.0, 1.0, 10.0)
    o = Oracle(m.elem_xyz, m.elem_vid, N, mat, law="nlshear")

    def ic(x):
        u = np.zeros(x.shape[:-1] + (10,))
        e = sw.eps0(x[..., 0])
        u[..., 3] = e
        u[..., 7] = np.vectorize(sw.v_of)(e)
        return u
    Q0 = o.project(ic)
    n = int(np.ceil(t_end / (0.5 * o.cfl_dt())))
    s = dgpkg.Solver(m.elem_xyz, m.elem_vid, N, law="nlshear")
    s.set_material(mat)
    if picard:
        s.set_predictor("picard", picard)
    s.set_state(to_abi(Q0))
    s.step(n, t_end / n)
    Q = from_abi(s.get_state()[0])
    pts, wq = tet_rule(N + 2)
    u = o.evaluate(Q, pts)
    x = o.xyz[:, 0, None, :] + np.einsum("edk,qk->eqd", o.J, pts, optimize=True)
    e, v = sw.sample(x[..., 0], t_end)
    dv = o.detJ[:, None] * wq[None, :] / (3 * h) ** 2
    return math.sqrt(np.sum(dv * (u[..., 3] - e) ** 2)), math.sqrt(np.sum(dv * (u[..., 7] - v) ** 2))


def test_picard_restores_the_order():
    """N = 2 on 8, 16 and 32 cells, to t = 1 (under a third of the time at which
    the characteristics cross, 3.6): the CK predictor's L2 errors fall at first order
    (1.2 measured between 16 and 32 cells), the Picard predictor's at the design
    order 3 (measured 3.0)."""
    ck = np.array([_simple_wave_errors(nx, 2, 0) for nx in (8, 16, 32)])
    pc = np.array([_simple_wave_errors(nx, 2, 2) for nx in (8, 16, 32)])
    o_ck = np.log2(ck[1] / ck[2])
    o_pc = np.log2(pc[:-1] / pc[1:])
    print("CK errors", ck.tolist(), "orders", o_ck, "Picard errors", pc.tolist(), "orders", o_pc)
    assert np.all(o_ck < 1.6), o_ck
    assert np.all(o_pc >= 2.6), o_pc
    assert np.all(pc[2] < 0.25 * ck[2])
