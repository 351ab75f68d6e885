"""GPU parity with boundary faces (Appendix A, absorbing and free surface):
libdg through the C-ABI against the FP64 oracle on boxes whose outer faces
are tagged, rough random data with damage on, and the exact rigid motion of a
free body."""
import math

import numpy as np
import pytest

from oracle import from_abi, mode_list, to_abi
from synthetic import rock_material
from synthetic.mesh import FACE_BC_ABSORBING, FACE_BC_FREE_SURFACE, kuhn_box_mesh

from parity_util import TOL_ALPHA, TOL_REL_L2, alpha_max_diff, make_oracle, make_solver, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    dgpkg.load_library()


def _box(cells, periodic, top, side, jitter=0.1, seed=5, length=4000.0):
    grids = [np.linspace(0.0, length, c + 1) for c in cells]
    return kuhn_box_mesh(*grids, periodic=periodic, jitter=jitter, seed=seed, top_bc=top, side_bc=side)


def _rough_state(E, N, seed, strain=3e-4, alpha=0.1):
    rng = np.random.default_rng(seed)
    deg = np.array([sum(m) for m in mode_list(N)])
    Q = rng.normal(size=(E, len(deg), 10)) * (0.5 ** deg)[None, :, None]
    Q[..., :6] *= strain
    Q[..., 6:9] *= strain * 6000.0 * 0.3
    Q[..., 9] *= 0.2 * alpha
    Q[:, 0, 9] = alpha / math.sqrt(6.0) + np.abs(Q[:, 0, 9])
    return Q


CASES = [
    # (N, cells, periodic, top tag, side tag)
    (1, (3, 3, 3), (False, False, False), FACE_BC_FREE_SURFACE, FACE_BC_ABSORBING),
    (2, (3, 3, 3), (False, False, False), FACE_BC_FREE_SURFACE, FACE_BC_ABSORBING),
    (3, (3, 3, 3), (True, True, False), FACE_BC_FREE_SURFACE, FACE_BC_ABSORBING),
    (4, (3, 3, 3), (False, False, False), FACE_BC_FREE_SURFACE, FACE_BC_ABSORBING),
    (4, (4, 3, 3), (False, True, True), FACE_BC_ABSORBING, FACE_BC_ABSORBING),
    (5, (3, 3, 2), (False, False, False), FACE_BC_FREE_SURFACE, FACE_BC_FREE_SURFACE),
]


@pytest.mark.parametrize("N,cells,periodic,top,side", CASES)
def test_box_with_boundary_faces(N, cells, periodic, top, side):
    """Rough random data, damage on, heterogeneous material, random local vertex
    order; a box with free-surface and/or absorbing outer faces (the face list
    mixes interior and boundary faces within the last tiles), 3 steps."""
    mesh = _box(cells, periodic, top, side, seed=N)
    rng = np.random.default_rng(40 + N)
    mesh = mesh.permuted(vertex_perm=np.array([rng.permutation(4) for _ in range(mesh.n_elem)]))
    mat = rock_material(mesh.n_elem)
    mat[:, 3] *= rng.uniform(0.5, 1.5, size=mesh.n_elem)
    mat[:, 0] *= rng.uniform(0.9, 1.1, size=mesh.n_elem)
    mat[:, 5] = 2e-6 * rng.uniform(0.5, 1.5, size=mesh.n_elem)
    o = make_oracle(mesh, mat, N)
    assert np.any(o.nbr < 0)
    Q0 = _rough_state(mesh.n_elem, N, seed=200 + N)
    dt = 0.5 * o.cfl_dt()
    s = make_solver(mesh, mat, N)
    s.set_state(to_abi(Q0))
    s.step(3, dt)
    q, _ = s.get_state()
    Q = o.run(Q0, dt, 3)
    errs = rel_l2(to_abi(from_abi(q) - Q0), Q - Q0, o.detJ)
    for name, e in errs.items():
        assert e <= TOL_REL_L2, (name, e)
    assert alpha_max_diff(q, Q, N) <= TOL_ALPHA
    # the boundary elements alone meet the bar too
    rows = np.nonzero((o.nbr < 0).any(axis=1))[0]
    errs_b = rel_l2(to_abi(from_abi(q) - Q0)[rows], (Q - Q0)[rows], o.detJ[rows])
    for name, e in errs_b.items():
        assert e <= TOL_REL_L2, ("boundary rows", name, e)


def test_free_body_moves_rigidly():
    """Uniform velocity, zero strain, free surfaces all round: an exact steady
    state of the scheme (zero traction on every face); 10 steps keep it to FP32
    rounding, damage on."""
    N = 3
    mesh = _box((3, 3, 3), (False, False, False), FACE_BC_FREE_SURFACE, FACE_BC_FREE_SURFACE, seed=9)
    mat = rock_material(mesh.n_elem, cd=1e-4)
    L = len(mode_list(N))
    Q0 = np.zeros((mesh.n_elem, L, 10))
    Q0[:, 0, 6:9] = np.array([0.3, -0.2, 0.5]) / math.sqrt(6.0)
    Q0[:, 0, 9] = 0.1 / math.sqrt(6.0)
    s = make_solver(mesh, mat, N)
    s.set_state(to_abi(Q0))
    s.step(10)
    q, _ = s.get_state()
    assert np.abs(from_abi(q) - Q0).max() <= 1e-6 * np.abs(Q0).max()
