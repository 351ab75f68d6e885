"""GPU parity under the IVM law (Eq. "ivm-model" without Murnaghan terms,
Eq. "effective-ivm" for the predictor and boundary Jacobians): rough random
data at several degrees, a closed box with free and absorbing faces, and
uniform-strain damage growth, each against the oracle with law="ivm"."""
import math

import numpy as np
import pytest

from oracle import Oracle, from_abi, mode_list, to_abi
from synthetic import periodic_cube_mesh
from synthetic.mesh import FACE_BC_ABSORBING, FACE_BC_FREE_SURFACE, kuhn_box_mesh

from parity_util import TOL_ALPHA, TOL_REL_L2, alpha_max_diff, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    dgpkg.load_library()


def _ivm_material(E, rng):
    mat = np.empty((E, 6))
    mat[:, 0] = 2700.0 * rng.uniform(0.9, 1.1, size=E)
    mat[:, 1] = 32e9
    mat[:, 2] = 32e9
    mat[:, 3] = 1e5 * rng.uniform(0.5, 2.0, size=E)      # gamma_b [Pa]
    mat[:, 4] = 1.0 * rng.uniform(0.5, 2.0, size=E)      # tau_b [s]
    mat[:, 5] = 0.0
    return mat


def _rough_state(E, N, seed, strain=3e-4, alpha=0.1):
    rng = np.random.default_rng(seed)
    deg = np.array([sum(m) for m in mode_list(N)])
    Q = rng.normal(size=(E, len(deg), 10)) * (0.5 ** deg)[None, :, None]
    Q[..., :6] *= strain
    Q[..., 6:9] *= strain * 6000.0 * 0.3
    Q[..., 9] *= 0.2 * alpha
    Q[:, 0, 9] = alpha / math.sqrt(6.0) + np.abs(Q[:, 0, 9])
    return Q


def _run_pair(mesh, mat, N, Q0, steps, face_bc=None):
    import paper_2502_09714_gb300 as dgpkg
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, face_bc=face_bc, law="ivm")
    dt = 0.5 * o.cfl_dt()
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, face_bc=face_bc, law="ivm")
    s.set_material(mat)
    s.set_state(to_abi(Q0))
    s.step(steps, dt)
    q, _ = s.get_state()
    return o, q, o.run(Q0, dt, steps)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_ivm_rough_state(N):
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=41)
    rng = np.random.default_rng(90 + N)
    mesh = mesh.permuted(vertex_perm=np.array([rng.permutation(4) for _ in range(mesh.n_elem)]))
    mat = _ivm_material(mesh.n_elem, rng)
    Q0 = _rough_state(mesh.n_elem, N, seed=500 + N)
    o, q, Q = _run_pair(mesh, mat, N, Q0, 3)
    assert np.abs(Q[:, 0, 9] - Q0[:, 0, 9]).max() > 1e-3          # the damage moved
    errs = rel_l2(to_abi(from_abi(q) - Q0), Q - Q0, o.detJ)
    for name, e in errs.items():
        assert e <= TOL_REL_L2, (name, e)
    assert alpha_max_diff(q, Q, N) <= TOL_ALPHA


def test_ivm_box_with_boundary_faces():
    N = 3
    g = np.linspace(0.0, 4000.0, 4)
    mesh = kuhn_box_mesh(g, g, g, periodic=(False, False, False), jitter=0.1, seed=8,
                         top_bc=FACE_BC_FREE_SURFACE, side_bc=FACE_BC_ABSORBING)
    rng = np.random.default_rng(7)
    mat = _ivm_material(mesh.n_elem, rng)
    Q0 = _rough_state(mesh.n_elem, N, seed=77)
    o, q, Q = _run_pair(mesh, mat, N, Q0, 3, face_bc=mesh.face_bc)
    errs = rel_l2(to_abi(from_abi(q) - Q0), Q - Q0, o.detJ)
    for name, e in errs.items():
        assert e <= TOL_REL_L2, (name, e)
    assert alpha_max_diff(q, Q, N) <= TOL_ALPHA


def test_ivm_uniform_strain_damage():
    """Uniform strain, v = 0, 20 steps: the damage of every element follows the
    oracle's (which converges to the exact ODE solution)."""
    N = 2
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=42)
    mat = _ivm_material(mesh.n_elem, np.random.default_rng(3))
    L = len(mode_list(N))
    Q0 = np.zeros((mesh.n_elem, L, 10))
    Q0[:, 0, :6] = np.array([3e-4, -1e-4, 6e-5, 1.2e-4, 0.0, -3e-5]) / math.sqrt(6.0)   # phi_0 = sqrt(6)
    o, q, Q = _run_pair(mesh, mat, N, Q0, 20)
    assert Q[:, 0, 9].max() > 1e-3
    assert alpha_max_diff(q, Q, N) <= TOL_ALPHA
