"""The host-to-host step (dg_step_host): chunked transfers overlapping the step
must give exactly the state of set_state / step / get_state, with sources and
receivers, on one member, with several chunks and a ragged last chunk; with
members it falls back to the plain sequence.  The face fluxes run in ranges as
soon as the predictors of both sides are done: the cases cover faces reaching
back to the first chunk (periodic wrap), boundary faces in every chunk (a box
with free-surface and absorbing sides), and an element order shuffled so that
most chunks' faces wait for the last chunk."""
import numpy as np
import pytest
import torch

from synthetic import periodic_cube_mesh, rock_material, workload_small_layered
from synthetic.mesh import kuhn_box_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    dgpkg.load_library()


def _state(E, L, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(E, 10, L)) * 1e-4
    q[:, 6:9, :] *= 2000.0
    q[:, 9, :] = np.abs(q[:, 9, :]) * 100.0
    return q.astype(np.float32)


def _mesh(case):
    if case == "periodic4":                       # 384 elements: one chunk
        return periodic_cube_mesh(4, 4000.0, jitter=0.1, seed=3)
    if case == "periodic13":                      # 13182 elements: three chunks, the last ragged
        return periodic_cube_mesh(13, 4000.0, jitter=0.1, seed=13)
    if case == "periodic32":                      # 196608 elements: nine chunks, the first and last halved
        return periodic_cube_mesh(32, 4000.0, jitter=0.1, seed=32)
    g = np.linspace(0.0, 4000.0, 13)              # 10368 elements: three chunks, boundary faces in each
    mesh = kuhn_box_mesh(g, g, g, periodic=(False, True, False), jitter=0.1, seed=5)
    if case == "box_shuffled":
        mesh = mesh.permuted(elem_perm=np.random.default_rng(7).permutation(mesh.n_elem))
    return mesh


@pytest.mark.parametrize("case", ["periodic4", "periodic13", "periodic32", "box", "box_shuffled"])
def test_step_host_equals_the_plain_sequence(case):
    import paper_2502_09714_gb300 as dgpkg
    N = 2
    mesh = _mesh(case)
    bc = mesh.face_bc if np.any(mesh.face_bc != 0) else None
    mat = rock_material(mesh.n_elem, cd=2e-6)
    E, L = mesh.n_elem, dgpkg.n_modes(N)
    src = [{"x": np.array([1900.0, 2100.0, 2000.0]), "m": np.array([1, -1, 0, 0.5, 0, 0]) * 1e13,
            "stf": 0, "f0": 2.0, "t0": 0.3}]
    rec = np.array([[1000.0, 1000.0, 1000.0], [3000.0, 2000.0, 1500.0]])
    q0 = _state(E, L, seed=E)
    runs = []
    for host in (False, True):
        s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, face_bc=bc, stream=torch.cuda.current_stream())
        s.set_material(mat)
        s.set_sources(src)
        s.set_receivers(rec)
        s.set_state(q0, 0.1)
        dt = s.dt
        if host:
            hin = torch.from_numpy(q0.copy()).pin_memory()
            hout = torch.empty_like(hin).pin_memory()
            s.step_host(hin.numpy(), hout.numpy(), dt)
            s.step_host(hout.numpy(), hout.numpy(), dt)   # input and output may alias
            q = hout.numpy().copy()
        else:
            s.set_state(q0, 0.1)
            s.step(1, dt)
            q1, _ = s.get_state(dtype=np.float32)
            s.set_state(q1, 0.1 + dt)
            s.step(1, dt)
            q, _ = s.get_state(dtype=np.float32)
        runs.append((q, s.time, s.read_receivers()))
        s.close()
    (qa, ta, ra), (qb, tb, rb) = runs
    assert np.array_equal(qa, qb)
    assert ta == pytest.approx(tb)
    assert np.array_equal(ra, rb)
