"""GPU parity of the ensemble form: M members with their own damage parameters
(xi0, C_d) and states advance in one set of launches per step; each member is
checked against the FP64 oracle run with that member's parameters."""
import math

import numpy as np
import pytest

from oracle import from_abi, mode_list, to_abi
from synthetic import periodic_cube_mesh, rock_material, workload_small_layered

from parity_util import TOL_ALPHA, TOL_REL_L2, alpha_max_diff, make_oracle, make_solver, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    dgpkg.load_library()


def _rough_state(E, N, seed, strain=3e-4, alpha=0.1):
    rng = np.random.default_rng(seed)
    deg = np.array([sum(m) for m in mode_list(N)])
    Q = rng.normal(size=(E, len(deg), 10)) * (0.5 ** deg)[None, :, None]
    Q[..., :6] *= strain
    Q[..., 6:9] *= strain * 6000.0 * 0.3
    Q[..., 9] *= 0.2 * alpha
    Q[:, 0, 9] = alpha / math.sqrt(6.0) + np.abs(Q[:, 0, 9])
    return Q


def _solver(mesh, mat, N, M, member_params):
    import paper_2502_09714_gb300 as dgpkg
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, members=M)
    s.set_material(mat, member_params)
    return s


@pytest.mark.parametrize("N,M", [(3, 3), (2, 5), (4, 2)])
def test_members_match_their_own_oracle_runs(N, M):
    """Rough random data per member; per-member, per-element xi0 in [-1, -0.6]
    and C_d log-uniform (scaled so the cells stay hyperbolic); 3 steps; every
    member meets the parity bar against the oracle with its own parameters."""
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=31)
    rng = np.random.default_rng(70 + N)
    mat = rock_material(mesh.n_elem)
    params = np.empty((M, mesh.n_elem, 2))
    params[..., 0] = rng.uniform(-1.0, -0.6, size=(M, mesh.n_elem))
    params[..., 1] = 2e-6 * np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=(M, mesh.n_elem)))
    states = np.stack([_rough_state(mesh.n_elem, N, seed=300 + 10 * N + m) for m in range(M)])
    s = _solver(mesh, mat, N, M, params)
    s.set_state(np.stack([to_abi(Q) for Q in states]))
    o0 = make_oracle(mesh, mat, N)
    dt = 0.5 * o0.cfl_dt()
    assert s.dt == pytest.approx(o0.cfl_dt(), rel=1e-12)
    s.step(3, dt)
    q, _ = s.get_state()
    assert q.shape == (M, mesh.n_elem, 10, len(mode_list(N)))
    for m in range(M):
        mat_m = mat.copy()
        mat_m[:, 4:6] = params[m]
        o = make_oracle(mesh, mat_m, N)
        Q = o.run(states[m], dt, 3)
        errs = rel_l2(to_abi(from_abi(q[m]) - states[m]), Q - states[m], o.detJ)
        for name, e in errs.items():
            assert e <= TOL_REL_L2, (m, name, e)
        assert alpha_max_diff(q[m], Q, N) <= TOL_ALPHA, m


def test_identical_members_reproduce_the_single_run():
    """Members with the same parameters and state give the same result as one
    member run alone: the per-element arithmetic does not depend on which
    copies share a tile."""
    N, M = 3, 4
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=32)
    mat = rock_material(mesh.n_elem, cd=2e-6)
    Q0 = _rough_state(mesh.n_elem, N, seed=9)
    single = make_solver(mesh, mat, N)
    single.set_state(to_abi(Q0))
    single.step(4)
    q1, _ = single.get_state()
    ens = _solver(mesh, mat, N, M, None)
    ens.set_state(np.stack([to_abi(Q0)] * M))
    ens.step(4)
    qm, _ = ens.get_state()
    scale = np.abs(q1).max()
    for m in range(M):
        np.testing.assert_allclose(qm[m], q1, rtol=0, atol=1e-6 * scale)
    assert ens.stats()["element_updates"] == 4 * M * mesh.n_elem


def test_members_with_source_and_receivers():
    """c2-shaped layered mesh at oracle size, point source and receivers in
    every member, two members with different damage parameters: states and
    receiver traces of each member against its own oracle run."""
    N, M = 3, 2
    w = workload_small_layered(n=3, order=N, m0=4e15)
    mesh, mat = w["mesh"], w["material"]
    params = np.empty((M, mesh.n_elem, 2))
    params[0] = mat[:, 4:6]
    params[1, :, 0] = -0.7
    params[1, :, 1] = 3.0 * mat[:, 5]
    s = _solver(mesh, mat, N, M, params)
    s.set_sources(w["sources"])
    s.set_receivers(w["receivers"])
    L = len(mode_list(N))
    t0 = 0.35
    s.set_state(np.zeros((M, mesh.n_elem, 10, L)), t0)
    steps = 10
    s.step(steps)
    q, _ = s.get_state()
    tr = s.read_receivers()
    assert tr.shape == (steps, M, len(w["receivers"]), 3)
    for m in range(M):
        mat_m = mat.copy()
        mat_m[:, 4:6] = params[m]
        o = make_oracle(mesh, mat_m, N, sources=w["sources"], receivers=w["receivers"])
        dt = o.cfl_dt()
        Q = np.zeros((mesh.n_elem, L, 10))
        rec = []
        t = t0
        for _ in range(steps):
            Q = o.step(Q, dt, t)
            t += dt
            rec.append(o.sample_receivers(Q))
        errs = rel_l2(q[m], Q, o.detJ)
        for name, e in errs.items():
            assert e <= TOL_REL_L2, (m, name, e)
        assert alpha_max_diff(q[m], Q, N) <= TOL_ALPHA
        rec = np.array(rec)
        assert np.abs(tr[:, m] - rec).max() <= 1e-4 * np.abs(rec).max(), m
