"""GPU parity: libdg (FP32 CUDA, through the C-ABI) against the FP64 oracle on
the same seeded inputs.  Bar: relative L2 <= 1e-4 per field group
(strains, velocities) and |alpha_gpu - alpha_oracle| <= 1e-5 at the volume
nodes, after the run."""
import math

import numpy as np
import pytest

from oracle import Oracle, from_abi, to_abi
from synthetic import (periodic_cube_mesh, rock_material, workload_c1, workload_c2,
                       workload_small_layered)

from parity_util import (TOL_ALPHA, TOL_REL_L2, alpha_max_diff, assert_parity, make_oracle,
                         make_solver, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    dgpkg.load_library()


def plane_p_wave(A, k, cp):
    def f(x):
        u = np.zeros(x.shape[:-1] + (10,))
        ph = np.sin(k * x[..., 0])
        u[..., 0] = A * ph
        u[..., 6] = -cp * A * ph
        return u
    return f


@pytest.mark.parametrize("damage", [False, True])
def test_c1_plane_wave_20_steps(damage):
    """384-tet periodic cube, N=2, plane P-wave of strain 1e-4, 20 steps at CFL 0.5."""
    w = workload_c1(damage=damage)
    mesh, mat, N = w["mesh"], w["material"], w["order"]
    o = make_oracle(mesh, mat, N, cfl=w["cfl"])
    cp = math.sqrt((mat[0, 1] + 2 * mat[0, 2]) / mat[0, 0])
    pw = w["plane_wave"]
    Q0 = o.project(plane_p_wave(pw["amplitude"], pw["k"], cp))
    dt = o.cfl_dt()
    s = make_solver(mesh, mat, N, cfl=w["cfl"])
    assert s.dt == pytest.approx(dt, rel=1e-12)
    s.set_state(to_abi(Q0))
    s.step(w["steps"], dt)
    q, t = s.get_state()
    assert t == pytest.approx(20 * dt)
    Q = o.run(Q0, dt, w["steps"])
    errs, da = assert_parity(q, Q, o.detJ, N)
    if damage:
        assert np.abs(Q[:, 0, 9]).max() > 1e-6      # damage did grow


def _random_state(mesh, N, seed, strain=3e-4, alpha=0.1):
    """Per-element random modal coefficients with a decaying spectrum (rough,
    discontinuous data; strains around 3e-4 so that the damage law is active
    without reaching loss of hyperbolicity within the run)."""
    rng = np.random.default_rng(seed)
    from oracle import mode_list
    deg = np.array([sum(m) for m in mode_list(N)])
    decay = 0.5 ** deg
    Q = rng.normal(size=(mesh.n_elem, len(deg), 10)) * decay[None, :, None]
    cp = 6000.0
    Q[..., :6] *= strain
    Q[..., 6:9] *= strain * cp * 0.3
    Q[..., 9] *= 0.2 * alpha
    Q[:, 0, 9] = alpha / math.sqrt(6.0) + np.abs(Q[:, 0, 9])
    return Q


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_random_rough_state_all_degrees(N):
    """Rough random data, damage on, random local vertex order in the input
    (the state basis follows the vertex ids), 162 tets (ragged last CTA), 3 steps."""
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=17)
    rng = np.random.default_rng(N)
    mesh = mesh.permuted(vertex_perm=np.array([rng.permutation(4) for _ in range(mesh.n_elem)]))
    mat = rock_material(mesh.n_elem)
    mat[:, 3] *= rng.uniform(0.5, 1.5, size=mesh.n_elem)     # heterogeneous gamma_r
    mat[:, 0] *= rng.uniform(0.9, 1.1, size=mesh.n_elem)     # heterogeneous density
    # damage-rate coefficient: alpha grows by ~1e-2 over the run at the large
    # low-degree time steps, so the cells stay hyperbolic
    mat[:, 5] = 2e-6 * rng.uniform(0.5, 1.5, size=mesh.n_elem)
    o = make_oracle(mesh, mat, N)
    Q0 = _random_state(mesh, N, seed=100 + N)
    dt = 0.5 * o.cfl_dt()
    s = make_solver(mesh, mat, N)
    s.set_state(to_abi(Q0))
    # the state round trip through the ABI is exact up to FP32 rounding
    q0, _ = s.get_state()
    np.testing.assert_allclose(q0, to_abi(Q0), rtol=0, atol=2e-6 * np.abs(Q0).max())
    s.step(3, dt)
    q, _ = s.get_state()
    Q = o.run(Q0, dt, 3)
    # compare the change over the run, which is what the step computes
    errs = rel_l2(to_abi(from_abi(q) - Q0), Q - Q0, o.detJ)
    for name, e in errs.items():
        assert e <= TOL_REL_L2, (name, e)
    assert alpha_max_diff(q, Q, N) <= TOL_ALPHA


@pytest.mark.parametrize("N,n", [(2, 3), (3, 4), (4, 3)])
def test_layered_point_source_and_receivers(N, n):
    """c2-shaped workload at oracle size: jittered two-layer cube, dip-slip point
    source, receivers; 12 steps from rest."""
    w = workload_small_layered(n=n, order=N, m0=4e15)
    mesh, mat = w["mesh"], w["material"]
    o = make_oracle(mesh, mat, N, sources=w["sources"], receivers=w["receivers"])
    dt = o.cfl_dt()
    # start in the middle of the wavelet so the source injects a large signal
    t0 = 0.35
    Q0 = np.zeros((mesh.n_elem, o.L, 10))
    s = make_solver(mesh, mat, N, sources=w["sources"], receivers=w["receivers"])
    s.set_state(to_abi(Q0), t0)
    steps = 12
    s.step(steps, dt)
    q, t = s.get_state()
    Q, tr = o.run(Q0, dt, steps, t0=t0, record=True)
    assert np.abs(Q).max() > 0
    assert_parity(q, Q, o.detJ, N)
    traces = s.read_receivers()
    assert traces.shape == (steps,) + tr.shape[1:]
    scale = np.abs(tr).max()
    assert scale > 0
    np.testing.assert_allclose(traces, tr, rtol=0, atol=1e-4 * scale)


def test_full_size_c2_sampled_step():
    """The 196,608-tet N=4 workload in the benchmark's launch configuration:
    run 40 steps on the GPU, then compare one more GPU step against the
    oracle's step from the GPU state on sampled elements."""
    w = workload_c2()
    mesh, mat = w["mesh"], w["material"]
    s = make_solver(mesh, mat, 4, sources=w["sources"], receivers=w["receivers"])
    E = mesh.n_elem
    s.set_state(np.zeros((E, 10, 35), np.float32), 0.3)
    s.step(40)
    qa, ta = s.get_state()
    # sample: the source element's neighbourhood (signal) + random elements
    rng = np.random.default_rng(5)
    energy = np.abs(qa).reshape(E, -1).max(axis=1)
    hot = np.argsort(energy)[-48:]
    rows = np.unique(np.concatenate([hot, rng.choice(E, 16, replace=False)]))
    o = make_oracle(mesh, mat, 4, sources=w["sources"], face_rows=rows)
    dt = s.dt
    assert dt == pytest.approx(o.cfl_dt(), rel=1e-12)
    s.step(1, dt)
    qb, _ = s.get_state()
    Qa = from_abi(qa)
    Qb_ora = o.step(Qa, dt, t=ta, rows=rows)
    Gb = from_abi(qb)[rows]
    # the bar applies to what the step computes, its change of the state: one step
    # changes the state by a small part of itself, so a bar on the state alone
    # would be |Q| / |dQ| times looser on the step's own arithmetic
    dG, dO = Gb - Qa[rows], Qb_ora - Qa[rows]
    for name, sl in (("strain", slice(0, 6)), ("velocity", slice(6, 9))):
        num = np.sqrt(np.sum(o.detJ[rows, None, None] * (dG[..., sl] - dO[..., sl]) ** 2))
        den = np.sqrt(np.sum(o.detJ[rows, None, None] * dO[..., sl] ** 2))
        assert den > 0 and num <= TOL_REL_L2 * den, (name, num / den)
    assert np.abs(Gb[..., 9] - Qb_ora[..., 9]).max() <= TOL_ALPHA


@pytest.mark.slow
def test_c2_shaped_full_run_500_steps():
    """The c2 workload's run length at a size the oracle finishes: the jittered
    two-layer cube at 4 cells per side (384 tets), N = 4, the dip-slip Ricker point
    source and the 64 receivers, 500 steps from rest at the CFL step, through the
    whole wavelet and its reflections and periodic wrap-arounds.  The bar is the
    state after the run (relative L2 per field group, absolute on alpha) and the
    receiver traces of every step.  The peak moment rate is 4e13 N m/s (peak strain
    about 2e-5, alpha up to 4.5e-4): on 1 km elements the point source's delta is
    rough at the quadrature nodes, and from 4e14 on the nonlinear step runs away
    next to the source near the wavelet's peak, in the FP64 oracle as well."""
    from parity_util import oracle_run_pool
    w = workload_small_layered(n=4, order=4, m0=4e13)
    mesh, mat, N = w["mesh"], w["material"], 4
    steps = w["steps"]
    assert steps == 500
    o = make_oracle(mesh, mat, N, sources=w["sources"], receivers=w["receivers"])
    dt = o.cfl_dt()
    Q0 = np.zeros((mesh.n_elem, o.L, 10))
    s = make_solver(mesh, mat, N, sources=w["sources"], receivers=w["receivers"])
    s.set_state(to_abi(Q0), 0.0)
    s.step(steps, dt)
    q, t = s.get_state()
    traces = s.read_receivers()
    Q, tr = oracle_run_pool(mesh, mat, N, Q0, dt, steps, sources=w["sources"], receivers=w["receivers"])
    assert t == pytest.approx(steps * dt)
    assert np.abs(Q[..., :9]).max() > 0 and np.abs(Q[..., 9]).max() > 0
    assert_parity(q, Q, o.detJ, N)
    assert traces.shape == tr.shape
    np.testing.assert_allclose(traces, tr, rtol=0, atol=1e-4 * np.abs(tr).max())


def test_zero_state_and_empty_calls():
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=2)
    mat = rock_material(mesh.n_elem)
    s = make_solver(mesh, mat, 3)
    from paper_2502_09714_gb300 import DGError
    with pytest.raises(DGError) as ei:
        s.step(1)
    assert ei.value.name == "DG_E_STATE"
    s.set_state(np.zeros((mesh.n_elem, 10, 20)))
    s.step(0)
    s.step(5)
    q, t = s.get_state()
    assert np.all(q == 0.0)
    assert t == pytest.approx(5 * s.dt)
    st = s.stats()
    # predictor, face fluxes and corrector per step
    assert st["steps"] == 5 and st["kernel_launches"] == 15 and st["element_updates"] == 5 * mesh.n_elem


def test_status_nonfinite_and_nonhyperbolic():
    from paper_2502_09714_gb300 import DGError
    mesh = periodic_cube_mesh(3, 4000.0)
    mat = rock_material(mesh.n_elem)
    s = make_solver(mesh, mat, 2)
    Q = np.zeros((mesh.n_elem, 10, 10))
    Q[7, 6, 3] = np.nan
    s.set_state(Q)
    with pytest.raises(DGError) as ei:
        s.step(1)
    assert ei.value.name == "DG_E_NONFINITE"
    # damage beyond loss of hyperbolicity: mu_eff = mu0 + alpha xi0 gamma_r < 0
    Q = np.zeros((mesh.n_elem, 10, 10))
    Q[:, 9, 0] = 2.0 / math.sqrt(6.0)
    s.set_state(Q)
    with pytest.raises(DGError) as ei:
        s.step(1)
    assert ei.value.name == "DG_E_NONHYPERBOLIC"


def test_source_outside_and_receiver_outside():
    from paper_2502_09714_gb300 import DGError
    mesh = periodic_cube_mesh(3, 4000.0)
    s = make_solver(mesh, rock_material(mesh.n_elem), 2)
    with pytest.raises(DGError) as ei:
        s.set_sources([{"x": [1e5, 0, 0], "m": [1, 0, 0, 0, 0, 0], "stf": 0, "f0": 2.0, "t0": 0.1}])
    assert ei.value.name == "DG_E_OUTSIDE"
    with pytest.raises(DGError) as ei:
        s.set_receivers([[0.0, 0.0, -50.0]])
    assert ei.value.name == "DG_E_OUTSIDE"


def test_profile_counts_kernels():
    w = workload_small_layered(n=3, order=2)
    s = make_solver(w["mesh"], w["material"], 2, sources=w["sources"], receivers=w["receivers"])
    s.set_state(np.zeros((w["mesh"].n_elem, 10, 10)), 0.3)
    s.profile(True)
    s.step(7)
    p = s.profile_read()
    assert p["predictor"]["launches"] == 7 and p["corrector"]["launches"] == 7
    assert p["faces"]["launches"] == 7
    assert p["source"]["launches"] == 7 and p["receivers"]["launches"] == 7
    assert p["corrector"]["total_ms"] > 0 and p["faces"]["total_ms"] > 0
    assert s.stats()["kernel_launches"] == 35


@pytest.mark.parametrize("N", [2, 3])
def test_anisotropic_prestrain_plane_wave(N):
    """Sec. 3.3's setting on the GPU: uniform pre-strain 1e-3 rotated by 30 degrees,
    alpha = 0.5, gamma_r = 37 GPa, C_d = 0, a small P-like plane perturbation along
    x; 12 steps against the oracle (the change over the run is compared)."""
    import test_oracle_anisotropy as ani
    from synthetic.mesh import kuhn_box_mesh
    t = ani._table()
    mat1 = np.array([t["rho"], t["lambda0"], t["mu0"], t["gamma_r"], t["xi0"], t["Cd"]])
    u0 = ani._pre_state(t, math.radians(30.0))
    w, V = np.linalg.eigh(ani._acoustic_tensor(u0, mat1))
    c, a = math.sqrt(w[2]), V[:, 2]
    Lx, n = 1.0 / t["k"], 4
    grids = [np.linspace(0.0, Lx, n + 1)] + [np.linspace(0.0, 3 * Lx / n, 4)] * 2
    mesh = kuhn_box_mesh(*grids, periodic=(True, True, True), jitter=0.1, seed=5)
    mat = np.tile(mat1, (mesh.n_elem, 1))
    o = make_oracle(mesh, mat, N)
    E = 0.5 * (np.outer([1.0, 0.0, 0.0], a) + np.outer(a, [1.0, 0.0, 0.0]))

    def init(x):
        g = t["A0"] * np.sin(2 * np.pi * t["k"] * x[..., 0])
        u = np.broadcast_to(u0, x.shape[:-1] + (10,)).copy()
        for p, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))):
            u[..., p] += E[i, j] * g
        u[..., 6:9] += -c * a * g[..., None]
        return u
    Q0 = o.project(init)
    dt = o.cfl_dt()
    s = make_solver(mesh, mat, N)
    s.set_state(to_abi(Q0))
    s.step(12, dt)
    q, _ = s.get_state()
    Q = o.run(Q0, dt, 12)
    assert_parity(q, Q, o.detJ, N)                      # the state, as the bar is defined
    # the perturbation alone is 400 times smaller than the FP32-stored pre-strain, so
    # its own relative error has an FP32 floor of about 1e-4; it must stay within 1e-3
    errs = rel_l2(to_abi(from_abi(q) - Q0), Q - Q0, o.detJ)
    for name, e in errs.items():
        assert e <= 1e-3, (name, e)
