"""GPU checks of the discrete adjoint (dg_adjoint_gradient): the misfit, its
gradient in xi0 and C_d and the gradient in the initial state against the
oracle's adjoint on the 384-tet cube and on a closed box with free-surface and
absorbing faces, invariance under the snapshot budget,
the state left untouched, the torch.autograd.Function, the refused
configurations, and, on the 82,944-tet adjoint workload, the second-order
Taylor remainder of the misfit along the gradient's own parameter directions.

Tolerance: the GPU runs the forward and the adjoint in FP32; the oracle in
FP64.  The gradient of a misfit is a difference of nearly equal products once
the residuals are small, so it is compared in relative L2 over the elements
with a bound of 2e-3 (FP32 rounding of ~1e3 accumulated products per value,
amplified by the steps of the run; measured up to 6e-4 at N = 4), and the
residual vector behind J to 1e-4 of the traces, like the states."""
import math

import numpy as np
import pytest

from oracle import Oracle, mode_list, to_abi
from oracle.adjoint import misfit_gradient
from synthetic import periodic_cube_mesh, workload_adjoint

pytestmark = pytest.mark.gpu

TOL_GRAD = 2e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    dgpkg.load_library()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(N, n_steps, seed=21):
    w = workload_adjoint(n=4, order=N, steps=n_steps)
    m = w["mesh"]
    # C_d scaled down so that the rough random state below keeps alpha under ~0.2
    for key in ("material", "material_ref"):
        w[key] = w[key].copy()
        w[key][:, 5] *= 0.75
    mat, mref = w["material"], w["material_ref"]
    o = Oracle(m.elem_xyz, m.elem_vid, N, mat)
    oref = Oracle(m.elem_xyz, m.elem_vid, N, mref)
    rng = np.random.default_rng(seed)
    deg = np.array([sum(mm) for mm in mode_list(N)])
    Q0 = rng.normal(size=(m.n_elem, o.L, 10)) * (0.5 ** deg)[None, :, None]
    Q0[..., :6] *= 2e-4
    Q0[..., 6:9] *= 0.6
    Q0[..., 9] *= 0.005
    Q0[:, 0, 9] = (0.02 + 0.03 * rng.uniform(size=m.n_elem)) / math.sqrt(6.0)
    for oo in (o, oref):
        oo.set_receivers(w["receivers"])
    dt = 0.5 * o.cfl_dt()
    _, ref = oref.run(Q0, dt, n_steps, record=True)
    return w, o, Q0, dt, ref


def _solver(w, N, Q0):
    import paper_2502_09714_gb300 as dgpkg
    m = w["mesh"]
    s = dgpkg.Solver(m.elem_xyz, m.elem_vid, N)
    s.set_material(w["material"])
    s.set_state(to_abi(Q0))
    s.set_receivers(w["receivers"])
    return s


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_adjoint_parity_with_oracle(N):
    n = 6
    w, o, Q0, dt, ref = _case(N, n)
    J, gx, gc, lq = misfit_gradient(o, Q0, dt, n, ref)
    s = _solver(w, N, Q0)
    Jg, gxg, gcg, lqg = s.adjoint_gradient(ref, n, dt, snapshots=3, grad_state=True)
    # J is a sum of squared residuals v - ref, and the residuals are small beside the
    # traces v: the GPU's residual vector may differ from the oracle's by the state
    # tolerance times the traces, |sqrt(J_gpu) - sqrt(J)| <= 1e-4 sqrt(1/2 dt sum v^2)
    _, v = o.run(Q0, dt, n, record=True)
    Jv = 0.5 * dt * float(np.sum(v * v))
    errs = {"J": abs(math.sqrt(Jg) - math.sqrt(J)) / math.sqrt(Jv), "xi0": _rel(gxg, gx), "cd": _rel(gcg, gc),
            "q0": _rel(lqg, to_abi(lq))}
    print(N, errs)
    assert errs["J"] <= 1e-4, errs
    assert errs["xi0"] <= TOL_GRAD and errs["cd"] <= TOL_GRAD and errs["q0"] <= TOL_GRAD, errs


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_adjoint_parity_with_boundary_faces(N):
    """A closed jittered box (162 tets) with a free-surface top and absorbing
    sides: the GPU gradient against the oracle's adjoint, whose boundary part is
    pinned by the dot-product tests on the same kind of box."""
    import paper_2502_09714_gb300 as dgpkg
    from synthetic.mesh import kuhn_box_mesh
    n = 6
    g = np.linspace(0.0, 4000.0, 4)
    mesh = kuhn_box_mesh(g, g, g, periodic=(False, False, False), jitter=0.1, seed=3)
    E = mesh.n_elem
    w = workload_adjoint(n=3, order=N, steps=n)
    mat, mref = w["material"].copy(), w["material_ref"].copy()
    mat[:, 5] *= 0.75
    mref[:, 5] *= 0.75
    rng = np.random.default_rng(50 + N)
    rec = rng.uniform(400.0, 3600.0, size=(16, 3))
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mat, face_bc=mesh.face_bc)
    oref = Oracle(mesh.elem_xyz, mesh.elem_vid, N, mref, face_bc=mesh.face_bc)
    for oo in (o, oref):
        oo.set_receivers(rec)
    deg = np.array([sum(mm) for mm in mode_list(N)])
    Q0 = rng.normal(size=(E, o.L, 10)) * (0.5 ** deg)[None, :, None]
    Q0[..., :6] *= 2e-4
    Q0[..., 6:9] *= 0.6
    Q0[..., 9] *= 0.005
    Q0[:, 0, 9] = (0.02 + 0.03 * rng.uniform(size=E)) / math.sqrt(6.0)
    dt = 0.5 * o.cfl_dt()
    _, ref = oref.run(Q0, dt, n, record=True)
    J, gx, gc, lq = misfit_gradient(o, Q0, dt, n, ref)
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, face_bc=mesh.face_bc)
    s.set_material(mat)
    s.set_state(to_abi(Q0))
    s.set_receivers(rec)
    Jg, gxg, gcg, lqg = s.adjoint_gradient(ref, n, dt, snapshots=3, grad_state=True)
    errs = {"xi0": _rel(gxg, gx), "cd": _rel(gcg, gc), "q0": _rel(lqg, to_abi(lq))}
    print(N, errs)
    assert errs["xi0"] <= TOL_GRAD and errs["cd"] <= TOL_GRAD and errs["q0"] <= TOL_GRAD, errs


def test_snapshot_budget_and_state_untouched():
    N, n = 2, 9
    w, o, Q0, dt, ref = _case(N, n, seed=5)
    s = _solver(w, N, Q0)
    q_before, t_before = s.get_state()
    budgets = (1, 2, 4, 0, n + 1)      # 0: as many as the free memory holds (here the whole history)
    runs = [s.adjoint_gradient(ref, n, dt, snapshots=k, grad_state=True, info=True) for k in budgets]
    q_after, t_after = s.get_state()
    assert np.array_equal(q_before, q_after) and t_before == t_after
    import paper_2502_09714_gb300 as dgpkg
    for k, r in zip(budgets, runs):
        assert r[4]["adjoint_steps"] == n
        assert r[4]["forward_steps"] == dgpkg.revolve_cost(n, k if k else n + 1) + 1
        assert r[0] == pytest.approx(runs[-1][0], rel=1e-12)
        for i in (1, 2, 3):
            assert np.allclose(r[i], runs[-1][i], rtol=0, atol=1e-6 * np.abs(runs[-1][i]).max())


def test_autograd_function():
    import torch
    import paper_2502_09714_gb300 as dgpkg
    N, n = 2, 4
    w, o, Q0, dt, ref = _case(N, n, seed=8)
    s = _solver(w, N, Q0)
    Jg, gxg, gcg = s.adjoint_gradient(ref, n, dt, snapshots=2)
    xi0 = torch.tensor(w["material"][:, 4], dtype=torch.float64, requires_grad=True)
    cd = torch.tensor(w["material"][:, 5], dtype=torch.float64, requires_grad=True)
    J = dgpkg.misfit_function().apply(xi0, cd, s, w["material"], ref, n, dt, 2)
    (3.0 * J).backward()
    assert float(J.detach()) == pytest.approx(Jg, rel=1e-12)
    assert np.allclose(xi0.grad.numpy(), 3.0 * gxg, rtol=1e-12, atol=0)
    assert np.allclose(cd.grad.numpy(), 3.0 * gcg, rtol=1e-12, atol=0)


def test_refused_configurations():
    import paper_2502_09714_gb300 as dgpkg
    N, n = 2, 2
    w, o, Q0, dt, ref = _case(N, n)
    m = w["mesh"]
    s = dgpkg.Solver(m.elem_xyz, m.elem_vid, N)
    s.set_material(w["material"])
    s.set_state(to_abi(Q0))
    s.R = len(w["receivers"])
    with pytest.raises(dgpkg.DGError, match="DG_E_STATE"):
        s.adjoint_gradient(ref, n, dt)                       # no receivers
    s.set_receivers(w["receivers"])
    s.set_predictor("picard", 2)
    with pytest.raises(dgpkg.DGError, match="DG_E_UNSUPPORTED"):
        s.adjoint_gradient(ref, n, dt)
    s.set_predictor("ck", 0)
    with pytest.raises(dgpkg.DGError, match="DG_E_ARG"):
        s.adjoint_gradient(ref, n, dt, snapshots=-1)
    s.set_rheology("ivm")
    mat = w["material"].copy()
    mat[:, 3:5] = (1e5, 1.0)
    s.set_material(mat)
    with pytest.raises(dgpkg.DGError, match="DG_E_UNSUPPORTED"):
        s.adjoint_gradient(ref, n, dt)


def test_taylor_remainder_on_the_adjoint_workload():
    """The 82,944-tet jittered cube of the adjoint workload at N = 3, in the
    launch configuration of the benchmark, from a rough damaged state (the
    recipe of the small cases) over 20 steps with 5 snapshots: along the
    direction d = (dJ/dxi0, dJ/dC_d), scaled per parameter, the first-order
    remainder |J(p + h d) - J(p) - h <g, d>| falls like h^2 (ratio about 4 per
    halving of h), which holds only if g is the gradient of the run the GPU
    takes."""
    import paper_2502_09714_gb300 as dgpkg
    n, N = 20, 3
    w = workload_adjoint(steps=n)
    m = w["mesh"]
    mat, mref = w["material"].copy(), w["material_ref"].copy()
    mat[:, 5] *= 0.75
    mref[:, 5] *= 0.75
    rng = np.random.default_rng(33)
    deg = np.array([sum(mm) for mm in mode_list(N)])
    Q0 = rng.normal(size=(m.n_elem, len(deg), 10)) * (0.5 ** deg)[None, :, None]
    Q0[..., :6] *= 2e-4
    Q0[..., 6:9] *= 0.6
    Q0[..., 9] *= 0.005
    Q0[:, 0, 9] = (0.02 + 0.03 * rng.uniform(size=m.n_elem)) / math.sqrt(6.0)
    q0 = to_abi(Q0)
    s = dgpkg.Solver(m.elem_xyz, m.elem_vid, N)
    s.set_material(mref)
    s.set_receivers(w["receivers"])
    s.set_state(q0)
    dt = s.dt
    s.step(n, dt)
    ref = s.read_receivers()
    s.set_material(mat)
    s.set_state(q0)
    J0, gx, gc = s.adjoint_gradient(ref, n, dt, snapshots=5)
    assert J0 > 0 and np.abs(gx).max() > 0 and np.abs(gc).max() > 0
    dx = 0.02 * gx / np.abs(gx).max()
    dc = 0.2 * mat[:, 5] * gc / np.abs(gc).max()
    lin = float(np.dot(gx, dx) + np.dot(gc, dc))
    rem = []
    for h in (1.0, 0.5, 0.25):
        mh = mat.copy()
        mh[:, 4] += h * dx
        mh[:, 5] += h * dc
        s.set_material(mh)
        s.set_state(q0)
        Jh = s.adjoint_gradient(ref, n, dt, snapshots=5)[0]
        rem.append(abs(Jh - J0 - h * lin))
    print("J0", J0, "h<g,d>", lin, "remainders", rem)
    assert rem[0] < 0.2 * abs(lin)
    assert 2.5 < rem[0] / rem[1] < 6.0 and 2.5 < rem[1] / rem[2] < 6.0, rem
