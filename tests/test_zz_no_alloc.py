"""The allocation-free step (dg_step_noalloc), for callers that cannot call
cudaMalloc while they step: it must give the same state as dg_step, call
after call, and refuse meshes larger than its fixed static scratch.

Both entry points run the same predictor, face-flux and corrector kernels on
the same FP32 input, element by element in the same order of operations, so
their states must agree bit for bit; a stale or misplaced region of the
shared static scratch would show up as a difference.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from synthetic import periodic_cube_mesh, rock_material

pytestmark = pytest.mark.gpu


def _state(E, L, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(E, 10, L)) * 1e-4
    q[:, 6:9, :] *= 2000.0
    q[:, 9, :] = np.abs(q[:, 9, :]) * 100.0
    return q.astype(np.float32)


def _compare(q_new, q_ref):
    np.testing.assert_array_equal(q_new, q_ref)


def test_noalloc_step_matches_dg_step_on_two_calls_in_a_row():
    import torch

    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    torch.cuda.set_device(0)
    N = 3
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=9)
    mat = rock_material(mesh.n_elem, cd=2e-6)
    E, L = mesh.n_elem, dgpkg.n_modes(N)
    stream = torch.cuda.current_stream()
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, stream=stream)
    s.set_material(mat)
    q0 = _state(E, L, seed=3)
    dt = s.dt
    # reference: the existing entry point, two steps
    s.set_state(q0)
    s.step(1, dt)
    ref1, _ = s.get_state()
    s.step(1, dt)
    ref2, _ = s.get_state()
    qa = torch.from_numpy(q0).cuda()
    qb = torch.empty_like(qa)
    s.step_noalloc(qa, qb, dt)
    torch.cuda.synchronize()
    _compare(qb.cpu().numpy().astype(np.float64), ref1)
    qa.copy_(qb)
    s.step_noalloc(qa, qb, dt)
    torch.cuda.synchronize()
    _compare(qb.cpu().numpy().astype(np.float64), ref2)
    # the context's own state was not touched by the allocation-free calls
    cur, _ = s.get_state()
    np.testing.assert_array_equal(cur, ref2)
    s.close()


def test_noalloc_step_rejects_meshes_beyond_its_scratch():
    import torch

    import paper_2502_09714_gb300 as dgpkg
    from paper_2502_09714_gb300 import DGError
    mesh = periodic_cube_mesh(10, 4000.0)          # 6000 elements > 2772 at N = 4
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, 4, stream=torch.cuda.current_stream())
    s.set_material(rock_material(mesh.n_elem))
    q = torch.zeros((mesh.n_elem, 10, 35), dtype=torch.float32, device="cuda")
    with pytest.raises(DGError) as ei:
        s.step_noalloc(q, q, 0.0)
    assert ei.value.name == "DG_E_ARG" and "2772-element capacity" in str(ei.value)
    s.close()


def test_noalloc_step_runs_the_picard_predictor():
    """With the Picard predictor selected the allocation-free step runs its
    iterations too (in place on the predictor output) and matches dg_step."""
    import torch

    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    N = 2
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=11)
    mat = rock_material(mesh.n_elem, cd=2e-6)
    E, L = mesh.n_elem, dgpkg.n_modes(N)
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, stream=torch.cuda.current_stream())
    s.set_material(mat)
    s.set_predictor("picard", 2)
    q0 = _state(E, L, seed=4)
    dt = s.dt
    s.set_state(q0)
    s.step(1, dt)
    ref, _ = s.get_state()
    qa = torch.from_numpy(q0).cuda()
    qb = torch.empty_like(qa)
    s.step_noalloc(qa, qb, dt)
    torch.cuda.synchronize()
    _compare(qb.cpu().numpy().astype(np.float64), ref)
    # and the Picard result differs from the CK one (the iterations did run)
    s.set_predictor("ck")
    s.set_state(q0)
    s.step(1, dt)
    ck, _ = s.get_state()
    assert np.abs(ck - ref).max() > 0
    s.close()
