"""The failure path of the bounded waits of the tensor-core kernels (predictor and
corrector), run without any fault: with a wait limit of 0 polls, the first wait on
the matrix products gives up at once.  Each kernel must then stop, drain its
products in flight with the default limit, free its tensor memory and return;
dg_step reports DG_E_CUDA ("timed out") and the context stays usable: the next step
at the default limit matches the oracle."""
import numpy as np
import pytest

from oracle import from_abi, to_abi
from synthetic import periodic_cube_mesh, rock_material

from parity_util import TOL_ALPHA, TOL_REL_L2, alpha_max_diff, make_oracle, make_solver, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [2, 3, 4])
def test_wait_timeout_is_reported_and_the_context_recovers(N):
    import paper_2502_09714_gb300 as dgpkg
    from paper_2502_09714_gb300 import DGError
    dgpkg.build()
    mesh = periodic_cube_mesh(3, 4000.0, jitter=0.1, seed=21)
    mat = rock_material(mesh.n_elem, cd=2e-6)
    o = make_oracle(mesh, mat, N)
    rng = np.random.default_rng(N)
    Q0 = rng.normal(size=(mesh.n_elem, o.L, 10)) * 1e-5
    Q0[..., 6:9] *= 3000.0
    Q0[..., 9] = 0.0
    dt = o.cfl_dt()
    s = make_solver(mesh, mat, N)
    s.set_state(to_abi(Q0))
    s.set_wait_limit(0)
    with pytest.raises(DGError) as ei:
        s.step(1, dt)
    assert ei.value.name == "DG_E_CUDA" and "timed out" in str(ei.value)
    # the context and the GPU are still usable: restore the state and step again
    s.set_wait_limit(-1)
    s.set_state(to_abi(Q0))
    s.step(2, dt)
    q, _ = s.get_state()
    Q = o.run(Q0, dt, 2)
    errs = rel_l2(to_abi(from_abi(q) - Q0), Q - Q0, o.detJ)
    for name, e in errs.items():
        assert e <= TOL_REL_L2, (name, e)
    assert alpha_max_diff(q, Q, N) <= TOL_ALPHA
    s.close()


def test_wait_limit_arguments():
    import paper_2502_09714_gb300 as dgpkg
    from paper_2502_09714_gb300 import DGError
    mesh = periodic_cube_mesh(3, 4000.0)
    s = make_solver(mesh, rock_material(mesh.n_elem), 2)
    s.set_wait_limit(1 << 20)
    s.set_wait_limit(-5)
    with pytest.raises(DGError) as ei:
        s.set_wait_limit(1 << 40)
    assert ei.value.name == "DG_E_ARG"
    s.close()
