"""The regional-shaped workload at full size (~4.35 M tets, N=4): graded box,
basin, layered background, free surface on top and absorbing elsewhere, about
6000 sub-fault sources and 64 surface receivers, in the launch configuration of
the benchmark.  20 GPU steps from the middle of the rupture, then one more GPU
step against the oracle's step from the GPU state on sampled elements (near the
hypocentre, on the free surface, on absorbing faces, in the basin, at random);
the bar applies to the step's change of the state."""
import numpy as np
import pytest

from oracle import from_abi, to_abi
from synthetic.regional import workload_c3

from parity_util import TOL_ALPHA, TOL_REL_L2, alpha_max_diff, rel_l2, submesh_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_2502_09714_gb300 as dgpkg
    dgpkg.build()
    dgpkg.load_library()


def test_regional_sampled_step():
    import paper_2502_09714_gb300 as dgpkg
    w = workload_c3()
    mesh, mat, N = w["mesh"], w["material"], w["order"]
    E = mesh.n_elem
    assert 3.99e6 <= E <= 4.41e6
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, N, face_bc=mesh.face_bc, cfl=w["cfl"])
    s.set_material(mat)
    s.set_sources(w["sources"])
    s.set_receivers(w["receivers"])
    t0 = 0.8                                        # the rupture has started around the hypocentre
    s.set_state(np.zeros((E, 10, 35), np.float32), t0)
    s.step(20)
    qa, ta = s.get_state()
    assert np.isfinite(qa).all()
    # the peak strain stays in the range the sources were scaled for
    assert np.abs(qa[:, 0:6, 0]).max() * np.sqrt(6.0) < 1e-2
    tr = s.read_receivers()
    assert tr.shape == (20, 64, 3) and np.isfinite(tr).all()
    # samples
    rng = np.random.default_rng(6)
    energy = np.abs(qa[:, 6:9]).reshape(E, -1).max(axis=1)
    hot = np.argsort(energy)[-24:]
    free = np.nonzero((mesh.face_bc == 1).any(axis=1))[0]
    absorb = np.nonzero((mesh.face_bc == 2).any(axis=1))[0]
    basin = np.nonzero(w["basin"])[0]
    rows = np.unique(np.concatenate([hot, rng.choice(free, 8, replace=False), rng.choice(absorb, 8, replace=False),
                                     rng.choice(basin, 8, replace=False), rng.choice(E, 8, replace=False)]))
    o, elems, rpos = submesh_oracle(mesh, mat, N, rows, sources=w["sources"])
    assert len(o.sources) > 0
    dt = s.dt
    s.step(1)
    qb, _ = s.get_state()
    Qa = from_abi(qa[elems])
    Qb = o.step(Qa, dt, ta, rows=rpos)
    # compare the step's change of the state (what the step computes), per field group
    dO = Qb - Qa[rpos]
    dG = to_abi(from_abi(qb[rows]) - Qa[rpos])
    assert np.abs(dO).max() > 0
    errs = rel_l2(dG, dO, o.detJ[rpos])
    for name, e in errs.items():
        assert e <= TOL_REL_L2, (name, e)
    assert alpha_max_diff(qb[rows], Qb, N) <= TOL_ALPHA
