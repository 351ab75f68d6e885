"""Helpers shared by the GPU parity tests: run the same seeded workload
through libdg (C-ABI) and through the FP64 oracle, and compare."""
from __future__ import annotations

import math

import numpy as np

from oracle import Oracle, eval_basis, from_abi, tet_rule, to_abi

# parity tolerances: relative L2 per field group, absolute on damage
TOL_REL_L2 = 1e-4
TOL_ALPHA = 1e-5
GROUPS = {"strain": slice(0, 6), "velocity": slice(6, 9)}


def _tags(mesh):
    bc = getattr(mesh, "face_bc", None)
    return bc if bc is not None and np.any(bc != 0) else None


def make_solver(mesh, material, order, cfl=0.5, sources=(), receivers=None, stream=None):
    import paper_2502_09714_gb300 as dgpkg
    s = dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, order, face_bc=_tags(mesh), cfl=cfl, stream=stream)
    s.set_material(material)
    if sources:
        s.set_sources(list(sources))
    if receivers is not None:
        s.set_receivers(receivers)
    return s


def make_oracle(mesh, material, order, cfl=0.5, sources=(), receivers=None, face_rows=None):
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, order, material, face_bc=_tags(mesh), cfl=cfl,
               face_rows=face_rows)
    if sources:
        o.set_sources(list(sources))
    if receivers is not None:
        o.set_receivers(receivers)
    return o


def rel_l2(q_gpu_abi, Q_ora, detJ, rows=None):
    """Relative L2 (modal coefficients weighted by |J|, orthonormal basis) per
    field group; q_gpu_abi in the ABI layout [E,10,L], Q_ora in [E,L,10]."""
    G = from_abi(q_gpu_abi)
    if rows is not None:
        G, Q_ora, detJ = G[rows], Q_ora[rows] if Q_ora.shape[0] != len(rows) else Q_ora, detJ[rows]
    w = detJ[:, None, None]
    out = {}
    for name, sl in GROUPS.items():
        num = np.sum(w * (G[..., sl] - Q_ora[..., sl]) ** 2)
        den = np.sum(w * Q_ora[..., sl] ** 2)
        out[name] = math.sqrt(num / den) if den > 0 else math.sqrt(num)
    return out


def alpha_max_diff(q_gpu_abi, Q_ora, order):
    """max over elements and volume nodes of |alpha_gpu - alpha_oracle|."""
    pts, _ = tet_rule(order + 1)
    V = eval_basis(order, pts)
    G = from_abi(q_gpu_abi)
    return float(np.max(np.abs(np.einsum("ql,el->eq", V, G[..., 9] - Q_ora[..., 9]))))


def assert_parity(q_gpu_abi, Q_ora, detJ, order, rel=TOL_REL_L2, alpha=TOL_ALPHA):
    errs = rel_l2(q_gpu_abi, Q_ora, detJ)
    da = alpha_max_diff(q_gpu_abi, Q_ora, order)
    for name, e in errs.items():
        assert e <= rel, f"{name} rel L2 {e:.3e} > {rel:.1e}"
    assert da <= alpha, f"alpha max diff {da:.3e} > {alpha:.1e}"
    return errs, da


__all__ = ["make_solver", "make_oracle", "rel_l2", "alpha_max_diff", "assert_parity", "to_abi",
           "from_abi", "TOL_REL_L2", "TOL_ALPHA"]


def face_neighbours(mesh):
    """[E, 4] element across each face (the face opposite local vertex f), -1 on
    boundary faces: vertex-id triples matched with one sort (no oracle code)."""
    vid = np.asarray(mesh.elem_vid)
    E = vid.shape[0]
    keys = np.empty((4 * E, 3), dtype=np.int64)
    for f in range(4):
        keys[f::4] = np.sort(np.delete(vid, f, axis=1), axis=1)
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    ks = keys[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    nbr = -np.ones(4 * E, dtype=np.int64)
    i = np.nonzero(same)[0]
    a, b = order[i], order[i + 1]
    nbr[a] = b // 4
    nbr[b] = a // 4
    return nbr.reshape(E, 4)


def submesh_oracle(mesh, material, order, rows, sources=(), law="cdm", cfl=0.5):
    """An oracle over `rows` and their face neighbours only, for stepping `rows`
    of a mesh too large for the oracle: faces of the neighbours that leave the
    sub-mesh are tagged absorbing (they only enter the neighbours' own updates,
    which are not compared).  Returns (oracle, element ids of the sub-mesh in
    global order, positions of `rows` in it).  Sources outside the sub-mesh are
    dropped."""
    from oracle import MeshError, Oracle
    nbr = face_neighbours(mesh)
    rows = np.unique(np.asarray(rows))
    nb = nbr[rows].ravel()
    elems = np.unique(np.concatenate([rows, nb[nb >= 0]]))
    pos = -np.ones(mesh.n_elem, dtype=np.int64)
    pos[elems] = np.arange(elems.size)
    bc = np.array(mesh.face_bc[elems], dtype=np.int8)
    inner = nbr[elems]
    leaving = (inner >= 0) & (pos[np.maximum(inner, 0)] < 0)
    bc[leaving] = 2
    o = Oracle(mesh.elem_xyz[elems], mesh.elem_vid[elems], order, material[elems], face_bc=bc, cfl=cfl,
               face_rows=pos[rows], law=law)
    kept = []
    for s in sources:
        try:
            o.locate(s["x"])
            kept.append(s)
        except MeshError:
            pass
    if kept:
        o.set_sources(kept)
    return o, elems, pos[rows]


# ---- a pool of oracle processes for long runs ----------------------------------
# Each worker holds its own Oracle of the whole mesh and steps one chunk of the
# elements; the parent gathers the chunks into the next state.  The pool is
# started with "spawn" (a worker forked from a process that has touched CUDA can
# hang), and each worker's BLAS is pinned to one thread.

_POOL_ORACLE = None


_ONE_THREAD = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _pool_init(args):
    global _POOL_ORACLE
    mesh_xyz, mesh_vid, face_bc, order, material, cfl, sources, receivers = args
    _POOL_ORACLE = Oracle(mesh_xyz, mesh_vid, order, material, face_bc=face_bc, cfl=cfl)
    if sources:
        _POOL_ORACLE.set_sources(list(sources))
    if receivers is not None:
        _POOL_ORACLE.set_receivers(receivers)


def _pool_step(job):
    Q, dt, t, rows = job
    return _POOL_ORACLE.step(Q, dt, t, rows=rows)


def oracle_run_pool(mesh, material, order, Q0, dt, n_steps, t0=0.0, cfl=0.5, sources=(), receivers=None,
                    workers=None):
    """The oracle's run (the same Oracle.step per element, chunked over processes).
    Returns the final state and, with receivers, the traces after every step."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    o = make_oracle(mesh, material, order, cfl=cfl, sources=sources, receivers=receivers)
    chunks = np.array_split(np.arange(mesh.n_elem), workers)
    init = (mesh.elem_xyz, mesh.elem_vid, _tags(mesh), order, material, cfl, list(sources), receivers)
    Q, t, traces = np.array(Q0, dtype=np.float64), t0, []
    saved = {k: os.environ.get(k) for k in _ONE_THREAD}
    os.environ.update({k: "1" for k in _ONE_THREAD})       # inherited by the workers at spawn
    try:
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"), initializer=_pool_init,
                                    initargs=(init,)) as ex:
            for _ in range(n_steps):
                parts = list(ex.map(_pool_step, [(Q, dt, t, c) for c in chunks]))
                Q = np.concatenate(parts, axis=0)
                t += dt
                if receivers is not None:
                    traces.append(o.sample_receivers(Q))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return (Q, np.array(traces)) if receivers is not None else Q


def _misfit_job(job):
    from oracle.adjoint import misfit
    xyz, vid, order, mat, sources, receivers, Q0, dt, n, ref, t0 = job
    o = Oracle(xyz, vid, order, mat)
    if sources:
        o.set_sources(list(sources))
    o.set_receivers(receivers)
    return misfit(o, Q0, dt, n, ref, t0=t0)[0]


def misfit_pool(mesh, order, materials, sources, receivers, Q0, dt, n_steps, ref, t0=0.0, workers=None):
    """The oracle's receiver misfit (oracle.adjoint.misfit) of one run per material
    table, the runs spread over spawn-started processes with one BLAS thread each."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    workers = workers or max(1, min(16, os.cpu_count() or 1, len(materials)))
    jobs = [(mesh.elem_xyz, mesh.elem_vid, order, m, list(sources), receivers, Q0, dt, n_steps, ref, t0)
            for m in materials]
    saved = {k: os.environ.get(k) for k in _ONE_THREAD}
    os.environ.update({k: "1" for k in _ONE_THREAD})
    try:
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_misfit_job, jobs))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
