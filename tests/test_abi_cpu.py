"""CPU checks of the C-ABI library: it builds, loads and exports every entry
point of include/dg.h; its host-side reference tables (computed in C++,
independently of the oracle) are exact quadratures and the same Dubiner basis;
mesh validation errors are reported before any device work."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_2502_09714_gb300 as dgpkg
from paper_2502_09714_gb300.dg import EXPORTS, DGError
from oracle import eval_basis, n_modes
from synthetic import periodic_cube_mesh
from synthetic.mesh import kuhn_box_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    dgpkg.build()
    return dgpkg.load_library()


def test_library_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "dg.h")).read()
    declared = set(re.findall(r"^\s*(?:dg_status|double|int64_t|int|const char\s*\*|void)\s+(dg_\w+)\s*\(",
                              header, flags=re.M))
    assert declared, "no declarations found"
    assert declared == set(EXPORTS)
    raw = ctypes.CDLL(dgpkg.LIB_PATH)
    for name in declared:
        assert hasattr(raw, name), name


def _check_chunk_plan(E, b):
    r16 = lambda x: (x + 15) // 16 * 16
    sizes = np.diff(b)
    assert b[0] == 0 and b[-1] == E, (E, b)
    assert np.all(sizes > 0), (E, b)
    assert np.all(b[1:-1] % 16 == 0), (E, b)
    assert len(sizes) <= 9, (E, b)
    if E <= 3 * 4096:                                 # chunks of 4096, the last shorter
        assert np.all(sizes[:-1] == 4096) and sizes[-1] <= 4096, (E, b)
        return
    edge = r16(max(4096, E // 16))
    assert sizes[0] == edge and edge <= sizes[-1] <= edge + 15, (E, b)
    mid = sizes[1:-1]
    assert 1 <= len(mid) <= 7, (E, b)
    assert np.all(mid[:-1] == mid[0]) and mid[0] % 16 == 0 and mid[0] >= 4096 and mid[-1] <= mid[0], (E, b)


def test_host_step_chunk_plan(lib):
    """The element chunks of dg_step_host: they tile the mesh in order, start on
    multiples of 16, and take the documented sizes (small first and last chunks,
    up to seven equal ones between), over sizes around every branch and random
    ones up to the 2^29 copies the library admits."""
    for E in (1, 15, 16, 17, 4095, 4096, 4097, 8192, 12287, 12288, 12289, 13182, 65535, 65536, 65537,
              196608, 4350240, (1 << 29) - 1):
        _check_chunk_plan(E, dgpkg.host_chunks(E))
    rng = np.random.default_rng(1)
    for E in rng.integers(1, 1 << 29, size=2000):
        _check_chunk_plan(int(E), dgpkg.host_chunks(int(E)))
    # the count comes back without a buffer, and bad arguments are refused
    assert lib.dg_host_chunks(4350240, None, 0) == 9
    assert lib.dg_host_chunks(0, None, 0) == -1
    assert lib.dg_host_chunks(100, None, 3) == -1
    with pytest.raises(DGError):
        dgpkg.host_chunks(0)


def test_n_modes(lib):
    for N in range(0, 7):
        assert lib.dg_n_modes(N) == (N + 1) * (N + 2) * (N + 3) // 6


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_host_volume_rule_exact(lib, N):
    t = dgpkg.reference_table(N, 0).reshape(-1, 4)
    assert t.shape[0] == (N + 1) ** 3
    n = N + 1
    for a in range(2 * n):
        for b in range(2 * n - a):
            for c in range(2 * n - a - b):
                want = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = np.sum(t[:, 3] * t[:, 0] ** a * t[:, 1] ** b * t[:, 2] ** c)
                assert got == pytest.approx(want, rel=1e-12, abs=1e-16)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_host_face_and_time_rules_exact(lib, N):
    f = dgpkg.reference_table(N, 1).reshape(-1, 3)
    n = N + 1
    for a in range(2 * n):
        for b in range(2 * n - a):
            want = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert 0.5 * np.sum(f[:, 2] * f[:, 0] ** a * f[:, 1] ** b) == pytest.approx(want, rel=1e-12)
    t = dgpkg.reference_table(N, 2).reshape(-1, 2)
    for d in range(2 * n):
        assert np.sum(t[:, 1] * t[:, 0] ** d) == pytest.approx(1.0 / (d + 1), rel=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_host_basis_is_the_abi_basis(lib, N):
    """The library's Dubiner basis (values and gradients) equals the oracle's at
    the library's own volume nodes: the state ABI means the same thing on both sides."""
    nodes = dgpkg.reference_table(N, 0).reshape(-1, 4)
    L = n_modes(N)
    V = dgpkg.reference_table(N, 3).reshape(-1, L)
    G = dgpkg.reference_table(N, 4).reshape(-1, L, 3)
    Vo, Go = eval_basis(N, nodes[:, :3], grad=True)
    np.testing.assert_allclose(V, Vo, atol=1e-12 * np.abs(Vo).max())
    np.testing.assert_allclose(G, Go, atol=1e-11 * np.abs(Go).max())
    M = V.T @ (nodes[:, 3:4] * V)
    np.testing.assert_allclose(M, np.eye(L), atol=1e-13)


def _create(mesh, order=2, **kw):
    return dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, order, **kw)


def test_mesh_validation_errors_before_device_work(lib):
    mesh = periodic_cube_mesh(3, 4000.0)
    vid = mesh.elem_vid.copy()
    vid[5, 2] = vid[5, 0]
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(mesh.elem_xyz, vid, 2)
    assert ei.value.name == "DG_E_MESH"
    flat = mesh.elem_xyz.copy()
    flat[3, 3] = 0.5 * (flat[3, 0] + flat[3, 1])
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(flat, mesh.elem_vid, 2)
    assert ei.value.name == "DG_E_MESH"
    # dropping one element leaves four faces unmatched
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(mesh.elem_xyz[1:], mesh.elem_vid[1:], 2)
    assert ei.value.name == "DG_E_MESH"
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, 9)
    assert ei.value.name == "DG_E_ORDER"
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, 2, members=0)
    assert ei.value.name == "DG_E_ARG"
    # a tag on a shared face, and an unknown tag, are mesh errors
    bc = np.zeros((mesh.n_elem, 4), np.int8)
    bc[0, 0] = 2
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, 2, face_bc=bc)
    assert ei.value.name == "DG_E_MESH"
    bc[0, 0] = 3
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, 2, face_bc=bc)
    assert ei.value.name == "DG_E_MESH"
    # a closed box with tagged outer faces passes validation (on a machine
    # without a GPU the first device allocation is what fails)
    g = np.linspace(0.0, 4000.0, 3)
    box = kuhn_box_mesh(g, g, g, periodic=(False, False, True), jitter=0.1)
    try:
        dgpkg.Solver(box.elem_xyz, box.elem_vid, 2, face_bc=box.face_bc)
    except DGError as err:
        assert err.name != "DG_E_MESH", str(err)
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(box.elem_xyz, box.elem_vid, 2)       # outer faces untagged
    assert ei.value.name == "DG_E_MESH"
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(mesh.elem_xyz[:0], mesh.elem_vid[:0], 2)
    assert ei.value.name == "DG_E_ARG"
    with pytest.raises(DGError) as ei:
        dgpkg.Solver(mesh.elem_xyz, mesh.elem_vid, 2, cfl=-1.0)
    assert ei.value.name == "DG_E_ARG"
