"""P6: stress- and damage-induced anisotropy (Sec. 3.3).  With the parameters of
the paper's CDM table (tests/golden/cdm_table_paper.txt) a uniform pre-strain
(1e-3 along a principal axis rotated about z) and damage alpha = 0.5, a small
plane perturbation along x travels at the speeds given by the acoustic tensor
Gamma_il = C_ixxl / rho of the tangent stiffness C = d sigma / d eps at the
pre-strain.  The oracle's wave speeds, measured by phase tracking, must match
those speeds and not the isotropic effective speeds of its predictor's
Jacobian (reading R1), which differ by about 16 % for the P wave here."""
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from oracle.rheology import cdm_stress, effective_lame
from synthetic.mesh import kuhn_box_mesh

SYM = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cdm_table_paper.txt")


def _table():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _pre_state(t, phi):
    c, s = math.cos(phi), math.sin(phi)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    E = R @ np.diag([t["pre_strain_xx"], 0.0, 0.0]) @ R.T
    u = np.zeros(10)
    for p, (i, j) in enumerate(SYM):
        u[p] = E[i, j]
    u[9] = t["alpha0"]
    return u


def _acoustic_tensor(u0, mat):
    """Gamma_il = C_ixxl / rho by central differences of the stress along the
    symmetric strain directions sym(e_x e_l)."""
    h = 1e-9
    G = np.zeros((3, 3))
    for l in range(3):
        dE = np.zeros((3, 3))
        dE[0, l] += 0.5
        dE[l, 0] += 0.5
        du = np.zeros(10)
        for p, (i, j) in enumerate(SYM):
            du[p] = dE[i, j]
        G[:, l] = (cdm_stress(u0 + h * du, mat)[:, 0] - cdm_stress(u0 - h * du, mat)[:, 0]) / (2 * h) / mat[0]
    return 0.5 * (G + G.T)


def _measured_speed(t, phi, mode, n=4, N=2, frac=0.25):
    mat1 = np.array([t["rho"], t["lambda0"], t["mu0"], t["gamma_r"], t["xi0"], t["Cd"]])
    u0 = _pre_state(t, phi)
    w, V = np.linalg.eigh(_acoustic_tensor(u0, mat1))
    c_ana, a = math.sqrt(w[mode]), V[:, mode]
    k, A0 = t["k"], t["A0"]
    Lx = 1.0 / k                                        # one wavelength of sin(2 pi k x)
    grids = [np.linspace(0.0, Lx, n + 1)] + [np.linspace(0.0, 3 * Lx / n, 4)] * 2
    mesh = kuhn_box_mesh(*grids, periodic=(True, True, True), jitter=0.1, seed=5)
    o = Oracle(mesh.elem_xyz, mesh.elem_vid, N, np.tile(mat1, (mesh.n_elem, 1)))
    Edyn = 0.5 * (np.outer([1.0, 0.0, 0.0], a) + np.outer(a, [1.0, 0.0, 0.0]))

    def init(x):
        g = A0 * np.sin(2 * np.pi * k * x[..., 0])
        u = np.broadcast_to(u0, x.shape[:-1] + (10,)).copy()
        for p, (i, j) in enumerate(SYM):
            u[..., p] += Edyn[i, j] * g
        u[..., 6:9] += -c_ana * a * g[..., None]         # right-going wave along +x
        return u
    Q = o.project(init)
    T = frac * Lx / c_ana
    n_steps = int(math.ceil(T / o.cfl_dt()))
    for _ in range(n_steps):
        Q = o.step(Q, T / n_steps)
    # phase of the velocity perturbation along a: v.a = -c A0 sin(2 pi k (x - c t))
    rng = np.random.default_rng(1)
    xs, vs = [], []
    for e in range(mesh.n_elem):
        x = rng.dirichlet(np.ones(4), size=3) @ mesh.elem_xyz[e]
        xs.append(x[:, 0])
        vs.append(o.evaluate_at(Q, e, x)[:, 6:9] @ a)
    xs, vs = np.concatenate(xs), np.concatenate(vs)
    M = np.stack([np.sin(2 * np.pi * k * xs), np.cos(2 * np.pi * k * xs), np.ones_like(xs)], axis=1)
    coef, *_ = np.linalg.lstsq(M, vs, rcond=None)
    theta = math.atan2(coef[1], -coef[0])
    c_num = theta / (2 * np.pi * k * T)
    lam, mu = effective_lame(u0, mat1)
    c_iso = (math.sqrt((lam + 2 * mu) / mat1[0]), math.sqrt(mu / mat1[0]))
    return c_ana, c_num, c_iso


def test_table_matches_the_paper_values():
    t = _table()
    assert t["Cd"] == 0.0 and t["alpha0"] == 0.5 and t["xi0"] == -0.75


@pytest.mark.parametrize("mode,name", [(2, "P"), (1, "qS"), (0, "S")])
def test_anisotropic_wave_speeds(mode, name):
    """Pre-strain rotated by 30 degrees about z: each of the three plane waves
    along x travels at its acoustic-tensor speed to within 0.3 %."""
    t = _table()
    c_ana, c_num, c_iso = _measured_speed(t, math.radians(30.0), mode)
    assert abs(c_num - c_ana) <= 3e-3 * c_ana, (name, c_ana, c_num)
    if name == "P":
        # the P speed is far from the isotropic effective P speed the predictor uses
        assert abs(c_iso[0] - c_ana) > 0.1 * c_ana
        assert abs(c_num - c_ana) < 0.02 * abs(c_iso[0] - c_ana)
