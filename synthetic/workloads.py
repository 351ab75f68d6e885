"""Seeded workload descriptions (materials, point sources, receivers).

Material rows are (rho, lambda0, mu0, gamma_r, xi0, C_d) in SI units, C_d in
1/(Pa s).  Field order of the state vector u is
(eps_xx, eps_yy, eps_zz, eps_xy, eps_yz, eps_zx, v_x, v_y, v_z, alpha), with
tensor (not engineering) shear strains.

Workloads:
  c1  periodic 4 km cube, 4^3 x 6 = 384 tets, N=2, homogeneous rock, plane P-wave.
  c2  periodic 4 km cube, 32^3 x 6 = 196,608 tets, +-10% jitter (seed 1), N=4,
      soft 600 m top layer over a halfspace, 45-degree dip-slip point source
      with a 2 Hz Ricker moment rate, 64 receivers on a jittered 8x8 grid (seed 2).
"""
from __future__ import annotations

import numpy as np

from .mesh import kuhn_box_mesh, periodic_cube_mesh

FIELD_NAMES = ("exx", "eyy", "ezz", "exy", "eyz", "ezx", "vx", "vy", "vz", "alpha")

# damage parameters of the rock (config c1): gamma_r, xi0, C_d [1/(Pa s)]
ROCK_GAMMA_R = 3.7e10
ROCK_XI0 = -0.8
ROCK_CD = 1.0e-4


def rock_material(n_elem, rho=2700.0, lam=32e9, mu=32e9, gamma_r=ROCK_GAMMA_R,
                  xi0=ROCK_XI0, cd=ROCK_CD):
    m = np.empty((n_elem, 6))
    m[:] = (rho, lam, mu, gamma_r, xi0, cd)
    return m


def uniform_material(n_elem, rho, lam, mu, gamma_r, xi0, cd):
    return rock_material(n_elem, rho, lam, mu, gamma_r, xi0, cd)


def lame_from_speeds(vp, vs, rho):
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return lam, mu


def two_layer_material(centroid_z, z_top, layer_thickness, soft=(1500.0, 500.0, 2000.0),
                       hard=(6000.0, 3500.0, 2700.0), xi0=ROCK_XI0, cd=ROCK_CD,
                       gamma_over_mu=ROCK_GAMMA_R / 32e9):
    """Per-element material of a soft top layer over a halfspace, chosen by the
    element centroid depth.  gamma_r scales with each layer's mu0 so that the
    soft layer keeps hyperbolicity at the damage levels of the run."""
    n = centroid_z.shape[0]
    m = np.empty((n, 6))
    for (vp, vs, rho), mask in ((hard, centroid_z < z_top - layer_thickness),
                                (soft, centroid_z >= z_top - layer_thickness)):
        lam, mu = lame_from_speeds(vp, vs, rho)
        m[mask] = (rho, lam, mu, gamma_over_mu * mu, xi0, cd)
    return m


def dip_slip_source(x, m0, f0=2.0, t0=0.45):
    """45-degree dip-slip double couple (fault normal (1,0,1)/sqrt2, slip
    (-1,0,1)/sqrt2): moment tensor m0*diag(-1,0,1).  Ricker moment rate with
    peak frequency f0 centred at t0; m0 is the peak moment rate [N m / s]."""
    return {"x": np.asarray(x, dtype=np.float64),
            "m": np.array([-m0, 0.0, m0, 0.0, 0.0, 0.0]),
            "stf": 0, "f0": float(f0), "t0": float(t0)}


def receiver_grid(nx, ny, extent_xy, z, jitter, seed=2):
    rng = np.random.default_rng(seed)
    xs = (np.arange(nx) + 0.5) * extent_xy[0] / nx
    ys = (np.arange(ny) + 0.5) * extent_xy[1] / ny
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.full(nx * ny, float(z))], axis=1)
    pts[:, :2] += rng.uniform(-jitter, jitter, size=(nx * ny, 2))
    return pts


def workload_c1(damage=True, sort_by_vid=False):
    """384-tet periodic cube, N=2, homogeneous rock; plane P-wave along x with
    strain amplitude 1e-4 and wavelength equal to the 4 km cube."""
    mesh = periodic_cube_mesh(4, 4000.0, jitter=0.0, sort_by_vid=sort_by_vid)
    mat = rock_material(mesh.n_elem, cd=ROCK_CD if damage else 0.0)
    return {"name": "c1 periodic cube 384 tets N=2", "mesh": mesh, "material": mat,
            "order": 2, "cfl": 0.5, "steps": 20,
            "plane_wave": {"amplitude": 1e-4, "k": 2.0 * np.pi / 4000.0, "kind": "P"}}


# peak moment rate of the c2 point source [N m/s]; sets the peak strain near
# the source to the 1e-3 range on the 125 m mesh
C2_M0 = 4.0e14


def workload_c2(n=32, side=4000.0, order=4, m0=C2_M0, sort_by_vid=True):
    """The 196,608-tet (n=32) jittered two-layer cube with a point source and
    64 receivers.  Smaller n gives the same workload at a smaller size."""
    mesh = periodic_cube_mesh(n, side, jitter=0.1, seed=1, sort_by_vid=sort_by_vid)
    cz = mesh.centroids()[:, 2]
    mat = two_layer_material(cz, z_top=side, layer_thickness=600.0 * side / 4000.0)
    src = dip_slip_source([0.5 * side, 0.5 * side, 0.75 * side], m0)
    h = side / n
    rec = receiver_grid(8, 8, (side, side), z=0.975 * side, jitter=min(0.5 * h, side / 32.0), seed=2)
    return {"name": f"c2 jittered two-layer cube {mesh.n_elem} tets N={order}",
            "mesh": mesh, "material": mat, "order": order, "cfl": 0.5, "steps": 500,
            "sources": [src], "receivers": rec}


def workload_c4(n=32, side=4000.0, order=3, members=32, seed=3, sort_by_vid=True):
    """The ensemble workload: c2's mesh, layers, source and receivers at degree
    3, with `members` parameter sets drawn per member (seeded):
    xi0 ~ U[-1.0, -0.6] and log C_d ~ U[log 1e-5, log 1e-3], C_d in 1/(Pa s).
    member_xi0_cd has the C-ABI layout [members][n_elem][2]."""
    w = workload_c2(n=n, side=side, order=order, sort_by_vid=sort_by_vid)
    rng = np.random.default_rng(seed)
    xi0 = rng.uniform(-1.0, -0.6, size=members)
    cd = np.exp(rng.uniform(np.log(1e-5), np.log(1e-3), size=members))
    E = w["mesh"].n_elem
    par = np.empty((members, E, 2))
    par[:, :, 0] = xi0[:, None]
    par[:, :, 1] = cd[:, None]
    w.update(name=f"c4 ensemble of {members} on the {E}-tet two-layer cube N={order}",
             members=members, member_xi0_cd=par)
    return w


def workload_small_layered(n=4, order=3, side=4000.0, m0=C2_M0, seed=1, sort_by_vid=False):
    """A c2-shaped workload at a size the oracle runs in seconds."""
    w = workload_c2(n=n, side=side, order=order, m0=m0, sort_by_vid=sort_by_vid)
    if seed != 1:
        w["mesh"] = periodic_cube_mesh(n, side, jitter=0.1, seed=seed, sort_by_vid=sort_by_vid)
        cz = w["mesh"].centroids()[:, 2]
        w["material"] = two_layer_material(cz, z_top=side, layer_thickness=600.0 * side / 4000.0)
    return w


# 1-D Riemann problem of the nonlinear shear law (Sec. 3.1): rho = mu = 1 and beta = 10
# as the paper sets them, lambda0 = 1 (not stated; it only sets the P speed), and a
# strain step at rest (eps_xy 0.01 | 0.02), inside the hyperbolic range of the law
RIEMANN_LEFT = (0.01, 0.0)      # (eps_xy, v_y) for x < 0
RIEMANN_RIGHT = (0.02, 0.0)     # (eps_xy, v_y) for x >= 0
RIEMANN_MATERIAL = (1.0, 1.0, 1.0, 10.0)   # rho, lambda0, mu0, beta


def workload_riemann(nx, order=2, half_length=1.2, t_end=0.5):
    """Quasi-1-D mesh for the plane shear Riemann problem: nx cells on
    [-half_length, half_length] in x (x = 0 a grid plane), 3 cells of the same
    width in y and z, periodic in all three directions, Kuhn 6-tet split.  The
    periodic seam at x = +-half_length starts a second wave fan; with speeds
    below 1 neither fan reaches |x| < half_length - t_end before t_end, the
    window `eval_half_width` where the solution is compared."""
    h = 2.0 * half_length / nx
    xs = np.linspace(-half_length, half_length, nx + 1)
    yz = np.linspace(0.0, 3.0 * h, 4)
    mesh = kuhn_box_mesh(xs, yz, yz, periodic=(True, True, True), sort_by_vid=True)
    mat = np.zeros((mesh.n_elem, 6))
    mat[:, :4] = RIEMANN_MATERIAL
    return {"name": f"plane shear Riemann problem nx={nx} N={order}", "mesh": mesh, "material": mat,
            "order": order, "left": RIEMANN_LEFT, "right": RIEMANN_RIGHT, "t_end": t_end, "h": h,
            "eval_half_width": half_length - t_end - 0.1}


def workload_adjoint(n=24, side=4000.0, order=3, n_receivers=32, steps=800, m0=C2_M0, seed=5):
    """The adjoint workload: a periodic jittered cube of n^3 x 6 tets (82,944 at
    n = 24) at degree 3 in homogeneous rock, the c2 dip-slip point source, 32
    receivers on a jittered 4 x 8 grid at three quarters of the height, and
    per-element damage parameters drawn with `seed`: xi0 ~ U[-1.0, -0.6] and
    log C_d ~ U[log 2e-6, log 2e-5] ("material"), which keeps the damage near the
    source below ~0.3 over the 800 steps.  The reference run that makes
    the traces to be fitted uses "material_ref": xi0 + 0.05 N(0, 1) and
    C_d exp(0.3 N(0, 1)), drawn with seed + 1.  The run starts from rest at
    t_start = 0.3 s, so that the whole Ricker pulse (peak at 0.45 s), the damage
    it drives and the waves scattered by that damage fall inside the 800 steps."""
    mesh = periodic_cube_mesh(n, side, jitter=0.1, seed=1, sort_by_vid=True)
    E = mesh.n_elem
    rng = np.random.default_rng(seed)
    mat = rock_material(E)
    mat[:, 4] = rng.uniform(-1.0, -0.6, size=E)
    mat[:, 5] = np.exp(rng.uniform(np.log(2e-6), np.log(2e-5), size=E))
    rng2 = np.random.default_rng(seed + 1)
    ref = mat.copy()
    ref[:, 4] += 0.05 * rng2.normal(size=E)
    ref[:, 5] *= np.exp(0.3 * rng2.normal(size=E))
    src = dip_slip_source([0.5 * side, 0.5 * side, 0.5 * side], m0)
    h = side / n
    rec = receiver_grid(4, 8, (side, side), z=0.75 * side, jitter=min(0.5 * h, side / 32.0), seed=seed + 2)
    return {"name": f"c5 adjoint on the {E}-tet jittered cube N={order}", "mesh": mesh,
            "material": mat, "material_ref": ref, "order": order, "cfl": 0.5, "steps": steps,
            "snapshots": 40, "sources": [src], "receivers": rec[:n_receivers], "t_start": 0.3}
