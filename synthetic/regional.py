"""Regional-shaped synthetic workload: a graded box with a sedimentary basin, a
layered background, free surface on top, absorbing sides and bottom, a
kinematic finite fault made of sub-fault point sources, and surface receivers.
It stands in for the paper's Gorkha runs (whose datasets are not available)
with their element type, degree, boundary mix, material contrast and source
style; everything is seeded.  Nothing here evaluates the numerical method.

Layout (km): x in [0, 120] (fault strike), y in [0, 80], z in [-40, 0], the
free surface at z = 0.
"""
from __future__ import annotations

import math

import numpy as np

from .mesh import FACE_BC_ABSORBING, FACE_BC_FREE_SURFACE, kuhn_box_mesh
from .workloads import ROCK_CD, ROCK_GAMMA_R, ROCK_XI0, lame_from_speeds

# background units 2-5 of the paper's velocity model (Sec. 4.1 table): depth range [km], vp, vs, rho
UNITS = ((0.0, 3.0, 5500.0, 3250.0, 2700.0),
         (3.0, 23.0, 5502.0, 3600.0, 2700.0),
         (23.0, 45.0, 6100.0, 3600.0, 2900.0),
         (45.0, 200.0, 8100.0, 4500.0, 3300.0))
BASIN = (450.0, 300.0, 1400.0)          # vp = 1.5 vs, rho of unit 1


def graded_axis(lo, hi, a, b, h_fine, h_max, growth):
    """Grid lines on [lo, hi]: spacing h_fine on [a, b], growing outward by at
    most `growth` per cell up to h_max, the outer cells scaled to end on lo/hi."""
    n_f = max(1, int(round((b - a) / h_fine)))
    core = np.linspace(a, b, n_f + 1)

    def outward(dist):
        if dist <= 0:
            return np.zeros(0)
        h, acc, hs = h_fine, 0.0, []
        while acc < dist:
            h = min(h * growth, h_max)
            hs.append(h)
            acc += h
        return np.array(hs) * (dist / acc)
    left = outward(a - lo)
    right = outward(hi - b)
    xs = np.concatenate([a - np.cumsum(left)[::-1], core, b + np.cumsum(right)])
    xs[0], xs[-1] = lo, hi
    return xs


def fault_sources(mu_of_depth, seed=4, length_km=120.0, width_km=50.0, dip_deg=7.0, top_y_km=15.0,
                  top_z_km=-2.0, sub_km=1.0, max_slip=0.15, v_rupture=2800.0, sigma=0.25):
    """Sub-fault point sources of a planar thrust fault (strike along x, dipping
    toward +y, rake 90 degrees): moment tensors mu A s (n u^T + u n^T) with a
    seeded smooth slip field rescaled to [0, max_slip] m, Gaussian moment rates
    of standard deviation sigma centred at the rupture time from the fault
    centre (speed v_rupture) plus 3 sigma.  The default peak slip of 0.15 m
    keeps the strain that one sub-fault puts into its host element (about
    A s / V for element volume V) near 1e-3, the level of the c2 source: the
    paper's metres of slip, concentrated by point sources into single elements
    of 0.3-1.2 km, would drive the damage past hyperbolicity within a step."""
    rng = np.random.default_rng(seed)
    ns, nd = int(round(length_km / sub_km)), int(round(width_km / sub_km))
    # smooth random slip: white noise low-passed in the Fourier domain
    w = rng.normal(size=(ns, nd))
    kx = np.fft.fftfreq(ns)[:, None]
    ky = np.fft.fftfreq(nd)[None, :]
    field = np.real(np.fft.ifft2(np.fft.fft2(w) * np.exp(-(kx * kx + ky * ky) / (2 * 0.03 ** 2))))
    slip = (field - field.min()) / (field.max() - field.min()) * max_slip
    dip = math.radians(dip_deg)
    c, s = math.cos(dip), math.sin(dip)
    n = np.array([0.0, s, c])                 # fault normal into the hanging wall
    u = np.array([0.0, -c, s])                # up-dip slip of the hanging wall
    T = np.outer(n, u) + np.outer(u, n)
    tens = np.array([T[0, 0], T[1, 1], T[2, 2], T[0, 1], T[1, 2], T[2, 0]])
    area = (sub_km * 1e3) ** 2
    hypo_i, hypo_j = (ns - 1) / 2.0, (nd - 1) / 2.0
    out = []
    for i in range(ns):
        for j in range(nd):
            x = (i + 0.5) * sub_km * 1e3
            y = (top_y_km + (j + 0.5) * sub_km * c) * 1e3
            z = (top_z_km - (j + 0.5) * sub_km * s) * 1e3
            dist = math.hypot((i - hypo_i) * sub_km, (j - hypo_j) * sub_km) * 1e3
            m0 = mu_of_depth(-z) * area * slip[i, j]
            out.append({"x": np.array([x, y, z]), "m": m0 * tens, "stf": 1, "sigma": sigma,
                        "t0": dist / v_rupture + 3 * sigma})
    return out


def workload_c3(order=4, h_fine=300.0, h_max=1200.0, growth=1.15, jitter=0.1, seed=1,
                basin_center=(60e3, 40e3), basin_axes=(10e3, 7.5e3, 600.0), sort_by_vid=True):
    """The regional-shaped run: ~4.2 M tets at the default spacings (300 m over
    the 20 x 15 km basin footprint and the top 600 m, growing by at most 1.15 per
    cell to h_max).  Free surface on top, absorbing elsewhere, damage on
    everywhere (gamma_r = 3.7/3.2 mu0, xi0 = -0.8, C_d = 1e-4), ~6000 sub-fault
    sources, 64 surface receivers over the basin."""
    bx, by = basin_center
    ax, ay, az = basin_axes
    xs = graded_axis(0.0, 120e3, bx - ax, bx + ax, h_fine, h_max, growth)
    ys = graded_axis(0.0, 80e3, by - ay, by + ay, h_fine, h_max, growth)
    zs = graded_axis(-40e3, 0.0, -az, 0.0, h_fine, h_max, growth)
    mesh = kuhn_box_mesh(xs, ys, zs, periodic=(False, False, False), jitter=jitter, seed=seed,
                         sort_by_vid=sort_by_vid, top_bc=FACE_BC_FREE_SURFACE, side_bc=FACE_BC_ABSORBING)
    cen = mesh.centroids()
    depth = -cen[:, 2]
    mat = np.empty((mesh.n_elem, 6))
    for top, bot, vp, vs, rho in UNITS:
        sel = (depth >= top * 1e3) & (depth < bot * 1e3)
        lam, mu = lame_from_speeds(vp, vs, rho)
        mat[sel] = (rho, lam, mu, ROCK_GAMMA_R / 32e9 * mu, ROCK_XI0, ROCK_CD)
    inside = ((cen[:, 0] - bx) / ax) ** 2 + ((cen[:, 1] - by) / ay) ** 2 + (cen[:, 2] / az) ** 2 <= 1.0
    lam, mu = lame_from_speeds(*BASIN)
    mat[inside] = (BASIN[2], lam, mu, ROCK_GAMMA_R / 32e9 * mu, ROCK_XI0, ROCK_CD)

    def mu_of_depth(d):
        for top, bot, vp, vs, rho in UNITS:
            if top * 1e3 <= d < bot * 1e3:
                return rho * vs * vs
        return UNITS[-1][4] * UNITS[-1][3] ** 2
    sources = fault_sources(mu_of_depth)
    rng = np.random.default_rng(2)
    gx, gy = np.meshgrid(np.linspace(bx - 1.5 * ax, bx + 1.5 * ax, 8), np.linspace(by - 1.5 * ay, by + 1.5 * ay, 8),
                         indexing="ij")
    rec = np.stack([gx.ravel(), gy.ravel(), np.full(64, -50.0)], axis=1)
    rec[:, :2] += rng.uniform(-0.5 * h_fine, 0.5 * h_fine, size=(64, 2))
    return {"name": f"c3 regional-shaped box {mesh.n_elem} tets N={order}", "mesh": mesh, "material": mat,
            "order": order, "cfl": 0.5, "steps": 2000, "sources": sources, "receivers": rec,
            "basin": inside, "grid_cells": (len(xs) - 1, len(ys) - 1, len(zs) - 1),
            "h_range": (float(min(np.diff(xs).min(), np.diff(ys).min(), np.diff(zs).min())),
                        float(max(np.diff(xs).max(), np.diff(ys).max(), np.diff(zs).max())))}
