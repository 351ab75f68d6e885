"""Exact solution of the 1-D Riemann problem of Sec. 3.1 (test infrastructure only).

The plane shear wave of Eq. "1d Riemann eqs": with eps = eps_xy and v = v_y,

    eps_t = v_x / 2,    rho v_t = sigma(eps)_x,

and the nonlinear shear relation of the same equation, taken here as the
plane-shear response of the oracle's isotropic law (reading R19):
sigma(eps) = 2 mu (1 - beta |eps|) eps.  The solver below is derived from these
two equations (the paper cites the solution without printing it) and restricts
itself to states with eps >= 0, where sigma = 2 mu (1 - beta eps) eps exactly.

Written as q_t + f(q)_x = 0 with q = (eps, v), f = (-v/2, -sigma/rho), the
Jacobian has the speeds -c and +c, c(eps) = sqrt(sigma'(eps) / (2 rho)), and the
right eigenvectors (1, 2c) and (1, -2c).  Hence:
  * 1-wave (speed -c): along a rarefaction dv/deps = +2c; a shock of speed
    s < 0 with s^2 = [sigma] / (2 rho [eps]) and [v] = -2 s [eps];
  * 2-wave (speed +c): along a rarefaction dv/deps = -2c; a shock with s > 0.
A k-wave is a shock when its characteristic speeds converge across it (Lax):
the 1-wave when c(eps_m) > c(eps_L), the 2-wave when c(eps_m) > c(eps_R).
The middle state solves v_1(eps_m) = v_2(eps_m) (bisection on a bracket of the
hyperbolic range sigma' > 0).
"""
from __future__ import annotations

import math

import numpy as np


class ShearRiemann:
    def __init__(self, left, right, rho=1.0, mu=1.0, beta=10.0):
        self.eL, self.vL = map(float, left)
        self.eR, self.vR = map(float, right)
        self.rho, self.mu, self.beta = float(rho), float(mu), float(beta)
        if min(self.eL, self.eR) < 0:
            raise ValueError("states with eps >= 0 only")
        for e in (self.eL, self.eR):
            if not self.dsigma(e) > 0:
                raise ValueError(f"state eps = {e} is not hyperbolic (sigma' <= 0)")
        self.em = self._middle()
        self.vm = self.v1(self.em)
        self.kind1 = "shock" if self.c(self.em) > self.c(self.eL) else "rarefaction"
        self.kind2 = "shock" if self.c(self.em) > self.c(self.eR) else "rarefaction"

    # ---------------- the relation and its speed ----------------
    def sigma(self, e):
        return 2.0 * self.mu * (1.0 - self.beta * abs(e)) * e

    def dsigma(self, e):
        return 2.0 * self.mu * (1.0 - 2.0 * self.beta * abs(e))

    def c(self, e):
        return math.sqrt(max(self.dsigma(e), 0.0) / (2.0 * self.rho))

    def e_of_c(self, c):
        """The eps >= 0 with c(eps) = c (c decreasing in eps for beta > 0)."""
        return (1.0 - self.rho * c * c / self.mu) / (2.0 * self.beta)

    def G(self, a, b):
        """int_a^b 2 c(s) ds for a, b >= 0, in closed form:
        2 sqrt(mu/rho) [-(1 - 2 beta s)^(3/2) / (3 beta)]_a^b (2 c (b - a) at beta = 0)."""
        k = 2.0 * math.sqrt(self.mu / self.rho)
        if self.beta == 0.0:
            return k * (b - a)
        F = lambda s: -((1.0 - 2.0 * self.beta * s) ** 1.5) / (3.0 * self.beta)
        return k * (F(b) - F(a))

    def shock_speed(self, ea, eb, family):
        jump = (self.sigma(eb) - self.sigma(ea)) / (2.0 * self.rho * (eb - ea))
        s = math.sqrt(jump)
        return -s if family == 1 else s

    # ---------------- wave curves ----------------
    def v1(self, em):
        """v of the states reachable from the left state by a 1-wave."""
        if em == self.eL:
            return self.vL
        if self.c(em) <= self.c(self.eL):
            return self.vL + self.G(self.eL, em)
        s = self.shock_speed(self.eL, em, 1)
        return self.vL - 2.0 * s * (em - self.eL)

    def v2(self, em):
        """v of the states from which the right state is reached by a 2-wave."""
        if em == self.eR:
            return self.vR
        if self.c(em) <= self.c(self.eR):
            return self.vR - self.G(self.eR, em)
        s = self.shock_speed(em, self.eR, 2)
        return self.vR + 2.0 * s * (self.eR - em)

    def _middle(self):
        lo = 0.0
        # sigma' > 0 for eps < 1 / (2 beta)
        hi = (1.0 - 1e-9) / (2.0 * self.beta) if self.beta > 0 else 10.0 * (self.eL + self.eR + 1.0)
        f = lambda e: self.v1(e) - self.v2(e)
        flo, fhi = f(lo), f(hi)
        if flo * fhi > 0:
            raise ValueError("no middle state with eps >= 0 in the hyperbolic range")
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            fm = f(mid)
            if (fm < 0) == (flo < 0):
                lo, flo = mid, fm
            else:
                hi = mid
        return 0.5 * (lo + hi)

    # ---------------- wave fan ----------------
    def speeds(self):
        """(first, last) speed of each wave: equal for a shock."""
        if self.kind1 == "shock":
            w1 = (self.shock_speed(self.eL, self.em, 1),) * 2
        else:
            w1 = (-self.c(self.eL), -self.c(self.em))
        if self.kind2 == "shock":
            w2 = (self.shock_speed(self.em, self.eR, 2),) * 2
        else:
            w2 = (self.c(self.em), self.c(self.eR))
        return w1, w2

    def sample(self, x, t):
        """(eps, v) at the points x (array) and time t > 0, the jump at x = 0."""
        x = np.asarray(x, dtype=np.float64)
        xi = x / t
        eps = np.empty_like(xi)
        v = np.empty_like(xi)
        (a1, b1), (a2, b2) = self.speeds()
        for k, z in np.ndenumerate(xi):
            if z < a1:
                e, w = self.eL, self.vL
            elif z < b1:                                   # inside the 1-rarefaction: -c(e) = z
                e = self.e_of_c(-z)
                w = self.vL + self.G(self.eL, e)
            elif z < a2:
                e, w = self.em, self.vm
            elif z < b2:                                   # inside the 2-rarefaction: c(e) = z
                e = self.e_of_c(z)
                w = self.vR - self.G(self.eR, e)
            else:
                e, w = self.eR, self.vR
            eps[k], v[k] = e, w
        return eps, v


class ShearSimpleWave:
    """Exact right-going simple wave of the same plane shear system (derived here,
    not printed in the paper), for convergence on smooth nonlinear solutions.

    The states lie on the integral curve of the 2-family through (eps_bar, v_bar),
    v = v_bar - G(eps_bar, eps), and eps is constant along the straight
    characteristics dx/dt = c(eps): eps(x, t) = eps0(xi) with x = xi + c(eps0(xi)) t.
    Initial strain eps0(x) = eps_bar + amp sin(2 pi x / length), periodic in x;
    exact until the characteristics cross (t < t_break)."""

    def __init__(self, eps_bar=0.01, amp=0.002, v_bar=0.0, length=1.0, rho=1.0, mu=1.0, beta=10.0):
        self.r = ShearRiemann((eps_bar, 0.0), (eps_bar, 0.0), rho=rho, mu=mu, beta=beta)
        self.eps_bar, self.amp, self.v_bar, self.length = float(eps_bar), float(amp), float(v_bar), float(length)
        if eps_bar - amp < 0 or not self.r.dsigma(eps_bar + amp) > 0:
            raise ValueError("the wave must stay in 0 <= eps < 1 / (2 beta)")
        k = 2 * math.pi / self.length
        xi = np.linspace(0.0, self.length, 4001)
        e = self.eps0(xi)
        dc = np.array([self.dc(x) for x in e]) * self.amp * k * np.cos(k * xi)
        self.t_break = float("inf") if np.min(dc) >= 0 else float(-1.0 / np.min(dc))

    def eps0(self, x):
        return self.eps_bar + self.amp * np.sin(2 * math.pi * np.asarray(x) / self.length)

    def dc(self, e):
        """d c / d eps = sigma''(eps) / (4 rho c) with sigma'' = -4 mu beta (eps > 0)."""
        return -4.0 * self.r.mu * self.r.beta / (4.0 * self.r.rho * self.r.c(e)) if self.r.beta else 0.0

    def v_of(self, e):
        return self.v_bar - self.r.G(self.eps_bar, e)

    def sample(self, x, t):
        """(eps, v) at the points x and time 0 <= t < t_break: the foot xi of the
        characteristic through (x, t) by Newton on xi + c(eps0(xi)) t = x (mod length)."""
        if not t < self.t_break:
            raise ValueError("the characteristics have crossed: no smooth solution")
        x = np.asarray(x, dtype=np.float64)
        k = 2 * math.pi / self.length
        c0 = self.r.c(self.eps_bar)
        xi = x - c0 * t
        for _ in range(60):
            e = self.eps0(xi)
            c = np.sqrt(np.maximum(2.0 * self.r.mu * (1.0 - 2.0 * self.r.beta * np.abs(e)), 0.0) / (2.0 * self.r.rho))
            dcde = np.where(c > 0, -self.r.mu * self.r.beta / (self.r.rho * np.maximum(c, 1e-300)), 0.0)
            f = xi + c * t - x
            df = 1.0 + dcde * self.amp * k * np.cos(k * xi) * t
            step = f / df
            xi = xi - step
            if np.max(np.abs(step)) < 1e-15 * self.length:
                break
        eps = self.eps0(xi)
        v = np.array([self.v_of(ev) for ev in np.ravel(eps)]).reshape(eps.shape)
        return eps, v
