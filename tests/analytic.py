"""Closed-form solutions the tests compare against (not the method itself).

- Plane Poiseuille start-up flow between walls at y_w and y_w + H driven by a
  body force g per unit volume (Eq. poiseuille_solution with nu0 = nu1 gives
  the steady parabola; the transient is the textbook Fourier-series solution
  of the diffusion equation with a source).
- Taylor-Green vortex (Eq. taylor_green, velocity lines; amplitude decays as
  exp(-2 nu k^2 t), kinetic energy as exp(-4 nu k^2 t)).
"""
from __future__ import annotations

import math
import numpy as np


def nu_of_tau(tau: float) -> float:
    """tau = (1 + 6 nu) / 2 (Sec. 2, after Eq. lbgk)."""
    return (2.0 * tau - 1.0) / 6.0


def poiseuille_steady(y, g, nu, y_w, H, rho=1.0):
    return g * (y - y_w) * (y_w + H - y) / (2.0 * rho * nu)


def poiseuille_startup(y, g, nu, y_w, H, t, rho=1.0, nterms=2001):
    """u(y, t) from rest: steady profile minus its decaying odd sine modes."""
    y = np.asarray(y, dtype=np.float64)
    u = poiseuille_steady(y, g, nu, y_w, H, rho)
    for n in range(1, nterms + 1, 2):
        coef = 4.0 * g * H * H / (rho * nu * math.pi ** 3 * n ** 3)
        u = u - coef * np.sin(n * math.pi * (y - y_w) / H) * math.exp(
            -n * n * math.pi * math.pi * nu * t / (H * H))
    return u


def taylor_green_u(n, u0, nu, t, D=3, nz=1):
    """Velocity field of the extruded 2D vortex at time t, [D, nz, n, n]."""
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")
    dec = math.exp(-2.0 * nu * k * k * t)
    u = np.zeros((D, nz, n, n))
    u[0] = -u0 * np.cos(k * X) * np.sin(k * Y) * dec
    u[1] = u0 * np.sin(k * X) * np.cos(k * Y) * dec
    return u


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def rho_errors(rg, ro, sel=None):
    """Density errors that a density near 1 cannot hide: the relative L2
    error of the deviation rho - 1, and the largest absolute error, over the
    selected nodes (all by default)."""
    rg = np.asarray(rg, dtype=np.float64)
    ro = np.asarray(ro, dtype=np.float64)
    if sel is not None:
        rg, ro = rg[sel], ro[sel]
    return rel_l2(rg - 1.0, ro - 1.0), float(np.abs(rg - ro).max())

