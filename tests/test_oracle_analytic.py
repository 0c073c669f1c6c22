"""The oracle against closed-form flows (CPU only).

- Plane Poiseuille start-up flow (Eq. poiseuille_solution with nu0 = nu1 and
  the textbook transient series), at the 64 x 32, tau = 0.8, g = 1e-6,
  5000-step channel; and the steady parabola to 1e-10 at
  tau = 1/2 + sqrt(3/16), where half-way bounce-back puts the wall exactly
  half a link beyond the last fluid node for LBGK.
- Taylor-Green vortex (Eq. taylor_green): second-order convergence of the
  velocity error under diffusive refinement, amplitude decay exp(-2 nu k^2 t),
  kinetic-energy decay exp(-4 nu k^2 t), and exact mass conservation.
"""
import math

import numpy as np
import pytest

import analytic as an
from oracle import BGK, MRT
from paper_1311_2404_gb300 import workloads as wl


def _channel_run(oracle_lib, nx, ny, tau, g, nsteps, model=BGK):
    p = oracle_lib.make_params(nx, ny, 1, D=2, model=model, tau=tau, force=(g, 0.0, 0.0))
    rho = np.ones((1, ny, nx))
    u = np.zeros((2, 1, ny, nx))
    mask = wl.channel_mask(nx, ny)
    F = oracle_lib.init(p, rho, u)
    F[:, mask.astype(bool)] = 0.0
    r, uu, _, _ = oracle_lib.run(p, F, nsteps, mask)
    return r, uu


def test_poiseuille_startup_64x32(oracle_lib):
    nx, ny, tau, g, T = 64, 32, 0.8, 1e-6, 5000
    r, uu = _channel_run(oracle_lib, nx, ny, tau, g, T)
    y = np.arange(1, ny - 1, dtype=np.float64)
    ux = uu[0, 0, 1:ny - 1, :]
    assert np.abs(ux - ux[:, :1]).max() < 1e-17          # uniform along x
    assert np.abs(uu[1]).max() < 1e-13                     # no cross flow (rounding)
    ref = an.poiseuille_startup(y, g, an.nu_of_tau(tau), 0.5, ny - 2, T)
    assert an.rel_l2(ux[:, 0], ref) < 1e-3
    # 5000 steps is not yet steady: the deficit is the slowest sine mode
    steady = an.poiseuille_steady(y, g, an.nu_of_tau(tau), 0.5, ny - 2)
    assert an.rel_l2(ux[:, 0], steady) > 2e-3


def test_poiseuille_parabola_exact_at_magic_tau(oracle_lib):
    ny, tau, g = 32, 0.5 + math.sqrt(3.0 / 16.0), 1e-6
    r, uu = _channel_run(oracle_lib, 4, ny, tau, g, 30000)
    y = np.arange(1, ny - 1, dtype=np.float64)
    ref = an.poiseuille_steady(y, g, an.nu_of_tau(tau), 0.5, ny - 2)
    assert an.rel_l2(uu[0, 0, 1:ny - 1, 0], ref) < 1e-10


def test_taylor_green_second_order(oracle_lib):
    tau, u0 = 0.8, 0.01
    nu = an.nu_of_tau(tau)
    errs = []
    for n in (16, 32, 64):
        k = 2 * math.pi / n
        t = int(round(0.25 / (nu * k * k)))
        rho, u = wl.taylor_green(n, u0, D=2)
        p = oracle_lib.make_params(n, n, 1, D=2, model=BGK, tau=tau)
        F = oracle_lib.init(p, rho, u)
        _, uu, _, _ = oracle_lib.run(p, F, t)
        errs.append(an.rel_l2(uu, an.taylor_green_u(n, u0, nu, t, D=2)))
    assert 3.6 < errs[0] / errs[1] < 4.4
    assert 3.6 < errs[1] / errs[2] < 4.4


@pytest.mark.parametrize("model", [BGK, MRT])
def test_taylor_green_d3q19_decay_and_mass(oracle_lib, model):
    """Extruded vortex on D3Q19 (one z plane stands for any number, the field
    being z-independent), 128^2, tau 0.6, u0 0.05, 250 steps (the same
    k^2 t as 256^2 at 1000 steps)."""
    n, tau, u0, T = 128, 0.6, 0.05, 250
    nu = an.nu_of_tau(tau)
    k = 2 * math.pi / n
    rho, u = wl.taylor_green(n, u0, nz=1, D=3)
    s = np.full(19, 1.0 / tau) if model == MRT else None
    p = oracle_lib.make_params(n, n, 1, D=3, model=model, tau=tau, s=s)
    F = oracle_lib.init(p, rho, u)
    m0 = F.sum()
    r, uu, _, _ = oracle_lib.run(p, F, T)
    assert an.rel_l2(uu, an.taylor_green_u(n, u0, nu, T, D=3)) < 2e-3
    E0 = 0.5 * (rho * (u * u).sum(0)).sum()
    E = 0.5 * (r * (uu * uu).sum(0)).sum()
    # O(k^2) lattice error: 6e-4 at 128^2, a quarter of that at 256^2
    assert abs(E / E0 / math.exp(-4 * nu * k * k * T) - 1) < 1e-3
    amp = np.abs(uu[0]).max() / u0
    assert abs(amp / math.exp(-2 * nu * k * k * T) - 1) < 2e-3
    assert abs(F.sum() - m0) < 1e-12 * m0
    assert abs(r.sum() - rho.sum()) < 1e-12 * rho.sum()


def test_taylor_green_256_at_1000_steps(oracle_lib):
    """The 256^3 extruded vortex (tau 0.6, u0 0.05, 1000 steps) computed on
    one z plane: velocity within 1e-3 of the analytic field, kinetic energy
    within 1e-4 of exp(-4 nu k^2 t)."""
    n, tau, u0, T = 256, 0.6, 0.05, 1000
    nu = an.nu_of_tau(tau)
    k = 2 * math.pi / n
    rho, u = wl.taylor_green(n, u0, nz=1, D=3)
    p = oracle_lib.make_params(n, n, 1, D=3, model=BGK, tau=tau)
    F = oracle_lib.init(p, rho, u)
    r, uu, _, _ = oracle_lib.run(p, F, T)
    assert an.rel_l2(uu, an.taylor_green_u(n, u0, nu, T, D=3)) < 1e-3
    E0 = 0.5 * (rho * (u * u).sum(0)).sum()
    E = 0.5 * (r * (uu * uu).sum(0)).sum()
    assert abs(E / E0 / math.exp(-4 * nu * k * k * T) - 1) < 1e-4
