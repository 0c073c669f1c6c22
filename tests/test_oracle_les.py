"""Pins of the oracle's regularized LBGK (Sec. 2.1.1), Smagorinsky LBGK
(Sec. 2.1.4, Eqs. smagorinsky and taut) and kinetic-energy / enstrophy
diagnostics (Sec. 5.2) against facts that do not come from the oracle:

* regularization leaves a non-equilibrium part that already lies in the
  second-order Hermite space unchanged (REG = LBGK there), removes every
  component with zero mass, momentum and momentum flux, conserves mass and
  momentum and relaxes the momentum flux by (1 - 1/tau);
* the Smagorinsky relaxation time solves the quadratic of Eq. taut for the
  flux tensor computed here from f - f_eq, reduces to LBGK at C_S = 0 and,
  for a Chapman-Enskog non-equilibrium part of strain rate S, gives the eddy
  viscosity nu_t = tau_t / 3 = 2 C_S^2 rho |S| (|S| = (S:S)^(1/2));
* E(0) = 3 u0^2 / 8 for the Kida field and its central-difference enstrophy
  has the closed form 3 u0^2 / 8 (2 sin^2 t + sin^2 3t), t = 2 pi / N (the
  modified wavenumbers sin(k t) of the stencil); for a random periodic field
  the stencil enstrophy equals the spectral sum with modified wavenumbers.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1311_2404_gb300 import workloads as wl


def _lat(D):
    e, w, _ = oracle.lattice(D)
    return e[:, :D].astype(np.float64), w


def _moments(f, e):
    rho = f.sum()
    j = e.T @ f
    P = (e.T * f) @ e
    return rho, j, P


def _near_eq(D, rng, amp=0.02):
    e, w = _lat(D)
    rho = 1.0 + 0.05 * rng.standard_normal()
    u = 0.05 * rng.standard_normal(D)
    f = oracle.feq(D, rho, u) * (1.0 + amp * rng.standard_normal(len(w)))
    return f


def _ghost_basis(D):
    """Orthonormal basis of the vectors g with sum g = 0, sum g e = 0 and
    sum g e e = 0 (the non-hydrodynamic subspace)."""
    e, _ = _lat(D)
    rows = [np.ones(len(e))] + [e[:, a] for a in range(D)]
    rows += [e[:, a] * e[:, b] for a in range(D) for b in range(a, D)]
    C = np.array(rows)
    _, s, vt = np.linalg.svd(C)
    rank = int((s > 1e-10).sum())
    return vt[rank:]


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("force", [False, True])
def test_reg_equals_lbgk_in_hermite_space(D, force):
    """f = f_eq(rho, v) + w_i 9/2 (e_i e_i - I/3) : Pi: the regularized
    non-equilibrium part is f_neq itself, so REG and LBGK agree."""
    rng = np.random.default_rng(11 + D)
    e, w = _lat(D)
    F = tuple(1e-4 * rng.standard_normal(D)) + (0.0,) * (3 - D) if force else (0, 0, 0)
    for _ in range(5):
        rho = 1.0 + 0.05 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(D)
        A = 1e-3 * rng.standard_normal((D, D))
        Pi = A + A.T
        H = np.einsum("ia,ib->iab", e, e) - np.eye(D)[None] / 3.0
        fneq = w * 4.5 * np.einsum("iab,ab->i", H, Pi)
        # v of the collision includes F/2 rho; put the equilibrium at that v
        j = rho * u - 0.5 * np.array(F[:D])
        v = (j + 0.5 * np.array(F[:D])) / rho
        f = oracle.feq(D, rho, v) + fneq
        # the equilibrium at (rho, v) carries momentum rho v; shift to j
        f += w * 3.0 * (e @ (j - rho * v))
        pr = oracle.make_params(D=D, model=oracle.REG, tau=0.7, force=F)
        pb = oracle.make_params(D=D, model=oracle.BGK, tau=0.7, force=F)
        fr, _, _, _ = oracle.collide(pr, f)
        fb, _, _, _ = oracle.collide(pb, f)
        assert np.allclose(fr, fb, rtol=0, atol=1e-15)


@pytest.mark.parametrize("D", [2, 3])
def test_reg_removes_ghost_components(D):
    """Adding any g with zero mass, momentum and momentum flux changes
    nothing after regularization, but does change LBGK's result."""
    rng = np.random.default_rng(7 * D)
    G = _ghost_basis(D)
    assert G.shape[0] == (19 - 10 if D == 3 else 9 - 6)
    pr = oracle.make_params(D=D, model=oracle.REG, tau=0.8, force=(1e-5, -2e-5, 0.0))
    pb = oracle.make_params(D=D, model=oracle.BGK, tau=0.8, force=(1e-5, -2e-5, 0.0))
    for _ in range(5):
        f = _near_eq(D, rng)
        g = 1e-3 * (rng.standard_normal(G.shape[0]) @ G)
        a, _, _, _ = oracle.collide(pr, f)
        b, _, _, _ = oracle.collide(pr, f + g)
        assert np.allclose(a, b, rtol=0, atol=2e-16)
        c, _, _, _ = oracle.collide(pb, f)
        d, _, _, _ = oracle.collide(pb, f + g)
        assert np.abs(c - d).max() > 1e-5


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("model", [oracle.REG, oracle.SMAG])
def test_les_conservation_and_flux_relaxation(D, model):
    """Mass is kept, momentum gains F; without force the momentum flux
    about the equilibrium relaxes by (1 - 1/tau) (tau the total relaxation
    time returned for SMAG)."""
    rng = np.random.default_rng(3 + D + 10 * model)
    e, _ = _lat(D)
    for force in [(0.0, 0.0, 0.0), (2e-5, -1e-5, 3e-5 if D == 3 else 0.0)]:
        p = oracle.make_params(D=D, model=model, tau=0.65, force=force, smag_cs=0.17)
        for _ in range(4):
            f = _near_eq(D, rng)
            rho, j, P = _moments(f, e)
            fp, r2, v2, info = oracle.collide(p, f)
            rho2, j2, P2 = _moments(fp, e)
            assert abs(rho2 - rho) < 1e-15
            assert np.allclose(j2, j + np.array(force[:D]), rtol=0, atol=1e-16)
            if not any(force):
                tau = info[0] if model == oracle.SMAG else 0.65
                v = j / rho
                Peq = rho * (np.outer(v, v) + np.eye(D) / 3.0)
                assert np.allclose(P2 - Peq, (1 - 1 / tau) * (P - Peq), rtol=0, atol=1e-15)


@pytest.mark.parametrize("D", [2, 3])
def test_smagorinsky_cs0_is_lbgk(D):
    rng = np.random.default_rng(5 + D)
    F = (1e-5, 2e-5, -1e-5 if D == 3 else 0.0)
    ps = oracle.make_params(D=D, model=oracle.SMAG, tau=0.6, force=F, smag_cs=0.0)
    pb = oracle.make_params(D=D, model=oracle.BGK, tau=0.6, force=F)
    for _ in range(5):
        f = _near_eq(D, rng)
        a, _, _, info = oracle.collide(ps, f)
        b, _, _, _ = oracle.collide(pb, f)
        assert info[0] == 0.6
        assert np.allclose(a, b, rtol=0, atol=1e-16)


@pytest.mark.parametrize("D", [2, 3])
def test_smagorinsky_tau_solves_eq_taut(D):
    """tau_t (tau0 + tau_t) = C_S^2 |Q| / c_s^4 with Q = sum e e (f - f_eq)
    computed here, f_eq the second-order polynomial equilibrium at v."""
    rng = np.random.default_rng(17 + D)
    e, w = _lat(D)
    tau0, cs = 0.52, 0.1
    F = (3e-5, 0.0, 0.0)
    p = oracle.make_params(D=D, model=oracle.SMAG, tau=tau0, force=F, smag_cs=cs)
    for _ in range(6):
        f = _near_eq(D, rng, amp=0.05)
        rho, j, _ = _moments(f, e)
        v = (j + 0.5 * np.array(F[:D])) / rho
        usq = v @ v
        eu = e @ v
        feq = w * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * usq)
        Q = (e.T * (f - feq)) @ e
        qn = math.sqrt((Q * Q).sum())
        _, _, _, info = oracle.collide(p, f)
        tt = info[0] - tau0
        assert tt > 0
        assert abs(tt * (tau0 + tt) - 9.0 * cs * cs * qn) <= 1e-13 * tau0 * tt


@pytest.mark.parametrize("D", [2, 3])
def test_smagorinsky_eddy_viscosity_of_a_shear(D):
    """Chapman-Enskog non-equilibrium part of a traceless strain rate S at
    total relaxation time tau: f_neq_i = -3 rho tau w_i (e_i e_i - I/3) : S.
    Then |Q| = 2 rho c_s^2 tau |S|; choosing tau_t first and
    |S| = tau_t / (6 C_S^2 rho), the oracle must return tau0 + tau_t, i.e.
    nu_t = tau_t / 3 = 2 C_S^2 rho |S|."""
    rng = np.random.default_rng(23 + D)
    e, w = _lat(D)
    tau0, cs = 0.55, 0.12
    p = oracle.make_params(D=D, model=oracle.SMAG, tau=tau0, smag_cs=cs)
    for tt in (1e-3, 0.02, 0.3):
        A = rng.standard_normal((D, D))
        S = A + A.T
        S -= np.trace(S) / D * np.eye(D)
        rho = 1.0 + 0.02 * rng.standard_normal()
        S *= (tt / (6 * cs * cs * rho)) / math.sqrt((S * S).sum())
        u = 0.03 * rng.standard_normal(D)
        tau = tau0 + tt
        H = np.einsum("ia,ib->iab", e, e) - np.eye(D)[None] / 3.0
        fneq = -3.0 * rho * tau * w * np.einsum("iab,ab->i", H, S)
        f = oracle.feq(D, rho, u) + fneq
        _, _, _, info = oracle.collide(p, f)
        assert abs(info[0] - tau) < 1e-12 * tau


def test_kida_initial_energy_and_enstrophy_closed_form():
    for n in (16, 24, 40):
        u0 = 0.05
        _, u = wl.kida(n, u0)
        E, Om = oracle.kinetic_energy_enstrophy(u)
        t = 2 * math.pi / n
        assert abs(E - 3 * u0 ** 2 / 8) < 1e-15
        ref = 3 * u0 ** 2 / 8 * (2 * math.sin(t) ** 2 + math.sin(3 * t) ** 2)
        assert abs(Om - ref) < 1e-13 * ref
        # the field is solenoidal under the same stencil
        d = lambda f, ax: 0.5 * (np.roll(f, -1, ax) - np.roll(f, 1, ax))   # noqa: E731
        div = d(u[0], 2) + d(u[1], 1) + d(u[2], 0)
        assert np.abs(div).max() < 1e-15


@pytest.mark.parametrize("D", [2, 3])
def test_enstrophy_equals_modified_wavenumber_spectrum(D):
    """Central differences act on Fourier mode k as i sin(2 pi k / n):
    the stencil enstrophy equals the Parseval sum of |i s x u_hat|^2."""
    rng = np.random.default_rng(99 + D)
    shape = (1, 12, 20) if D == 2 else (10, 12, 14)
    u = rng.standard_normal((D,) + shape)
    E, Om = oracle.kinetic_energy_enstrophy(u)
    nz, ny, nx = shape
    sz = np.sin(2 * np.pi * np.fft.fftfreq(nz) * 1.0)[:, None, None] * np.ones(shape)
    sy = np.sin(2 * np.pi * np.fft.fftfreq(ny))[None, :, None] * np.ones(shape)
    sx = np.sin(2 * np.pi * np.fft.fftfreq(nx))[None, None, :] * np.ones(shape)
    uh = np.fft.fftn(u, axes=(1, 2, 3))
    V = nx * ny * nz
    if D == 3:
        wx = sy * uh[2] - sz * uh[1]
        wy = sz * uh[0] - sx * uh[2]
        wz = sx * uh[1] - sy * uh[0]
        w2 = np.abs(wx) ** 2 + np.abs(wy) ** 2 + np.abs(wz) ** 2
    else:
        w2 = np.abs(sx * uh[1] - sy * uh[0]) ** 2
    Om_spec = 0.5 * w2.sum() / V ** 2
    E_spec = 0.5 * (np.abs(uh) ** 2).sum() / V ** 2
    assert abs(E - E_spec) < 1e-12 * E
    assert abs(Om - Om_spec) < 1e-12 * Om
