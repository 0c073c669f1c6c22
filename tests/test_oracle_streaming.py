"""Pins of the oracle's streaming, walls and whole-run behaviour (CPU only).

- The C oracle (pull streaming, AB) equals an independent NumPy formulation
  (push streaming with np.roll, velocity set enumerated in another order) on
  small grids with walls and forcing, LBGK and MRT.
- Lattice-translation covariance (bitwise), a rest state stays at rest
  (to the rounding of sum w = 1), mirror symmetry, exact mass conservation.
"""
import numpy as np
import pytest

import oracle.np_oracle as npo
from oracle import BGK, MRT, ELBM
from paper_1311_2404_gb300 import workloads as wl


def _perm(oracle_lib, D):
    """Index map from the NumPy oracle's velocity order to the C oracle's."""
    ec, _, _ = oracle_lib.lattice(D)
    en, _, _ = npo.velocities(D)
    return np.array([int(np.flatnonzero((ec == v).all(axis=1))[0]) for v in en])


@pytest.mark.parametrize("D,model,shape,with_mask,force", [
    (2, BGK, (1, 10, 12), True, (2e-5, -1e-5, 0.0)),
    (2, BGK, (1, 9, 7), False, (0.0, 0.0, 0.0)),
    (3, BGK, (6, 7, 8), True, (1e-5, 2e-5, -1e-5)),
    (3, MRT, (5, 6, 7), True, (1e-5, 0.0, 3e-6)),
    (3, MRT, (4, 4, 5), False, (0.0, 0.0, 0.0)),
])
def test_pull_oracle_equals_push_numpy(oracle_lib, D, model, shape, with_mask, force):
    nz, ny, nx = shape
    rho, u = wl.random_state(nx, ny, nz, D, seed=7)
    mask = None
    if with_mask:
        rng = np.random.default_rng(3)
        mask = (rng.random(shape) < 0.15).astype(np.uint8)
        mask[:, 0, :] = 1
    tau = 0.7
    p = oracle_lib.make_params(nx, ny, nz, D=D, model=model, tau=tau, force=force)
    F = oracle_lib.init(p, rho, u)
    if mask is not None:
        F[:, mask.astype(bool)] = 0.0
    perm = _perm(oracle_lib, D)
    Fn = F[perm].copy()
    nsteps = 6
    rc, uc, _, _ = oracle_lib.run(p, F, nsteps, mask)
    s = np.array(list(p.s)) if model == MRT else None
    Fn, rn, vn = npo.run(D, Fn, nsteps, tau, force, mask, s)
    assert np.abs(rc - rn).max() < 1e-14
    assert np.abs(uc - vn[:D]).max() < 1e-15
    assert np.abs(F[perm] - Fn).max() < 1e-14


@pytest.mark.parametrize("D,model", [(2, BGK), (3, BGK), (3, MRT), (3, ELBM)])
def test_translation_covariance_bitwise(oracle_lib, D, model):
    nx, ny, nz = 9, 8, (1 if D == 2 else 6)
    rho, u = wl.random_state(nx, ny, nz, D, seed=11)
    p = oracle_lib.make_params(nx, ny, nz, D=D, model=model, tau=0.6, force=(1e-5, 0, 0))
    F = oracle_lib.init(p, rho, u)
    sh = (0 if D == 2 else 2, 3, 5)
    F2 = np.roll(F, sh, axis=(1, 2, 3)).copy()
    r1, u1, _, _ = oracle_lib.run(p, F, 5)
    r2, u2, _, _ = oracle_lib.run(p, F2, 5)
    assert np.array_equal(np.roll(r1, sh, axis=(0, 1, 2)), r2)
    assert np.array_equal(np.roll(u1, sh, axis=(1, 2, 3)), u2)


@pytest.mark.parametrize("D,model", [(2, BGK), (3, BGK), (3, MRT), (2, ELBM), (3, ELBM)])
def test_rest_state_stays_at_rest(oracle_lib, D, model):
    """Uniform rest with walls: f = w is a fixed point of every operator."""
    nx, ny, nz = 6, 5, (1 if D == 2 else 4)
    p = oracle_lib.make_params(nx, ny, nz, D=D, model=model, tau=0.6)
    rho = np.ones((nz, ny, nx))
    u = np.zeros((D, nz, ny, nx))
    F = oracle_lib.init(p, rho, u)
    F0 = F.copy()
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    mask[:, 0, :] = 1
    F[:, mask.astype(bool)] = 0.0
    r, uu, _, _ = oracle_lib.run(p, F, 4, mask)
    fl = ~mask.astype(bool)
    # exact up to the rounding of sum(w) = 1 in FP64
    assert np.abs(F[:, fl] - F0[:, fl]).max() < 1e-15
    assert np.abs(uu[:, fl]).max() < 1e-15 and np.abs(r[fl] - 1.0).max() < 1e-15


def test_mirror_symmetry(oracle_lib):
    """Reflecting x -> -x (and u_x -> -u_x) commutes with the update."""
    D, nx, ny, nz = 3, 8, 7, 5
    rho, u = wl.random_state(nx, ny, nz, D, seed=12)
    p = oracle_lib.make_params(nx, ny, nz, D=D, model=MRT, tau=0.6)
    F = oracle_lib.init(p, rho, u)
    rho_m = rho[:, :, ::-1].copy()
    u_m = u[:, :, :, ::-1].copy()
    u_m[0] *= -1
    Fm = oracle_lib.init(p, rho_m, u_m)
    r1, u1, _, _ = oracle_lib.run(p, F, 4)
    r2, u2, _, _ = oracle_lib.run(p, Fm, 4)
    # a reflection x -> -x maps node x to node (nx - x) mod nx for the pull
    # stencil; with the field reversed as [::-1] the image of x is nx-1-x,
    # i.e. a reflection about x = (nx - 1)/2, which the periodic lattice also has.
    assert np.abs(r1[:, :, ::-1] - r2).max() < 1e-15
    assert np.abs(u1[0][:, :, ::-1] + u2[0]).max() < 1e-15
    assert np.abs(u1[1][:, :, ::-1] - u2[1]).max() < 1e-15


@pytest.mark.parametrize("D,model", [(2, BGK), (3, MRT), (3, ELBM)])
def test_mass_conserved_over_run(oracle_lib, D, model):
    nx, ny, nz = 12, 10, (1 if D == 2 else 6)
    rho, u = wl.random_state(nx, ny, nz, D, seed=13)
    mask = wl.channel_mask(nx, ny, nz)
    p = oracle_lib.make_params(nx, ny, nz, D=D, model=model, tau=0.55, force=(1e-5, 0, 0))
    F = oracle_lib.init(p, rho, u)
    F[:, mask.astype(bool)] = 0.0
    m0 = F.sum()
    oracle_lib.run(p, F, 20, mask)
    assert abs(F.sum() - m0) < 1e-12 * m0
