"""Pins of the oracle's velocity / pressure boundary nodes (the equilibrium,
Zou-He and regularized conditions the paper lists in Sec. 2.3):

* the reconstructed node carries exactly the prescribed moments: mass and
  momentum j = rho v - F/2 (so the collision reports v), with rho from
  rho (1 - v_n) = S_0 + 2 S_out - F_n/2 recomputed here;
* Zou-He leaves the known populations alone and, on D2Q9, equals the
  closed form of Zou & He (1997) written out here;
* the regularized node has no non-hydrodynamic (ghost) component;
* a Couette flow between a half-way bounce-back wall and a velocity
  boundary row reaches the exact linear profile.
"""
import numpy as np
import pytest

import oracle
from oracle import BC_VELOCITY, BC_PRESSURE, BC_EQUILIBRIUM, BC_ZOUHE, BC_REGULARIZED

CODES = [2, 3, 15, 27]


def _dim(code):
    return 2 if code in (2, 9) else 3


def _near_eq(code, rng, amp=0.02):
    D = _dim(code)
    rho = 1.0 + 0.03 * rng.standard_normal()
    u = 0.04 * rng.standard_normal(D)
    fe = oracle.feq(code, rho, u)
    return fe * (1.0 + amp * rng.standard_normal(len(fe)))


@pytest.mark.parametrize("code", CODES)
@pytest.mark.parametrize("method", [BC_EQUILIBRIUM, BC_ZOUHE, BC_REGULARIZED])
@pytest.mark.parametrize("kind", [BC_VELOCITY, BC_PRESSURE])
def test_bc_node_moments(code, method, kind):
    D = _dim(code)
    e, w, opp = oracle.lattice(code)
    ef = e[:, :D].astype(float)
    rng = np.random.default_rng(100 + code + 10 * method + kind)
    for normal in [s * (a + 1) for a in range(D) for s in (1, -1)]:
        ax, sg = abs(normal) - 1, np.sign(normal)
        n = np.zeros(D)
        n[ax] = sg
        for force in ([0.0] * 3, [2e-5, -1e-5, 3e-5]):
            F = np.array(force[:D])
            vbc = 0.05 * rng.standard_normal(3)
            rbc = 1.0 + 0.02 * rng.standard_normal()
            p = oracle.make_params(D=code, model=oracle.BGK, tau=0.7, force=tuple(force))
            oracle.set_bc(p, 3, kind, method, int(normal), vbc if kind == BC_VELOCITY else [rbc])
            f = _near_eq(code, rng)
            g = oracle.bc_node(p, 3, f)
            en = ef @ n
            S0, So = f[en == 0].sum(), f[en < 0].sum()
            if kind == BC_VELOCITY:
                v = vbc[:D]
                rho = (S0 + 2 * So - 0.5 * F @ n) / (1 - v @ n)
            else:
                rho = rbc
                v = n * (1 - (S0 + 2 * So - 0.5 * F @ n) / rho)
            assert abs(g.sum() - rho) < 2e-15
            assert np.abs(ef.T @ g - (rho * v - 0.5 * F)).max() < 2e-15
            if method == BC_ZOUHE:
                known = en <= 0
                assert np.array_equal(g[known], f[known])


def test_zou_he_d2q9_closed_form():
    """Zou & He's reconstruction at a wall with inward normal +y, written in
    their D2Q9 notation (1 east, 2 north, 3 west, 4 south, 5 NE, 6 NW, 7 SW,
    8 SE): f2 = f4 + 2/3 rho v_y, f5 = f7 - (f1 - f3)/2 + rho v_y/6 + rho v_x/2,
    f6 = f8 + (f1 - f3)/2 + rho v_y/6 - rho v_x/2."""
    e, _, _ = oracle.lattice(2)
    idx = {tuple(v[:2]): i for i, v in enumerate(e)}
    k = {1: idx[(1, 0)], 2: idx[(0, 1)], 3: idx[(-1, 0)], 4: idx[(0, -1)], 5: idx[(1, 1)],
         6: idx[(-1, 1)], 7: idx[(-1, -1)], 8: idx[(1, -1)], 0: idx[(0, 0)]}
    rng = np.random.default_rng(5)
    p = oracle.make_params(D=2, model=oracle.BGK, tau=0.8)
    for _ in range(10):
        vx, vy = 0.05 * rng.standard_normal(2)
        oracle.set_bc(p, 0, BC_VELOCITY, BC_ZOUHE, 2, [vx, vy])
        f = _near_eq(2, rng)
        g = oracle.bc_node(p, 0, f)
        F = {j: f[k[j]] for j in range(9)}
        rho = (F[0] + F[1] + F[3] + 2 * (F[4] + F[7] + F[8])) / (1 - vy)
        assert abs(g[k[2]] - (F[4] + 2 / 3 * rho * vy)) < 1e-16
        assert abs(g[k[5]] - (F[7] - 0.5 * (F[1] - F[3]) + rho * vy / 6 + rho * vx / 2)) < 1e-16
        assert abs(g[k[6]] - (F[8] + 0.5 * (F[1] - F[3]) + rho * vy / 6 - rho * vx / 2)) < 1e-16


@pytest.mark.parametrize("code", CODES)
def test_regularized_node_has_no_ghost_part(code):
    D = _dim(code)
    e, w, _ = oracle.lattice(code)
    ef = e[:, :D].astype(float)
    rows = [np.ones(len(w))] + [ef[:, a] for a in range(D)]
    rows += [ef[:, a] * ef[:, b] for a in range(D) for b in range(a, D)]
    _, s, vt = np.linalg.svd(np.array(rows))
    ghost = vt[int((s > 1e-10).sum()):]
    rng = np.random.default_rng(9 + code)
    F = [1e-5, 2e-5, -1e-5]
    p = oracle.make_params(D=code, model=oracle.BGK, tau=0.7, force=tuple(F))
    for normal in (1, -2, 3 if D == 3 else 2):
        oracle.set_bc(p, 1, BC_VELOCITY, BC_REGULARIZED, normal, 0.04 * rng.standard_normal(3))
        g = oracle.bc_node(p, 1, _near_eq(code, rng, amp=0.05))
        rho = g.sum()
        v = (ef.T @ g + 0.5 * np.array(F[:D])) / rho
        # remove the equilibrium and the F/2 momentum term: what is left is
        # w_i times a polynomial of degree <= 2 in e_i (the Hermite space)
        rest = g - oracle.feq(code, rho, v) + 1.5 * w * (ef @ np.array(F[:D]))
        assert np.abs(ghost @ (rest / w)).max() < 1e-13


@pytest.mark.parametrize("code", CODES)
@pytest.mark.parametrize("method", [BC_ZOUHE, BC_REGULARIZED])
@pytest.mark.parametrize("tau", [0.8, 1.3])
def test_couette_between_wall_and_velocity_row(code, method, tau):
    """Solid row y = 0 (half-way bounce-back: wall at y = 1/2), velocity
    boundary row y = ny - 1 moving at U along x: the steady profile is
    exactly linear, u_x = U (y - 1/2) / (ny - 3/2), at any tau."""
    D = _dim(code)
    ny, U = 12, 0.05
    nx, nz = 3, (1 if D == 2 else 2)
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    mask[:, 0, :] = 1
    mask[:, ny - 1, :] = 2
    p = oracle.make_params(nx, ny, nz, D=code, model=oracle.BGK, tau=tau)
    oracle.set_bc(p, 0, BC_VELOCITY, method, -2, [U, 0.0, 0.0])
    rho0 = np.ones((nz, ny, nx))
    u0 = np.zeros((D, nz, ny, nx))
    Fd = oracle.init(p, rho0, u0)
    steps = int(40 * ny * ny / ((tau - 0.5) / 3 * np.pi ** 2)) + 200
    _, u, _, _ = oracle.run(p, Fd, steps, mask)
    y = np.arange(1, ny)
    ref = U * (y - 0.5) / (ny - 1.5)
    got = u[0, :, 1:, :]
    assert np.abs(got - ref[None, :, None]).max() < 1e-10 * U
    assert np.abs(u[1:, :, 1:, :]).max() < 1e-12
