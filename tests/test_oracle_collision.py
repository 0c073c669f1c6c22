"""Pins of the oracle's equilibria and collision operators (CPU only).

Each check is fixed by the paper or by mathematics, not by the oracle itself:
moments of f_eq (Eq. lb_macro on Eq. equilibrium; the paper notes the same
check), exact conservation of each collision, MRT reducing to LBGK when all
rates are 1/tau, ELBM at alpha = 2 reducing to LBGK (Sec. 2.1.3), g(alpha)
against the H-function difference evaluated directly in 50-digit arithmetic,
H non-increase, and the small-deviation expansion of the alpha root.
"""
import math

import mpmath
import numpy as np
import pytest

from oracle import (BGK, MRT, ELBM, FIXED2, NEWTON, SERIES_GUARDED, ROOT_GUARDED, AL_CONV,
                    AL_GUARDED)


def _dim(code):
    return 2 if code in (2, 9) else 3


def _rand_f(oracle_lib, D, rng, u_amp=0.05, noise=0.02, kind=0):
    u = rng.uniform(-u_amp, u_amp, _dim(D))
    rho = 1.0 + rng.uniform(-0.05, 0.05)
    fe = oracle_lib.feq(D, rho, u, kind)
    f = fe * (1.0 + noise * rng.standard_normal(len(fe)))
    return f


@pytest.mark.parametrize("code", [2, 3, 15, 27])
def test_polynomial_feq_moments(oracle_lib, code):
    D = _dim(code)
    e, w, _ = oracle_lib.lattice(code)
    ef = e[:, :D].astype(float)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, D)
        fe = oracle_lib.feq(code, rho, u, 0)
        assert abs(fe.sum() - rho) < 1e-15
        assert np.abs(ef.T @ fe - rho * u).max() < 1e-15
        P = np.einsum("i,ia,ib->ab", fe, ef, ef)
        assert np.abs(P - rho * (np.eye(D) / 3 + np.outer(u, u))).max() < 1e-15


def test_entropic_feq_d3q27_is_exact_minimiser(oracle_lib):
    """D3Q27 is the tensor product of three D1Q3 sets (its weights factor as
    (2/3, 1/6, 1/6)^3), so the printed product form is the exact constrained
    H-minimiser there, as on D2Q9: mass and momentum hold without
    restoration and ln(f_eq / w) is affine in e.  On D3Q15 it is not."""
    e, w, _ = oracle_lib.lattice(27)
    ef = e.astype(float)
    w1 = {0: 2 / 3, 1: 1 / 6}
    for i in range(27):
        assert abs(w[i] - np.prod([w1[abs(int(c))] for c in e[i]])) < 1e-17
    A = np.column_stack([np.ones(27), ef])
    rng = np.random.default_rng(27)
    for _ in range(20):
        rho = rng.uniform(0.9, 1.1)
        u = rng.uniform(-0.1, 0.1, 3)
        fe = oracle_lib.feq(27, rho, u, 1)
        assert abs(fe.sum() - rho) < 1e-15
        assert np.abs(ef.T @ fe - rho * u).max() < 1e-15
        lhs = np.log(fe / w)
        coef, *_ = np.linalg.lstsq(A, lhs, rcond=None)
        assert np.abs(A @ coef - lhs).max() < 1e-14
        # restoring changes nothing beyond rounding
        assert np.abs(oracle_lib.feq(27, rho, u, 2) - fe).max() < 4e-16
    # on D3Q15 the raw product misses mass by far more than rounding
    raw15 = oracle_lib.feq(15, 1.0, np.array([0.08, -0.05, 0.03]), 1)
    assert abs(raw15.sum() - 1.0) > 1e-9


def test_entropic_feq_d2q9_is_constrained_minimiser(oracle_lib):
    """On D2Q9 the printed product form (read with 3u^2) conserves mass and
    momentum exactly and ln(f_eq/w) is affine in e (the Lagrange condition of
    minimising H = sum f ln(f/w) under those constraints)."""
    e, w, _ = oracle_lib.lattice(2)
    ef = e[:, :2].astype(float)
    rng = np.random.default_rng(2)
    A = np.column_stack([np.ones(9), ef])
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.15, 0.15, 2)
        fe = oracle_lib.feq(2, rho, u, 1)
        assert abs(fe.sum() - rho) < 1e-15
        assert np.abs(ef.T @ fe - rho * u).max() < 1e-15
        lhs = np.log(fe / w)
        coef, *_ = np.linalg.lstsq(A, lhs, rcond=None)
        assert np.abs(A @ coef - lhs).max() < 1e-14
        # and it agrees with the polynomial equilibrium to O(u^2)
        fp = oracle_lib.feq(2, rho, u, 0)
        assert np.abs(fe - fp).max() < 2.0 * np.abs(u).max() ** 3


def test_garbled_entropic_factor_breaks_mass(oracle_lib):
    """The printed first factor 2 - sqrt(1 + u^2) does not conserve mass; the
    3u^2 reading does.  Evaluated directly here from the printed formula."""
    e, w, _ = oracle_lib.lattice(2)
    u = np.array([0.1, -0.05])

    def product(c3):
        out = np.zeros(9)
        for i in range(9):
            p = w[i]
            for a in range(2):
                s = math.sqrt(1 + c3 * u[a] ** 2)
                p *= (2 - s) * ((2 * u[a] + math.sqrt(1 + 3 * u[a] ** 2)) / (1 - u[a])) ** e[i, a]
            out[i] = p
        return out

    assert abs(product(3.0).sum() - 1.0) < 1e-15
    assert abs(product(1.0).sum() - 1.0) > 1e-3
    assert np.abs(product(3.0) - oracle_lib.feq(2, 1.0, u, 1)).max() < 1e-15


def test_entropic_feq_d3q19_restored(oracle_lib):
    e, w, _ = oracle_lib.lattice(3)
    ef = e.astype(float)
    rng = np.random.default_rng(3)
    for _ in range(20):
        rho = rng.uniform(0.9, 1.1)
        u = rng.uniform(-0.08, 0.08, 3)
        raw = oracle_lib.feq(3, rho, u, 1)
        fe = oracle_lib.feq(3, rho, u, 2)
        # the raw product misses the constraints at O(u^3) only
        assert abs(raw.sum() - rho) < 5 * np.abs(u).max() ** 3 + 1e-15
        assert abs(fe.sum() - rho) < 1e-15
        assert np.abs(ef.T @ fe - rho * u).max() < 1e-15
        fp = oracle_lib.feq(3, rho, u, 0)
        assert np.abs(fe - fp).max() < 2.0 * np.abs(u).max() ** 3


@pytest.mark.parametrize("code,model", [(2, BGK), (3, BGK), (3, MRT), (2, ELBM), (3, ELBM),
                                        (15, BGK), (27, BGK), (15, ELBM), (27, ELBM)])
def test_collision_conserves_mass_and_momentum(oracle_lib, code, model):
    """Collision conserves mass; momentum grows by exactly the force F."""
    D = _dim(code)
    e, _, _ = oracle_lib.lattice(code)
    ef = e[:, :D].astype(float)
    rng = np.random.default_rng(4)
    for force in ((0.0, 0.0, 0.0), (1e-4, -3e-5, 2e-5)):
        p = oracle_lib.make_params(D=code, model=model, tau=0.57,
                                   force=force[:D] + (0.0,) * (3 - D), skip_eps=0.0)
        for _ in range(10):
            f = _rand_f(oracle_lib, code, rng)
            fo, rho, v, info = oracle_lib.collide(p, f)
            assert abs(fo.sum() - f.sum()) < 1e-15
            dj = ef.T @ fo - ef.T @ f
            assert np.abs(dj - np.array(force[:D])).max() < 2e-16
            # reported velocity is the force-shifted one (Eq. edm_momentum)
            assert np.allclose(v[:D], (ef.T @ f + 0.5 * np.array(force[:D])) / f.sum(),
                               atol=1e-16, rtol=0)


def test_mrt_with_equal_rates_is_lbgk(oracle_lib):
    rng = np.random.default_rng(5)
    tau = 0.55
    for force in ((0, 0, 0), (1e-5, 2e-6, -3e-6)):
        pb = oracle_lib.make_params(D=3, model=BGK, tau=tau, force=force)
        pm = oracle_lib.make_params(D=3, model=MRT, tau=tau, force=force, s=np.full(19, 1 / tau))
        for _ in range(10):
            f = _rand_f(oracle_lib, 3, rng)
            fb, *_ = oracle_lib.collide(pb, f)
            fm, *_ = oracle_lib.collide(pm, f)
            assert np.abs(fb - fm).max() < 1e-15


def test_mrt_relaxes_only_nonconserved_moments(oracle_lib):
    """With the default rates, the moments with s = 0 are unchanged (no force)
    and every other moment relaxes toward its equilibrium by (1 - s)."""
    rng = np.random.default_rng(6)
    M, _ = oracle_lib.mrt_matrix()
    tau = 0.55
    p = oracle_lib.make_params(D=3, model=MRT, tau=tau)
    s = np.array(list(p.s))
    f = _rand_f(oracle_lib, 3, rng)
    fo, rho, v, _ = oracle_lib.collide(p, f)
    fe = oracle_lib.feq(3, rho, v, 0)
    m, mo, me = M @ f, M @ fo, M @ fe
    assert np.abs(mo - (m - s * (m - me))).max() < 1e-13


def test_elbm_alpha2_is_lbgk(oracle_lib):
    """Sec. 2.1.3: with alpha = 2 the ELBM update is the LBGK update (with the
    entropic equilibrium)."""
    rng = np.random.default_rng(7)
    tau = 0.6
    for code in (2, 3, 15, 27):
        D = _dim(code)
        p = oracle_lib.make_params(D=code, model=ELBM, tau=tau, alpha_mode=FIXED2)
        for _ in range(5):
            f = _rand_f(oracle_lib, code, rng)
            rho = f.sum()
            e, _, _ = oracle_lib.lattice(code)
            u = (e[:, :D].T @ f) / rho
            fe = oracle_lib.feq(code, rho, u, 2)
            fo, *_ = oracle_lib.collide(p, f)
            assert np.abs(fo - (f + (fe - f) / tau)).max() < 1e-15


def _H_mp(f, w):
    return mpmath.fsum(mpmath.mpf(fi) * mpmath.log(mpmath.mpf(fi) / mpmath.mpf(wi))
                       for fi, wi in zip(f, w))


def test_g_matches_direct_entropy_difference(oracle_lib):
    """g(alpha) equals H(f + alpha Delta) - H(f) evaluated directly in 50
    digits (the FP64 direct difference would cancel catastrophically)."""
    mpmath.mp.dps = 50
    rng = np.random.default_rng(8)
    for D in (2, 3):
        _, w, _ = oracle_lib.lattice(D)
        for _ in range(5):
            f = _rand_f(oracle_lib, D, rng, noise=0.01)
            rho = f.sum()
            e, _, _ = oracle_lib.lattice(D)
            u = (e[:, :D].T @ f) / rho
            fe = oracle_lib.feq(D, rho, u, 2)
            d = fe - f
            for alpha in (0.5, 1.0, 1.7, 2.0, 2.3):
                g, gp = oracle_lib.elbm_g(D, f, fe, alpha)
                fa = [mpmath.mpf(fi) + mpmath.mpf(alpha) * mpmath.mpf(di) for fi, di in zip(f, d)]
                ref = _H_mp(fa, w) - _H_mp(f, w)
                # derivative, by the exact formula sum Delta (ln(fa/w) + 1)
                refp = mpmath.fsum(mpmath.mpf(di) * (mpmath.log(fai / mpmath.mpf(wi)) + 1)
                                   for di, fai, wi in zip(d, fa, w))
                scale = float(mpmath.fsum(mpmath.mpf(fi) * (mpmath.mpf(di) / mpmath.mpf(fi)) ** 2
                                          for fi, di in zip(f, d)))
                assert abs(g - float(ref)) < 1e-13 * scale + 1e-18
                assert abs(gp - float(refp)) < 1e-12 * scale + 1e-17


def test_alpha_root_and_entropy_non_increase(oracle_lib):
    rng = np.random.default_rng(9)
    for D in (2, 3):
        _, w, _ = oracle_lib.lattice(D)
        e, _, _ = oracle_lib.lattice(D)
        p = oracle_lib.make_params(D=D, model=ELBM, tau=0.5005, skip_eps=0.0)
        for _ in range(20):
            f = _rand_f(oracle_lib, D, rng, noise=0.05)
            rho = f.sum()
            u = (e[:, :D].T @ f) / rho
            fe = oracle_lib.feq(D, rho, u, 2)
            a, evals, status, resid = oracle_lib.elbm_alpha(p, f, fe)
            assert status == AL_CONV
            assert 1.0 < a
            assert resid < 1e-12
            # alpha is the non-trivial root: g < 0 just below it, > 0 just above
            gl, _ = oracle_lib.elbm_g(D, f, fe, a * (1 - 1e-6))
            gh, _ = oracle_lib.elbm_g(D, f, fe, a * (1 + 1e-6))
            assert gl < 0 < gh
            # H(f') <= H(f) for f' = f + alpha beta Delta, beta = 1/(2 tau) <= 1
            fo, *_ = oracle_lib.collide(p, f)
            assert float(_H_mp(fo, w) - _H_mp(f, w)) <= 1e-15


def test_alpha_series_small_deviation(oracle_lib):
    """For small departures from the exact minimiser (D2Q9) the root follows
    alpha = 2 + a3/(3 a2) + 4 a3^2/(9 a2^2) - 2 a4/(3 a2) + O(eps^3), obtained
    by expanding g(alpha)/alpha = 0 in powers of x = Delta/f: shrinking the
    same departure threefold must shrink the series error about 27-fold
    (the first-order term alone only about 9-fold)."""
    rng = np.random.default_rng(10)
    e, _, _ = oracle_lib.lattice(2)
    p = oracle_lib.make_params(D=2, model=ELBM, tau=0.6, skip_eps=0.0, tol=1e-15)
    for _ in range(10):
        u = rng.uniform(-0.05, 0.05, 2)
        fe0 = oracle_lib.feq(2, 1.0 + rng.uniform(-0.05, 0.05), u, 0)
        xi = rng.standard_normal(9)
        err2, err1 = [], []
        for amp in (3e-2, 1e-2):
            f = fe0 * (1.0 + amp * xi)
            rho = f.sum()
            fe = oracle_lib.feq(2, rho, (e[:, :2].T @ f) / rho, 2)
            a, *_ = oracle_lib.elbm_alpha(p, f, fe)
            _, ak = oracle_lib.elbm_features(2, f, fe)
            s1 = 2 + ak[3] / (3 * ak[2])
            s2 = s1 + 4 * ak[3] ** 2 / (9 * ak[2] ** 2) - 2 * ak[4] / (3 * ak[2])
            err2.append(abs(a - s2))
            err1.append(abs(a - s1))
            assert abs(a - 2) < 10 * math.sqrt(ak[2] / rho)
        assert err2[1] < err2[0] / 15.0
        assert err1[1] > err1[0] / 15.0
        assert err2[1] < err1[1]


def test_guarded_series_mode_agrees_with_newton(oracle_lib):
    rng = np.random.default_rng(11)
    for D in (2, 3):
        e, _, _ = oracle_lib.lattice(D)
        pn = oracle_lib.make_params(D=D, model=ELBM, tau=0.51, skip_eps=0.0)
        ps = oracle_lib.make_params(D=D, model=ELBM, tau=0.51, skip_eps=0.0,
                                    alpha_mode=SERIES_GUARDED)
        ev_n = ev_s = 0
        for _ in range(20):
            f = _rand_f(oracle_lib, D, rng, noise=0.01)
            rho = f.sum()
            u = (e[:, :D].T @ f) / rho
            fe = oracle_lib.feq(D, rho, u, 2)
            an = oracle_lib.elbm_alpha(pn, f, fe)
            as_ = oracle_lib.elbm_alpha(ps, f, fe)
            assert abs(an[0] - as_[0]) < 1e-9
            assert as_[2] in (AL_GUARDED, AL_CONV)
            ev_n += an[1]
            ev_s += as_[1]
        assert ev_s < ev_n


def test_near_equilibrium_skip(oracle_lib):
    f = oracle_lib.feq(3, 1.0, [0.01, 0.0, 0.0], 2) * (1 + 1e-5)
    f = f / f.sum()
    p = oracle_lib.make_params(D=3, model=ELBM, tau=0.6, skip_eps=1e-3)
    e, _, _ = oracle_lib.lattice(3)
    u = (e.T @ f) / f.sum()
    fe = oracle_lib.feq(3, f.sum(), u, 2)
    a = oracle_lib.elbm_alpha(p, f, fe)
    assert a[0] == 2.0 and a[1] == 0


def test_truncated_series_root_order_and_guarded_mode(oracle_lib):
    """The ROOT_GUARDED guess: the root of g(alpha)/alpha with g's series in
    alpha truncated after a_6 and the node's own A.  Truncation drops terms
    a_k alpha^(k-1) / (k (k-1)) with k >= 7, i.e. x^5 relative to a_2: shrinking
    a departure threefold must shrink the guess's error about 3^5 = 243-fold.
    It also covers the restored D3Q19 equilibrium, which is not the H
    minimiser and on which the second-order guess (derived for the minimiser)
    keeps an error that only shrinks like the restoration term.  The guarded
    mode from this guess returns Newton's root within 1e-10 after one
    evaluation."""
    rng = np.random.default_rng(12)
    e, _, _ = oracle_lib.lattice(3)
    pn = oracle_lib.make_params(D=3, model=ELBM, tau=0.6, skip_eps=0.0, tol=1e-15)
    pr = oracle_lib.make_params(D=3, model=ELBM, tau=0.6, skip_eps=0.0,
                                alpha_mode=ROOT_GUARDED, guard_steps=1)
    for _ in range(8):
        u = rng.uniform(-0.05, 0.05, 3)
        fe0 = oracle_lib.feq(3, 1.0, u, 2)
        xi = rng.standard_normal(19)
        errs = []
        for amp in (3e-2, 1e-2):
            f = fe0 * (1.0 + amp * xi)
            rho = f.sum()
            fe = oracle_lib.feq(3, rho, (e.T @ f) / rho, 2)
            a, *_ = oracle_lib.elbm_alpha(pn, f, fe)
            _, ak = oracle_lib.elbm_features(3, f, fe)
            w = oracle_lib.lattice(3)[1]
            d = fe - f
            A1 = float((d * np.log(f / w)).sum() + d.sum())
            errs.append(abs(a - oracle_lib.series_root_guess(ak, A1)))
            ar, evals, status, resid = oracle_lib.elbm_alpha(pr, f, fe)
            assert abs(ar - a) < 1e-10 and resid < 1e-12
            assert status == AL_GUARDED and evals == 1
        assert errs[1] < errs[0] / 100.0


def _h_minimiser(e, w, rho, u):
    """The exact entropic equilibrium: f_i = w_i exp(l_0 + l . e_i), the
    minimiser of H = sum f ln(f / w) with mass rho and momentum rho u, its four
    multipliers found by Newton's method on the constraints (NumPy)."""
    A = np.hstack([np.ones((len(w), 1)), e.astype(float)])
    target = np.concatenate([[rho], rho * np.asarray(u, dtype=float)])
    lam = np.zeros(4)
    lam[0] = math.log(rho)
    for _ in range(60):
        f = w * np.exp(A @ lam)
        step = np.linalg.solve(A.T @ (f[:, None] * A), A.T @ f - target)
        lam -= step
        if np.abs(step).max() < 1e-17:
            break
    return w * np.exp(A @ lam)


@pytest.mark.parametrize("code", [19, 15, 27])
def test_entropic_equilibrium_against_the_h_minimiser(oracle_lib, code):
    """Reading 3's equilibrium on the 3-D lattices against an independent
    computation, the H minimiser found numerically.  D3Q27: the product form
    is that minimiser (agreement to rounding).  D3Q19 / D3Q15: the product
    form is not; it agrees to O(u^5) (halving u divides the difference by
    ~32), and with mass and momentum restored to O(u^6) (~64) -- a wrong sign,
    index or factor in either part would break these orders."""
    e, w, _ = oracle_lib.lattice(code)
    rng = np.random.default_rng(code)
    for _ in range(4):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        rho = 1.0 + 0.01 * rng.standard_normal()
        err_r, err_p = [], []
        for s in (0.04, 0.02, 0.01):
            fm = _h_minimiser(e, w, rho, s * d)
            err_r.append(np.abs(oracle_lib.feq(code, rho, s * d, 2) - fm).max())
            err_p.append(np.abs(oracle_lib.feq(code, rho, s * d, 1) - fm).max())
        if code == 27:
            assert max(err_r + err_p) < 1e-15
            continue
        assert err_r[0] < 1e-8 * rho
        for k in range(2):
            assert 50 < err_r[k] / err_r[k + 1] < 80, err_r
            assert 25 < err_p[k] / err_p[k + 1] < 40, err_p
