"""Second, independent FP64 formulation of LBGK / MRT steps with NumPy.

TEST INFRASTRUCTURE ONLY.  It exists to pin the C oracle's streaming and wall
handling with a different formulation: push streaming (post-collision F_i at x
moves to x + e_i, the left side of Eq. lbgk) done with np.roll on whole
fields, and half-way bounce-back (Sec. 2.3) as "a population that would enter
a solid node returns to its origin in the opposite direction within the same
step".  Its velocity set is enumerated in a different order from the C
oracle's (x-component slowest) so that an order-dependent mistake on either
side shows up.  Collision is written with whole-field array expressions.
Meant for grids up to ~16^3.
"""
from __future__ import annotations

import numpy as np


def velocities(D: int):
    """(e [Q,3], w [Q], opp [Q]); enumeration ex slowest, weights by |e|^2
    from Table bgkweights."""
    wt = {2: (4 / 9, 1 / 9, 1 / 36), 3: (1 / 3, 1 / 18, 1 / 36)}[D]
    es = []
    zr = (-1, 0, 1) if D == 3 else (0,)
    for ex in (1, 0, -1):
        for ey in (1, 0, -1):
            for ez in zr:
                if ex * ex + ey * ey + ez * ez <= 2:
                    es.append((ex, ey, ez))
    e = np.array(es, dtype=np.int64)
    w = np.array([wt[int((v * v).sum())] for v in e])
    opp = np.array([int(np.flatnonzero((e == -v).all(axis=1))[0]) for v in e])
    return e, w, opp


def feq_poly(e, w, rho, u):
    """Eq. equilibrium over whole fields; rho [...], u [3, ...] -> [Q, ...]."""
    eu = np.tensordot(e.astype(np.float64), u, axes=(1, 0))
    u2 = (u * u).sum(axis=0)
    return w[:, None, None, None] * rho[None] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * u2[None])


def guo_term(e, w, v, F):
    """w_i [3 (e_i - v) + 9 (e_i . v) e_i] . F per node (Eq. guo_force without
    its (1 - 1/(2 tau)) factor)."""
    Fv = np.asarray(F, dtype=np.float64).reshape(3, 1, 1, 1)
    ef = e.astype(np.float64)
    eF = ef @ np.asarray(F, dtype=np.float64)                # [Q]
    vF = (v * Fv).sum(axis=0)                                # [...]
    ev = np.tensordot(ef, v, axes=(1, 0))                    # [Q, ...]
    return w[:, None, None, None] * (3 * (eF[:, None, None, None] - vF[None]) +
                                     9 * ev * eF[:, None, None, None])


def mrt_basis(e):
    """Moment polynomials of d'Humieres et al. (2002) evaluated on e (rows)."""
    x, y, z = (e[:, 0].astype(float), e[:, 1].astype(float), e[:, 2].astype(float))
    e2 = x * x + y * y + z * z
    rows = [np.ones_like(x), 19 * e2 - 30, (21 * e2 ** 2 - 53 * e2 + 24) / 2,
            x, (5 * e2 - 9) * x, y, (5 * e2 - 9) * y, z, (5 * e2 - 9) * z,
            3 * x * x - e2, (3 * e2 - 5) * (3 * x * x - e2), y * y - z * z,
            (3 * e2 - 5) * (y * y - z * z), x * y, y * z, x * z,
            x * (y * y - z * z), y * (z * z - x * x), z * (x * x - y * y)]
    return np.array(rows)


def collide(D, F, tau, force=(0, 0, 0), mrt_s=None):
    """Collide every node of F [Q, nz, ny, nx] (post-streaming) -> post-collision.
    Returns (Fpost, rho, v)."""
    e, w, _ = velocities(D)
    ef = e.astype(np.float64)
    rho = F.sum(axis=0)
    j = np.tensordot(ef.T, F, axes=(1, 0))                   # [3, ...]
    Fv = np.asarray(list(force) + [0.0] * (3 - len(force)), dtype=np.float64)
    v = (j + 0.5 * Fv.reshape(3, 1, 1, 1)) / rho[None]
    fe = feq_poly(e, w, rho, v)
    Ft = guo_term(e, w, v, Fv)
    if mrt_s is None:
        out = F - (F - fe) / tau + (1 - 0.5 / tau) * Ft
    else:
        M = mrt_basis(e)
        S = np.asarray(mrt_s, dtype=np.float64)
        m = np.tensordot(M, F, axes=(1, 0))
        me = np.tensordot(M, fe, axes=(1, 0))
        mF = np.tensordot(M, Ft, axes=(1, 0))
        mp = m - S[:, None, None, None] * (m - me) + (1 - 0.5 * S)[:, None, None, None] * mF
        out = np.tensordot(np.linalg.inv(M), mp, axes=(1, 0))
    return out, rho, v


def stream_push(D, Fpost, mask=None):
    """Push streaming with periodic wrap and half-way bounce-back."""
    e, _, opp = velocities(D)
    out = np.zeros_like(Fpost)
    solid = None if mask is None else (np.asarray(mask) != 0)
    for i, v in enumerate(e):
        shift = (int(v[2]), int(v[1]), int(v[0]))
        moved = np.roll(Fpost[i], shift=shift, axis=(0, 1, 2))
        if solid is None:
            out[i] += moved
            continue
        # destination solid?  (destination of the population leaving x is x+e_i)
        dest_solid = np.roll(solid, shift=tuple(-s for s in shift), axis=(0, 1, 2))
        # populations arriving from fluid-or-solid sources into fluid nodes
        out[i] += np.where(solid, 0.0, np.roll(np.where(dest_solid, 0.0, Fpost[i]),
                                               shift=shift, axis=(0, 1, 2)))
        # populations that hit a solid destination come back reversed
        out[opp[i]] += np.where(dest_solid & ~solid, Fpost[i], 0.0)
    return out


def run(D, F0post, nsteps, tau, force=(0, 0, 0), mask=None, mrt_s=None):
    """F0post: post-collision state at t (Q in this module's order).
    Returns (F, rho, v) after nsteps, rho/v of the last step (solids 0)."""
    F = F0post.copy()
    rho = v = None
    solid = None if mask is None else (np.asarray(mask) != 0)
    for _ in range(nsteps):
        f = stream_push(D, F, mask)
        if solid is not None:
            # solid nodes receive nothing; give them a harmless state to collide
            e, w, _ = velocities(D)
            f = np.where(solid[None], w[:, None, None, None], f)
        F, rho, v = collide(D, f, tau, force, mrt_s)
        if solid is not None:
            F = np.where(solid[None], 0.0, F)
            rho = np.where(solid, 0.0, rho)
            v = np.where(solid[None], 0.0, v)
    return F, rho, v
