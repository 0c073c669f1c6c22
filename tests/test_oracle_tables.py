"""Pins of the oracle's lattice tables and MRT basis (CPU only).

Checked against what the paper prints (Table bgkweights, Listing bb's D2Q9
swap pairs) and against exact lattice identities (isotropy up to 4th order,
orthogonality of the d'Humieres basis)."""
import os
from fractions import Fraction

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _weights_table():
    rows = {}
    with open(os.path.join(GOLD, "bgk_weights.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            rows[name] = [None if v == "-" else Fraction(v) for v in vals]
    return rows


LATTICES = [(2, "D2Q9", 9), (3, "D3Q19", 19), (15, "D3Q15", 15), (27, "D3Q27", 27)]


@pytest.mark.parametrize("code,name,Q", LATTICES)
def test_weights_match_paper_table(oracle_lib, code, name, Q):
    e, w, _ = oracle_lib.lattice(code)
    table = _weights_table()[name]
    assert len(w) == Q
    counts = [0, 0, 0, 0]
    for ei, wi in zip(e, w):
        n2 = int((ei * ei).sum())
        counts[n2] += 1
        assert table[n2] is not None
        assert wi == pytest.approx(float(table[n2]), abs=1e-16)
    # every link length the table lists is present, with all its links
    D = 2 if Q == 9 else 3
    full = {2: [1, 4, 4, 0], 3: [1, 6, 12, 8]}[D]
    for k in range(4):
        assert counts[k] == (full[k] if table[k] is not None else 0)
    # the table's rows sum to one over their links (exact rational check)
    assert sum(c * table[k] for k, c in enumerate(counts) if c) == 1


@pytest.mark.parametrize("code", [2, 3, 15, 27])
def test_isotropy(oracle_lib, code):
    e, w, _ = oracle_lib.lattice(code)
    D = 2 if code == 2 else 3
    e = e[:, :D].astype(np.float64)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ e).max() < 1e-16
    m2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(m2, np.eye(D) / 3, atol=1e-16)
    m3 = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    assert np.abs(m3).max() < 1e-16
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(D)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) +
           np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-16)


def test_opposites_match_listing_pairs(oracle_lib):
    e, _, opp = oracle_lib.lattice(2)
    pairs = np.loadtxt(os.path.join(GOLD, "bounce_back_pairs_d2q9.txt"), dtype=int)
    for ex, ey, ox, oy in pairs:
        i = int(np.flatnonzero((e[:, 0] == ex) & (e[:, 1] == ey))[0])
        j = int(np.flatnonzero((e[:, 0] == ox) & (e[:, 1] == oy))[0])
        assert opp[i] == j and opp[j] == i


@pytest.mark.parametrize("D", [2, 3, 15, 27])
def test_opposite_is_involution(oracle_lib, D):
    e, _, opp = oracle_lib.lattice(D)
    assert (opp[opp] == np.arange(len(opp))).all()
    assert (e[opp] == -e).all()


def test_mrt_basis_orthogonal_integer(oracle_lib):
    M, Mi = oracle_lib.mrt_matrix()
    assert np.array_equal(M, np.round(M))
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0.0
    # norms of the d'Humieres rows: rho 19, e 2394, eps 252, j 10, q 40, ...
    expect = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    assert np.array_equal(np.diag(G), np.array(expect, dtype=float))
    assert np.allclose(Mi @ M, np.eye(19), atol=1e-13)
    # row 0 is mass, rows 3/5/7 are the momentum components
    e, _, _ = oracle_lib.lattice(3)
    assert np.array_equal(M[0], np.ones(19))
    assert np.array_equal(M[3], e[:, 0]) and np.array_equal(M[5], e[:, 1])
    assert np.array_equal(M[7], e[:, 2])
