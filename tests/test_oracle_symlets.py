"""Pins for the oracle's least-asymmetric Daubechies filters (symlets,
Table 1's sym rows): Table 1 prints equal DB2 / sym2 and DB3 / sym3 rows;
the chosen filter is the least asymmetric of every real filter that the
same construction admits, checked by a brute force with numpy's own root
finder; the sym2 row of Table 1 is reproduced like the DB2 row."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import dense, tables, wavelets as W

Sym = tables.Sym
GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def _table1():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, dim, *vals = line.split()
        out[(name, int(dim))] = [float(v) for v in vals]
    return out


def _h(p):
    return np.array([float(v) for v in tables.daubechies_mp(p)])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_short_symlets_are_the_extremal_phase_filters(p):
    """For p <= 3 the only real choices are a filter and its mirror image, so
    the least-asymmetric filter oriented like the extremal-phase one is that
    filter (Table 1: the DB2 / sym2 and DB3 / sym3 rows are equal)."""
    assert np.array_equal(_h(Sym(p)), _h(p))


def _all_real_candidates(p):
    """Every real choice of one zero per reciprocal pair of Daubechies'
    construction (complex pairs of roots of P chosen together), from numpy's
    own root finder in float64: (zeros, h) per choice."""
    ys = np.roots([float(math.comb(p - 1 + k, k)) for k in range(p)][::-1]) if p > 1 else []
    pairs = []
    for y in ys:
        b = 2 - 4 * y
        d = np.sqrt(b * b - 4 + 0j)
        pairs.append(((b + d) / 2, (b - d) / 2))
    groups, left = [], list(range(len(pairs)))
    while left:
        i = left.pop(0)
        if abs(ys[i].imag) < 1e-9:
            groups.append([i])
        else:
            j = min(left, key=lambda k: abs(ys[k] - np.conj(ys[i])))
            left.remove(j)
            groups.append([i, j])
    out = []
    for choice in itertools.product((0, 1), repeat=len(groups)):
        zeros = [pairs[i][c] for g, c in zip(groups, choice) for i in g]
        poly = np.array([1.0 + 0j])
        for _ in range(p):
            poly = np.convolve(poly, [1.0, 1.0])
        for z in zeros:
            poly = np.convolve(poly, [-z, 1.0])
        h = poly.real
        out.append((np.array(zeros), np.sqrt(2) * h / h.sum()))
    return out


def _asymmetry_of_zeros(z):
    """Phase of prod (e^{-iw} - z_k) relative to w = 0, unwrapped, against its
    least-squares line through the origin: mean squared distance on 256
    midpoints of (0, pi).  The (1 + e^{-iw})^p factor of m0 has linear phase
    there and is left out."""
    w = np.pi * (np.arange(256) + 0.5) / 256
    v = np.prod(np.exp(-1j * w)[:, None] - z[None, :], axis=1) / np.prod(1 - z)
    ph = np.unwrap(np.angle(v))
    ph -= 2 * np.pi * np.round(ph[0] / (2 * np.pi))
    return np.mean((ph - (ph @ w) / (w @ w) * w) ** 2)


def _zeros_of(h, p):
    """Zeros of m0(z) = sum_n h_n z^n other than the p-fold zero at -1
    (numpy roots; the p roots nearest -1 are that zero)."""
    r = np.roots(h[::-1])
    return r[np.argsort(np.abs(r + 1))][p:]


@pytest.mark.parametrize("p", [4, 5, 6, 7, 8, 10])
def test_symlet_is_least_asymmetric_of_all_real_choices(p):
    hs = _h(Sym(p))
    cands = _all_real_candidates(p)
    assert len(cands) >= 4 and len(cands) & (len(cands) - 1) == 0   # 2^groups choices
    a = [_asymmetry_of_zeros(z) for z, _ in cands]
    assert _asymmetry_of_zeros(_zeros_of(hs, p)) <= min(a) * (1 + 1e-6)
    # it is one of the candidates, the least asymmetric one or its mirror image,
    # and not the extremal-phase filter
    i = int(np.argmin(a))
    assert min(np.abs(cands[i][1] - hs).max(), np.abs(cands[i][1][::-1] - hs).max()) < 1e-10
    assert np.abs(hs - _h(p)).max() > 0.1
    # energy in the first half of the taps
    e = hs ** 2
    assert (np.arange(hs.size) @ e) < (hs.size - 1) / 2 * e.sum()


def _mu(R, q, p):
    U = dense.U1d_scaling(R, q, p, W.VMP)
    return 1.0 / np.linalg.svd(U, compute_uv=False)[-1]


def test_table1_sym2_row():
    """Table 1, sym2 (VMP), through the symlet tables of the oracle (kept apart
    from the DB2 ones): 1D at M = 2^7 and 2D at M = 2^10 as for DB2."""
    tab = _table1()
    for q in range(1, 5):
        assert abs(_mu(7, q, Sym(2)) - tab[("sym2", 1)][q - 1]) < 2e-3
        assert abs(_mu(5, q, Sym(2)) ** 2 - tab[("sym2", 2)][q - 1]) < 4e-3


def test_table1_sym4_to_sym6_recorded():
    """Table 1 rows sym4..sym6 are not reproduced to the printed precision
    (the paper's boundary construction differs, as for DB3..DB6); the values
    of this reading lie within 3% of the printed ones, at least 1 and
    decreasing in q.  Recorded so that a change shows up."""
    tab = _table1()
    for p in (4, 5, 6):
        mus = [_mu(7, q, Sym(p)) for q in (1, 2, 3, 4)]
        assert all(m >= 1 - 1e-12 for m in mus)
        assert all(a > b for a, b in zip(mus, mus[1:]))
        assert all(abs(m - t) < 0.03 * t for m, t in zip(mus, tab[(f"sym{p}", 1)]))
