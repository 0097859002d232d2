"""Pins for the oracle's filters, cell integrals and restricted Gram (Sec. 3.2,
Lemma 3.4 / Sec. 4.1 taps)."""
from math import sqrt

import numpy as np
import pytest

from oracle import tables


def test_haar_and_db2_closed_forms():
    np.testing.assert_allclose(tables.daubechies(1), [1 / sqrt(2)] * 2, atol=1e-15)
    s3 = sqrt(3)
    want = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * sqrt(2))
    np.testing.assert_allclose(tables.daubechies(2), want, atol=2e-16)


def test_db3_closed_form():
    """Daubechies' closed form for three vanishing moments."""
    a, b = sqrt(10), sqrt(5 + 2 * sqrt(10))
    want = np.array([1 + a + b, 5 + a + 3 * b, 10 - 2 * a + 2 * b,
                     10 - 2 * a - 2 * b, 5 + a - 3 * b, 1 + a - b]) / (16 * sqrt(2))
    np.testing.assert_allclose(tables.daubechies(3), want, atol=3e-16)


@pytest.mark.parametrize("p", list(range(1, 11)) + [tables.Sym(p) for p in range(4, 11)])
def test_filter_conditions(p):
    """sum h = sqrt2, sum_k h_k h_{k+2l} = delta_l, and p vanishing moments:
    sum_k (-1)^k k^i h_k = 0 for i < p (g_k = (-1)^k h_{1-k} kills x^i)."""
    h = tables.daubechies(p)
    k = np.arange(-p + 1, p + 1)
    assert abs(h.sum() - sqrt(2)) < 1e-14
    for l in range(p):
        v = float(np.dot(h[: 2 * p - 2 * l], h[2 * l:]))
        assert abs(v - (1.0 if l == 0 else 0.0)) < 1e-14
    for i in range(p):
        assert abs(np.sum((-1.0) ** k * k.astype(float) ** i * h)) < 1e-12 * (p ** i + 1)
    g = tables.wavelet_filter(p)
    assert abs(g.sum()) < 1e-14
    # extremal phase in this orientation: the first coefficient is the largest
    # |partial energy| (minimum delay read from the left); symlets are oriented
    # by their energy centre instead (test_oracle_symlets)
    if not isinstance(p, tables.Sym):
        assert h[0] > 0


@pytest.mark.parametrize("p,q", [(1, 0), (1, 3), (2, 1), (2, 4), (3, 2), (4, 1), (6, 2), (8, 1),
                                 (tables.Sym(4), 2), (tables.Sym(8), 1)])
def test_cell_integral_invariants(p, q):
    I = tables.cell_integrals(p, q)
    Q = 2 ** q
    ts = sorted(I)
    assert ts[0] == (-p + 1) * Q and ts[-1] == p * Q - 1
    assert abs(sum(I.values()) - 1.0) < 1e-14                       # int phi = 1
    for t in range(Q):                                                # partition of unity
        s = sum(I.get(t + Q * n, 0.0) for n in range(-2 * p, 2 * p + 1))
        assert abs(s - 1.0 / Q) < 1e-14
    if p == 1:
        for t in ts:
            assert abs(I[t] - (1.0 / Q if 0 <= t < Q else 0.0)) < 1e-15
    if q > 0:                                                         # nested cells
        Ic = tables.cell_integrals(p, q - 1)
        for t, v in Ic.items():
            assert abs(I.get(2 * t, 0.0) + I.get(2 * t + 1, 0.0) - v) < 1e-15


@pytest.mark.parametrize("p", [3, 4, tables.Sym(4)])
def test_cell_integrals_against_quadrature(p):
    """Brute force: trapezoid sums of cascade point values at level 14."""
    K = 14
    P = tables.phi_dyadic(p, K)
    q = 2
    I = tables.cell_integrals(p, q)
    sub = 2 ** (K - q)
    for t, v in I.items():
        vals = np.array([P.get(t * sub + i, 0.0) for i in range(sub + 1)])
        quad = (vals.sum() - 0.5 * (vals[0] + vals[-1])) / 2 ** K
        assert abs(quad - v) < 2e-6, (t, quad, v)


@pytest.mark.parametrize("p", [3, 4])
def test_restricted_gram_against_quadrature(p):
    """G_{a,b} = int_0^inf phi(x-a) phi(x-b) dx vs. point-value quadrature."""
    K = 13
    P = tables.phi_dyadic(p, K)
    S = 2 ** K
    xs = np.arange(0, 3 * p * S + 1)
    for a in range(-p + 1, p):
        for b in range(a, p):
            fa = np.array([P.get(x - a * S, 0.0) for x in xs])
            fb = np.array([P.get(x - b * S, 0.0) for x in xs])
            f = fa * fb
            quad = (f.sum() - 0.5 * (f[0] + f[-1])) / S
            assert abs(quad - float(tables.gram_left_mp(p, a, b))) < 5e-6


@pytest.mark.parametrize("p", [2, 3, 5])
def test_gram_left_plus_right_is_identity_and_psd(p):
    tr = list(range(-p + 1, p))
    G = np.array([[float(tables.gram_left_mp(p, a, b)) for b in tr] for a in tr])
    assert np.all(np.linalg.eigvalsh(G) > -1e-14)
    assert np.allclose(G, G.T, atol=0)
