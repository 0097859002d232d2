"""Pins for the oracle's Walsh functions and Hadamard matrix (Sec. 3.1)."""
import os

import numpy as np
import pytest

from oracle import fast, walsh

GOLD = os.path.join(os.path.dirname(__file__), "golden", "walsh_figure3.txt")


def test_walsh_matches_figure3():
    """Figure 3 (Sec. 3.1) draws w_0..w_7; their signs on the 8 cells."""
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    for n_str, pat in rows:
        n = int(n_str)
        want = np.array([1 if c == "+" else -1 for c in pat])
        got = walsh.walsh(n, np.arange(8), 3)
        assert np.array_equal(got, want), (n, got, want)
        # the same values on a finer dyadic grid (constant on each cell)
        fine = walsh.walsh(n, np.arange(64), 6)
        assert np.array_equal(fine, np.repeat(want, 8))


@pytest.mark.parametrize("L", [1, 3, 5, 7])
def test_sequency_sign_changes(L):
    """Sec. 3.1: w_n has exactly n sign changes (on [0,1))."""
    N = 2 ** L
    H = walsh.hadamard(N)
    for n in range(N):
        assert walsh.sign_changes(H[n]) == n


@pytest.mark.parametrize("L", [1, 2, 4, 6, 8])
def test_hadamard_orthogonal_symmetric(L):
    """H H^T = N I (orthogonality of the w_n on the cells) and H = H^T
    (second identity of Lemma 3.3 with n, l < 2^L)."""
    N = 2 ** L
    H = walsh.hadamard(N)
    assert np.array_equal(H @ H.T, N * np.eye(N))
    assert np.array_equal(H, H.T)


def test_lemma_3_3_identities():
    rng = np.random.default_rng(11)
    L = 9
    for _ in range(400):
        n = int(rng.integers(0, 1 << 12))
        x, y = (int(v) for v in rng.integers(0, 1 << L, 2))
        # w_n(x (+) y) = w_n(x) w_n(y)
        assert walsh.walsh(n, x ^ y, L) == walsh.walsh(n, x, L) * walsh.walsh(n, y, L)
        # w_n(2^-j l) = w_l(2^-j n) for n, l < 2^j
        j = int(rng.integers(1, 10))
        a, b = (int(v) for v in rng.integers(0, 1 << j, 2))
        assert walsh.walsh(a, b, j) == walsh.walsh(b, a, j)
        # w_n(2^-j x) = w_{floor(n / 2^j)}(x): x = k / 2^L scaled by 2^-j
        j = int(rng.integers(0, 5))
        k = int(rng.integers(0, 1 << L))
        assert walsh.walsh(n, k, L + j) == walsh.walsh(n >> j, k, L)


@pytest.mark.parametrize("L", [0, 1, 3, 6, 10])
def test_fwht_equals_hadamard_matrix(L):
    """The oracle's FWHT computes the N sums of Sec. 3.1 (sum_k w_n(k/N) x_k)."""
    N = 2 ** L
    rng = np.random.default_rng(L)
    x = rng.standard_normal((3, N))
    H = walsh.hadamard(N) if N <= 256 else None
    got = fast.fwht(x)
    if H is not None:
        np.testing.assert_allclose(got, x @ H.T, rtol=0, atol=1e-12 * N)
    # linearity / involution: H H = N I
    np.testing.assert_allclose(fast.fwht(got), N * x, rtol=0, atol=1e-10 * N)


def test_sequency_row_is_gray_bitreverse_free_definition():
    """r(n) derived digit by digit reproduces the full Walsh row."""
    L = 7
    N = 2 ** L
    r = fast.sequency_row(N)
    k = np.arange(N)
    for n in range(N):
        pc = np.array([bin(int(v)).count("1") for v in (r[n] & k)])
        assert np.array_equal((-1) ** pc, walsh.walsh(n, k, L))
