"""Walsh functions and the sequency-ordered Hadamard matrix (oracle).

Test infrastructure only.  Everything follows Def. 3.1 digit by digit:
for n = n^(1) 2^0 + n^(2) 2^1 + ... and x = x^(1) 2^-1 + x^(2) 2^-2 + ...,
w_n(x) = (-1)^{sum_j (n^(j) + n^(j+1)) x^(j)}.
Only dyadic points x = k / 2^L are needed; their expansion is finite.
"""
import numpy as np


def _ndigit(n, j):
    """n^(j): the j-th binary digit of the integer n (j >= 1, n^(1) = LSB)."""
    return (n >> (j - 1)) & 1


def _xdigit(k, L, j):
    """x^(j) of x = k / 2^L (0 <= k < 2^L): digits beyond L are zero."""
    if j > L:
        return 0 * k
    return (k >> (L - j)) & 1


def walsh(n, k, L):
    """w_n(k / 2^L) for integer arrays n, k (broadcasting), straight from
    Def. 3.1.  Digits of n above 2L do not matter because x^(j) = 0 for
    j > L; we still sum up to the highest digit of n for clarity."""
    n = np.asarray(n, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    top = max(int(n.max()).bit_length() if n.size else 0, L) + 1
    e = np.zeros(np.broadcast(n, k).shape, dtype=np.int64)
    for j in range(1, top + 1):
        e = e + (_ndigit(n, j) + _ndigit(n, j + 1)) * _xdigit(k, L, j)
    return np.where(e % 2 == 0, 1, -1).astype(np.int64)


def hadamard(N):
    """Sequency-ordered Hadamard matrix of Sec. 3.1 (0-based):
    H[n, k] = w_n(k / N), entries +-1, unnormalised."""
    L = int(N).bit_length() - 1
    assert 1 << L == N
    n = np.arange(N)[:, None]
    k = np.arange(N)[None, :]
    return walsh(n, k, L).astype(np.float64)


def xor_dyadic(a, b):
    """x (+) y of Def. 3.2 for dyadic rationals given as (numerator, L)."""
    return a ^ b


def sign_changes(row):
    """Number of sign changes along a sampled function."""
    row = np.asarray(row)
    return int(np.sum(row[1:] != row[:-1]))
