"""Reconstruction bases on [0,1] (oracle, test infrastructure only).

Sec. 3.2 of the paper: for level j the scaling basis B_{phi,j} holds p left
replacement functions, the interior phi_{j,m} for m = p..2^j-p-1, and p right
replacement functions; "rep" is either the periodic extension or the
vanishing-moments-preserving (Cohen-Daubechies-Vial) boundary functions.
C_{psi,j} = B_{phi,J0} u B_{psi,J0} u ... u B_{psi,j-1} is the wavelet basis
and the change of basis between the two is the DWT matrix W (Remark 4.2).

Layouts:
* 1D coefficient vectors of C_{psi,R}: [phi_{J0,.} | psi_{J0,.} | ... |
  psi_{R-1,.}], each level ordered by translate m = 0..2^j-1.
* 2D (Mallat square basis): the J0 scaling block in the top-left 2^J0 x 2^J0
  corner; at level j the detail blocks sit at [0:2^j, 2^j:2^{j+1}],
  [2^j:2^{j+1}, 0:2^j] and [2^j:2^{j+1}, 2^j:2^{j+1}].
"""
from functools import lru_cache

import numpy as np

from . import tables

PER, VMP = 0, 1


def default_J0(p):
    """Coarsest level: the p left and p right VMP edge functions at level J0
    must have disjoint supports, 2 (2p - 1) <= 2^J0.  Sec. 3.2 only asks
    J0 >= log2(2p) (some phi_{j,m} inside [0,1]); disjoint edges need one
    more doubling for p >= 2, and p = 1 needs 2^J0 >= 2 so that the left and
    the right replacement function are not the same function."""
    J = 0
    while (1 << J) < 2 * (2 * p - 1):
        J += 1
    return J


def cell_matrix(R, q, p, bd):
    """T[k, m] = int_{k/N}^{(k+1)/N} phi^rep_{R,m}, N = 2^{R+q}, M = 2^R.

    phi_{R,m}(x) = 2^{R/2} phi(2^R x - m), so the cell integral is
    2^{-R/2} I_q[k - 2^q m]; the edge functions are finite sums of
    translates (left: restricted to [0, inf), right: to (-inf, 0] after the
    change of variable y = 2^R (x - 1)), and periodic ones wrap mod N.
    """
    M, N = 2 ** R, 2 ** (R + q)
    I = tables.cell_integrals(p, q)
    T = np.zeros((N, M))
    if bd == PER:
        for m in range(M):
            for t, v in I.items():
                T[(t + 2 ** q * m) % N, m] += v
        return T * 2.0 ** (-R / 2)
    EL, ER = tables.edge_cells(p, q)
    n = EL.shape[1]
    for m in range(p, M - p):
        for t, v in I.items():
            T[t + 2 ** q * m, m] = v
    for m in range(p):
        T[:n, m] = EL[m]
        T[N - 1 - np.arange(n), M - 1 - m] = ER[m]
    return T * 2.0 ** (-R / 2)


@lru_cache(maxsize=None, typed=True)
def synthesis_matrix(j, p, bd):
    """S_j (2^{j+1} x 2^{j+1}): column c holds the B_{phi,j+1} coordinates of
    phi^rep_{j,c} (c < 2^j) or psi^rep_{j,c-2^j}; s_{j+1} = S_j [s_j; d_j]."""
    n0, n1 = 2 ** j, 2 ** (j + 1)
    h = tables.daubechies(p)
    g = tables.wavelet_filter(p)
    S = np.zeros((n1, n1))
    ks = range(-p + 1, p + 1)
    if bd == PER:
        for m in range(n0):
            for k in ks:
                S[(2 * m + k) % n1, m] += h[k + p - 1]
                S[(2 * m + k) % n1, n0 + m] += g[k + p - 1]
        return S
    PL, QL = tables.edge_blocks(p, "L")
    PR, QR = tables.edge_blocks(p, "R")
    for m in range(p):
        S[:PL.shape[1], m] = PL[m]
        S[:QL.shape[1], n0 + m] = QL[m]
        S[n1 - PR.shape[1]:, n0 - 1 - m] = PR[m][::-1]
        S[n1 - QR.shape[1]:, 2 * n0 - 1 - m] = QR[m][::-1]
    for m in range(p, n0 - p):
        for k in ks:
            S[2 * m + k, m] = h[k + p - 1]
            S[2 * m + k, n0 + m] = g[k + p - 1]
    return S


def idwt_matrix(R, J0, p, bd):
    """W^{-1} (M x M): C_{psi,R} coefficients -> B_{phi,R} coefficients."""
    M = 2 ** R
    W = np.eye(M)
    for j in range(J0, R):
        Sj = np.eye(M)
        Sj[:2 ** (j + 1), :2 ** (j + 1)] = synthesis_matrix(j, p, bd)
        W = Sj @ W
    return W


def idwt1d(x, J0, p, bd):
    R = int(x.shape[-1]).bit_length() - 1
    return x @ idwt_matrix(R, J0, p, bd).T


def dwt1d(s, J0, p, bd):
    R = int(s.shape[-1]).bit_length() - 1
    return s @ idwt_matrix(R, J0, p, bd)


def idwt2d(X, J0, p, bd):
    """Mallat IDWT on an M x M array (batch dims allowed in front)."""
    R = int(X.shape[-1]).bit_length() - 1
    X = np.array(X, dtype=np.float64, copy=True)
    for j in range(J0, R):
        n1 = 2 ** (j + 1)
        S = synthesis_matrix(j, p, bd)
        X[..., :n1, :n1] = S @ X[..., :n1, :n1] @ S.T
    return X


def dwt2d(X, J0, p, bd):
    """Mallat DWT (transpose of ``idwt2d``)."""
    R = int(X.shape[-1]).bit_length() - 1
    X = np.array(X, dtype=np.float64, copy=True)
    for j in range(R - 1, J0 - 1, -1):
        n1 = 2 ** (j + 1)
        S = synthesis_matrix(j, p, bd)
        X[..., :n1, :n1] = S.T @ X[..., :n1, :n1] @ S
    return X


def level_of_index(R, J0):
    """Level j of each 1D coefficient index (the J0 scaling block counts as
    level J0)."""
    lev = np.empty(2 ** R, dtype=np.int64)
    lev[:2 ** J0] = J0
    for j in range(J0, R):
        lev[2 ** j:2 ** (j + 1)] = j
    return lev
