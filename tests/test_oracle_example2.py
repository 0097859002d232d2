"""Pins of the oracle's sampling model against the paper's Example 2 (Sec. 6):
the truncated Walsh series and generalised sampling with DB2 boundary
wavelets of f(t1, t2) = cos(3 pi t1 / 2) sin(3 pi t2) from its 32 x 32 first
Walsh samples (relative errors printed in the figure caption,
tests/golden/example2.txt).

Both reconstructions are separable for this separable f: the 2D samples are
c1 (x) c2 with c_n = <f_i, w_n> (Def. 3.1), the truncated Walsh series is the
product of the 1D series, and the generalised-sampling least-squares problem
min ||(A (x) A) z - c1 (x) c2|| (A = P_N U P_M in any orthonormal basis of the
reconstruction space, Sec. 1.2) is solved by A^+ c1 (x) A^+ c2.  The errors
are then exact L2 errors on [0, 1]^2 from 1D inner products."""
import os

import numpy as np
import pytest

from oracle import dense, walsh, wavelets as W

scipy_integrate = pytest.importorskip("scipy.integrate")

GOLD = os.path.join(os.path.dirname(__file__), "golden", "example2.txt")
F1 = (lambda t: np.cos(1.5 * np.pi * t))
F2 = (lambda t: np.sin(3.0 * np.pi * t))
NS = 32          # Walsh samples per dimension
TOL = 5e-4       # the paper's point evaluation moves the 4th decimal


def _gold():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        out[k] = float(v)
    return out


def _cells(f, n):
    """exact integrals of f over the cells [k/n, (k+1)/n)"""
    quad = scipy_integrate.quad
    return np.array([quad(f, k / n, (k + 1) / n)[0] for k in range(n)])


def _norm2(f):
    return scipy_integrate.quad(lambda t: f(t) ** 2, 0.0, 1.0, limit=200)[0]


def _walsh_coeffs(f, n):
    """<f, w_k> for k < n: w_k is constant on cells of width 1/n (Def. 3.1)"""
    return walsh.hadamard(n) @ _cells(f, n)


def test_truncated_walsh_series_error():
    """TW: f~ = sum_{n < 32} <f, w_n> w_n per dimension, evaluated from the
    oracle's Walsh functions on a grid 8 times finer than the cells and
    integrated exactly against f (f~ is constant on the fine cells)."""
    L = 8
    n = 2 ** L
    err2_num, fnorm2 = 1.0, 1.0
    parts = []
    for f in (F1, F2):
        c = _walsh_coeffs(f, NS)
        # w_k(j / n) for the fine grid: the first 5 digits decide the value
        wfine = np.array([[walsh.walsh(k, j, L) for j in range(n)] for k in range(NS)], dtype=np.float64)
        ft = c @ wfine                             # f~ on the fine cells
        inner = np.dot(ft, _cells(f, n))          # <f, f~>
        parts.append((_norm2(f), inner, np.sum(ft ** 2) / n))
    (a1, i1, g1), (a2, i2, g2) = parts
    err = np.sqrt((a1 * a2 - 2 * i1 * i2 + g1 * g2) / (a1 * a2))
    assert abs(err - _gold()["TW"]) < TOL, err


def _gs_1d(f, p, R):
    q = int(np.log2(NS)) - R
    A = dense.U1d_scaling(R, q, p, W.VMP)             # 32 x M, orthonormal basis of V_R
    z, *_ = np.linalg.lstsq(A, _walsh_coeffs(f, NS), rcond=None)
    # <f, phi_m> from Parseval on the first 2^12 Walsh functions (smooth f:
    # the tail is far below the tolerance)
    nf = 2 ** 12
    Af = dense.U1d_scaling(R, 12 - R, p, W.VMP)
    fr = _walsh_coeffs(f, nf) @ Af
    return _norm2(f), fr @ z, z @ z


def test_generalised_sampling_db2_error():
    """GS with DB2 (p = 2, VMP boundaries) at M = 16 x 16 (R = 4, q = 1)."""
    (a1, i1, g1), (a2, i2, g2) = _gs_1d(F1, 2, 4), _gs_1d(F2, 2, 4)
    err = np.sqrt((a1 * a2 - 2 * i1 * i2 + g1 * g2) / (a1 * a2))
    assert abs(err - _gold()["DB2"]) < TOL, err
