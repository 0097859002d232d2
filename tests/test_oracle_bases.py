"""Pins for the oracle's bases on [0,1]: boundary scaling functions, boundary
wavelets and the DWT (Sec. 3.2, Remark 4.2)."""
import numpy as np
import pytest

from oracle import tables, wavelets as W

PER, VMP = W.PER, W.VMP
Sym = tables.Sym


def _cellint_poly(k, N):
    e = np.arange(N + 1) / N
    return (e[1:] ** (k + 1) - e[:-1] ** (k + 1)) / (k + 1)


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8, Sym(4), Sym(6)])
def test_vmp_space_reproduces_polynomials(p):
    """Sec. 3.2: VMP boundary functions keep x^k, k < p, in V_j: the cell
    integrals of x^k lie in the range of T (exactly, not approximately)."""
    R, q = W.default_J0(p) + 1, 2
    T = W.cell_matrix(R, q, p, VMP)
    N = T.shape[0]
    for k in range(p):
        c = _cellint_poly(k, N)
        sol, *_ = np.linalg.lstsq(T, c, rcond=None)
        assert np.linalg.norm(T @ sol - c) < 1e-12 * np.linalg.norm(c)
    if p > 4:
        return                  # x^p is approximated to ~1e-11 and beyond
    # and x^p is not reproduced (so the test can fail)
    c = _cellint_poly(p, N)
    sol, *_ = np.linalg.lstsq(T, c, rcond=None)
    assert np.linalg.norm(T @ sol - c) > 1e-9 * np.linalg.norm(c)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8, Sym(4), Sym(6)])
@pytest.mark.parametrize("bd", [PER, VMP])
def test_scaling_basis_orthonormal(p, bd):
    """B_{phi,j} is orthonormal: as q grows, N T^T T -> I (the projection onto
    piecewise constants converges), and sigma_max(sqrt(N) T) <= 1."""
    R = W.default_J0(p)
    errs = []
    for q in (3, 6, 9):
        T = W.cell_matrix(R, q, p, bd)
        N = T.shape[0]
        G = N * T.T @ T
        assert np.linalg.norm(G, 2) <= 1 + 1e-12
        errs.append(np.abs(G - np.eye(G.shape[0])).max())
    assert errs[-1] < 0.2 * errs[0] + 1e-12 and errs[-1] < 5e-3


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8, Sym(4), Sym(6)])
def test_edge_functions_exact_orthonormality_and_support(p):
    # exact orthonormality, evaluated at the tables' working precision (the
    # float64 product cancels: translate coefficients are large where the
    # restricted translates are tiny)
    Amp, trL, Bmp, trR = tables._edges_mp(p)
    for E, tr, gram in ((Amp, trL, tables.gram_left_mp), (Bmp, trR, tables.gram_right_mp)):
        for a in range(p):
            for b in range(p):
                v = sum(E[a][i] * gram(p, tr[i], tr[j]) * E[b][j]
                        for i in range(len(tr)) for j in range(len(tr)))
                assert abs(float(v) - (1.0 if a == b else 0.0)) < 1e-30
    A, trL, B, trR = tables.edge_coefficients(p)
    for m in range(p):
        # supp phi^left_m = [0, p+m]: no translate beyond n = m
        assert all(A[m, j] == 0 or n <= m for j, n in enumerate(trL))
        assert A[m, trL.index(m)] > 0
        # supp phi^right_m = [-m-p, 0]: no translate below n = -m-1
        assert all(B[m, j] == 0 or n >= -m - 1 for j, n in enumerate(trR))
        assert B[m, trR.index(-m - 1)] > 0
    # cell integrals vanish outside the stated supports
    q = 2
    T = W.cell_matrix(W.default_J0(p) + 1, q, p, VMP)
    N, M = T.shape
    for m in range(p):
        assert np.all(T[2 ** q * (p + m):, m] == 0)
        assert np.all(T[: N - 2 ** q * (p + m), M - 1 - m] == 0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 8, Sym(4), Sym(5)])
@pytest.mark.parametrize("bd", [PER, VMP])
def test_dwt_orthogonal(p, bd):
    J0 = W.default_J0(p)
    for R in (J0, J0 + 1, J0 + 3):
        Wi = W.idwt_matrix(R, J0, p, bd)
        assert np.abs(Wi @ Wi.T - np.eye(2 ** R)).max() < 1e-13


@pytest.mark.parametrize("p", [2, 3, 4, 6, Sym(4), Sym(6)])
def test_vmp_wavelets_have_vanishing_moments_at_edges(p):
    """VMP (Sec. 3.2): detail coefficients of x^k (k < p) vanish, including
    the boundary wavelets; the periodic basis loses this at the edges."""
    J0 = W.default_J0(p)
    R, q = J0 + 2, 2
    for bd, expect_zero in ((VMP, True), (PER, False)):
        T = W.cell_matrix(R, q, p, bd)
        Wi = W.idwt_matrix(R, J0, p, bd)
        worst = 0.0
        for k in range(1, p):
            c, *_ = np.linalg.lstsq(T, _cellint_poly(k, T.shape[0]), rcond=None)
            x = Wi.T @ c                       # C_{psi,R} coefficients
            worst = max(worst, np.abs(x[2 ** J0:]).max())
        if expect_zero:
            assert worst < 1e-12
        else:
            assert worst > 1e-4


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8, Sym(4), Sym(8)])
def test_boundary_wavelet_supports(p):
    """psi^left_m uses level-1 coordinates up to p + 2m only (supp [0, p+m]);
    same mirrored on the right; p = 1 reduces to the Haar wavelet."""
    for side in ("L", "R"):
        P, Q = tables.edge_blocks(p, side)
        for m in range(p):
            nz = np.flatnonzero(np.abs(Q[m]) > 1e-15)
            assert nz.max() == p + 2 * m
        assert np.abs(P @ P.T - np.eye(p)).max() < 1e-13
        assert np.abs(Q @ Q.T - np.eye(p)).max() < 1e-13
        assert np.abs(P @ Q.T).max() < 1e-13
    if p == 1:
        for bd_p in range(1):
            S_per = W.synthesis_matrix(3, 1, PER)
            S_vmp = W.synthesis_matrix(3, 1, VMP)
            assert np.abs(S_per - S_vmp).max() < 1e-15


@pytest.mark.parametrize("p", [2, 3, 4])
def test_periodic_dwt_constant_and_shift(p):
    """Periodic DWT: the constant function (all level-R coefficients 2^{-R/2})
    has no details and J0 coefficients 2^{-J0/2}; shifting s by 2 shifts every
    subband by 1 (circular convolution, Sec. 3.2)."""
    J0, R = 2, 6
    Wi = W.idwt_matrix(R, J0, p, PER)
    s = np.full(2 ** R, 2.0 ** (-R / 2))
    x = Wi.T @ s
    assert np.abs(x[2 ** J0:]).max() < 1e-14
    assert np.abs(x[: 2 ** J0] - 2.0 ** (-J0 / 2)).max() < 1e-14
    S = W.synthesis_matrix(R - 1, p, PER)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(2 ** R)
    a = S.T @ v
    b = S.T @ np.roll(v, 2)
    n0 = 2 ** (R - 1)
    assert np.abs(np.roll(a[:n0], 1) - b[:n0]).max() < 1e-14
    assert np.abs(np.roll(a[n0:], 1) - b[n0:]).max() < 1e-14


def test_mallat_2d_is_levelwise_separable():
    p, bd = 2, VMP
    J0 = W.default_J0(p)
    R = J0 + 2
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2 ** R, 2 ** R))
    S = W.idwt2d(X, J0, p, bd)
    np.testing.assert_allclose(W.idwt2d(X.T, J0, p, bd), S.T, atol=1e-13)
    np.testing.assert_allclose(W.dwt2d(S, J0, p, bd), X, atol=1e-13)
