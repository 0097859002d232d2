"""Pins for the oracle's U (Sec. 1.2, Sec. 4, Algorithm 1, Algorithm 2, Table 1,
Remark 4.3)."""
import os

import numpy as np
import pytest

from oracle import dense, fast, tables, walsh, wavelets as W

PER, VMP = W.PER, W.VMP
GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def _table1():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, dim, *vals = line.split()
        out[(name, int(dim))] = [float(v) for v in vals]
    return out


def _mu(R, q, p):
    U = dense.U1d_scaling(R, q, p, VMP)
    return 1.0 / np.linalg.svd(U, compute_uv=False)[-1]


GOLD_ORACLE = os.path.join(os.path.dirname(__file__), "golden", "table1_oracle.txt")


def _table1_oracle():
    """Rows of table1_oracle.txt: (name, dim, q) -> (oracle, printed, agrees)."""
    out = {}
    for line in open(GOLD_ORACLE):
        if line.startswith("#") or not line.strip():
            continue
        name, dim, q, v, pr, _, ok = line.split()
        out[(name, int(dim), int(q))] = (float(v), float(pr), ok == "1")
    return out


def _mu_cell(name, dim, q):
    p = int(name[-1])
    pp = tables.Sym(p) if name.startswith("sym") else p
    R = 7 if dim == 1 else 5
    U = dense.U1d_scaling(R, q, pp, VMP)
    m = 1.0 / np.linalg.svd(U, compute_uv=False)[-1]
    return m if dim == 1 else m * m


def test_table1_printed_cells_reproduced_to_printed_precision():
    """Table 1 (Sec. 4), mu = 1 / sigma_M(P_N U P_M), VMP boundary: every cell
    that the recorded comparison marks as agreeing is reproduced by the oracle
    to the printed precision, |mu - printed| <= 5e-4 (1D at M = 2^7; 2D at
    M = 2^5 x 2^5, where P_N U P_M is a Kronecker product, so mu is the square
    of the 1D value).  These are DB2 / sym2 at q = 1 and 4 (1D), sym4 at q = 4
    (1D) and DB4 at q = 4 (2D).  The other cells are not reproduced by this
    reading of the boundary functions; their differences are pinned as numbers
    by the next test."""
    tab = _table1_oracle()
    agreeing = [k for k, (_, _, ok) in tab.items() if ok]
    assert ("DB2", 1, 1) in agreeing and ("DB2", 1, 4) in agreeing
    for name, dim, q in agreeing:
        printed = _table1()[(name, dim)][q - 1]
        assert abs(_mu_cell(name, dim, q) - printed) <= 5e-4, (name, dim, q)


def test_table1_every_cell_recorded():
    """Every cell of Table 1 (1D and 2D, DB2..DB6, sym2..sym6, q = 1..4): the
    oracle's mu equals the value recorded beside the printed one in
    tests/golden/table1_oracle.txt (written by make_table1_oracle.py from the
    oracle alone), so the disagreement with the printed table (e.g. DB3 1D
    q = 1: 4.0856 against 2.610; DB2 1D q = 2: 1.0512 against 1.050) is a
    stated number and any change to the boundary space shows up here.  The
    printed table itself is checked against the recorded one, so the two
    files cannot drift apart."""
    tab = _table1_oracle()
    printed = _table1()
    assert len(tab) == 80
    for (name, dim, q), (v, pr, ok) in tab.items():
        assert pr == printed[(name, dim)][q - 1]
        assert ok == (abs(v - pr) <= 5e-4)
        assert abs(_mu_cell(name, dim, q) - v) <= 2e-6 * v, (name, dim, q)
    # sym2 / sym3 are the extremal-phase filters (the printed rows are equal)
    for dim in (1, 2):
        for q in (1, 2, 3, 4):
            assert tab[("sym2", dim, q)][0] == tab[("DB2", dim, q)][0]
            assert tab[("sym3", dim, q)][0] == tab[("DB3", dim, q)][0]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("bd", [PER, VMP])
def test_norm_at_most_one(p, bd):
    J0 = W.default_J0(p)
    U = dense.U1d(J0 + 1, 1, p, bd, J0)
    assert np.linalg.norm(U, 2) <= 1 + 1e-12


@pytest.mark.parametrize("q", [0, 1, 3])
def test_haar_U_is_isometry(q):
    """Remark 4.3: with Haar and N = M, P_M U P_M = H W^{-1} is orthogonal; for
    q > 0 the Haar functions are still piecewise constant on the sampling
    cells, so U^T U = I."""
    R = 4
    U = dense.U1d(R, q, 1, PER, 1)
    np.testing.assert_allclose(U.T @ U, np.eye(2 ** R), atol=1e-13)
    if q == 0:
        np.testing.assert_allclose(U @ U.T, np.eye(2 ** R), atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("bd", [PER, VMP])
def test_constant_function(p, bd):
    """<1, w_n> = delta_{n0}: the coefficients of f = 1 map to e_0."""
    J0 = W.default_J0(p)
    R, q = J0 + 1, 2
    T = W.cell_matrix(R, q, p, bd)
    N = T.shape[0]
    c, *_ = np.linalg.lstsq(T, np.full(N, 1.0 / N), rcond=None)
    x = W.idwt_matrix(R, J0, p, bd).T @ c
    y = dense.U1d(R, q, p, bd, J0) @ x
    e0 = np.zeros(N)
    e0[0] = 1
    np.testing.assert_allclose(y, e0, atol=1e-13)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_linear_function_walsh_coefficients(p):
    """f(x) = x lies in the VMP space for p >= 2; its Walsh coefficients are
    1/2 at n = 0, -2^{-k-1} at n = 2^k - 1 (w_{2^k-1} is the k-th Rademacher
    function) and 0 elsewhere."""
    J0 = W.default_J0(p)
    R, q = J0 + 1, 2
    T = W.cell_matrix(R, q, p, VMP)
    N = T.shape[0]
    e = np.arange(N + 1) / N
    c, *_ = np.linalg.lstsq(T, (e[1:] ** 2 - e[:-1] ** 2) / 2, rcond=None)
    x = W.idwt_matrix(R, J0, p, VMP).T @ c
    y = dense.U1d(R, q, p, VMP, J0) @ x
    want = np.zeros(N)
    want[0] = 0.5
    k = 1
    while 2 ** k - 1 < N:
        want[2 ** k - 1] = -(2.0 ** (-k - 1))
        k += 1
    np.testing.assert_allclose(y, want, atol=1e-13)


@pytest.mark.parametrize("p", [3, 4])
@pytest.mark.parametrize("bd", [PER, VMP])
def test_brute_force_inner_products(p, bd):
    """U_{n,m} = <phi^rep_{R,m}, w_n> by trapezoid quadrature of cascade point
    values of phi (no cell integrals, no I_q): w_n is constant on each grid
    interval, so the only error is the quadrature of phi."""
    J0 = W.default_J0(p)
    R, q = J0, 1
    M, N = 2 ** R, 2 ** (R + q)
    K = 16                                   # x grid: x_i = i / 2^K
    P = tables.phi_dyadic(p, K - R)          # phi at multiples of 2^-(K-R)
    A, trL, B, trR = tables.edge_coefficients(p)
    xs = np.arange(2 ** K + 1)
    S = 2 ** (K - R)                         # phi argument 2^R x - m = (i - m S) / S

    def phi_at(num):
        return np.array([P.get(int(v), 0.0) for v in num])

    cols = np.zeros((xs.size, M))
    for m in range(M):
        if bd == PER:
            v = sum(phi_at(xs - (m + w * M) * S) for w in (-1, 0, 1))
        elif p <= m < M - p:
            v = phi_at(xs - m * S)
        elif m < p:
            v = sum(A[m, j] * phi_at(xs - n * S) for j, n in enumerate(trL))
        else:
            v = sum(B[M - 1 - m, j] * phi_at(xs - (n + M) * S) for j, n in enumerate(trR))
        cols[:, m] = 2 ** (R / 2) * v
    trap = 0.5 * (cols[:-1] + cols[1:]) / 2 ** K
    wn = walsh.walsh(np.arange(N)[:, None], xs[None, :-1], K)
    Ubf = wn @ trap
    U = dense.U1d_scaling(R, q, p, bd)
    assert np.abs(Ubf - U).max() < 2e-5


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("bd", [PER, VMP])
def test_dense_equals_algorithm1(p, bd):
    """The dense definition and Algorithm 1 (sum_l D_l H_l, Prop. 4.4 edges,
    Lemma 3.4) agree, forward and adjoint."""
    J0 = W.default_J0(p)
    rng = np.random.default_rng(p + 10 * bd)
    for R, q in ((J0, 1), (J0 + 2, 2)):
        M, N = 2 ** R, 2 ** (R + q)
        x = rng.standard_normal((2, M))
        y = rng.standard_normal((2, N))
        np.testing.assert_allclose(fast.forward1d(x, R, q, p, bd, J0),
                                   dense.forward1d(x, R, q, p, bd, J0), atol=1e-13)
        np.testing.assert_allclose(fast.adjoint1d(y, R, q, p, bd, J0),
                                   dense.adjoint1d(y, R, q, p, bd, J0), atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("bd", [PER, VMP])
def test_dense_equals_algorithm2(p, bd):
    J0 = W.default_J0(p)
    R, q = J0 + 1, 1
    M, N = 2 ** R, 2 ** (R + q)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((M, M))
    om = np.sort(rng.choice(N * N, size=N * N // 3, replace=False))
    y = rng.standard_normal(om.size)
    np.testing.assert_allclose(fast.forward2d(x, R, q, p, bd, J0, om),
                               dense.forward2d(x, R, q, p, bd, J0, om), atol=1e-13)
    np.testing.assert_allclose(fast.adjoint2d(y, R, q, p, bd, J0, om),
                               dense.adjoint2d(y, R, q, p, bd, J0, om), atol=1e-13)


def test_2d_is_kronecker_of_1d():
    """With Omega = all and J0 = R (no IDWT), alpha = G xi G^T equals the
    Kronecker product (G (x) G) vec(xi)."""
    p, R, q = 2, 3, 1
    G = dense.G1d(R, q, p, VMP)
    rng = np.random.default_rng(5)
    xi = rng.standard_normal((2 ** R, 2 ** R))
    a = dense.forward2d(xi, R, q, p, VMP, R)
    np.testing.assert_allclose(a, np.kron(G, G) @ xi.ravel(), atol=1e-13)


@pytest.mark.parametrize("bd", [PER, VMP])
def test_dot_product_adjoint(bd):
    p = 3
    J0 = W.default_J0(p)
    R, q = J0 + 1, 1
    M, N = 2 ** R, 2 ** (R + q)
    rng = np.random.default_rng(9)
    om = np.sort(rng.choice(N * N, size=N * N // 4, replace=False))
    x = rng.standard_normal((M, M))
    y = rng.standard_normal(om.size)
    lhs = np.dot(dense.forward2d(x, R, q, p, bd, J0, om), y)
    rhs = np.sum(x * dense.adjoint2d(y, R, q, p, bd, J0, om))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)
