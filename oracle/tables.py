"""High-precision tables for the oracle (test infrastructure only).

Everything here is input independent: it depends on the number of vanishing
moments p (the paper's nu) and, for the cell integrals, on q.  All arithmetic
is done in mpmath at ``DPS`` digits and the results are returned as float64
numpy arrays (or dicts of floats) so that the rest of the oracle can use plain
numpy.

Conventions (Sec. 3.2): supp(phi) = supp(psi) = [-p+1, p]; the scaling filter
h_k lives on k = -p+1..p and phi(x) = sqrt(2) sum_k h_k phi(2x - k); the
wavelet filter is g_k = (-1)^k h_{1-k}.
"""
from fractions import Fraction
from functools import lru_cache
from math import comb

import mpmath as mp
import numpy as np

DPS = 60


def _mp():
    mp.mp.dps = DPS
    return mp


# ----------------------------------------------------------------------------
# Daubechies filters (Sec. 3.2: orthonormal, compactly supported, p vanishing
# moments, minimal support).  "Daubechies wavelet" = extremal phase; the
# symlets of Table 1 are the least-asymmetric choice among the same family.
# ----------------------------------------------------------------------------
class Sym(int):
    """p for the least-asymmetric Daubechies filter (symlet) with p vanishing
    moments.  It behaves as the integer p everywhere; the table caches are
    typed, so its tables are kept apart from the extremal-phase ones."""

    def __repr__(self):
        return f"Sym({int(self)})"


def _reciprocal_roots(m, p):
    """Daubechies' construction: |m0(xi)|^2 = cos^{2p}(xi/2) P(sin^2(xi/2))
    with P(y) = sum_{k<p} C(p-1+k, k) y^k.  Each root y of P gives a
    reciprocal pair z, 1/z of z^2 - (2 - 4y) z + 1.  Returns the pairs as
    (z outside the unit circle, its reciprocal), one per root of P."""
    if p == 1:
        return []
    coeffs = [m.mpf(comb(p - 1 + k, k)) for k in range(p)][::-1]
    out = []
    for y in m.polyroots(coeffs, maxsteps=400, extraprec=4 * DPS):
        b = 2 - 4 * y
        d = m.sqrt(b * b - 4)
        z1, z2 = (b + d) / 2, (b - d) / 2
        out.append((z1, z2) if abs(z1) > 1 else (z2, z1))
    return out


def _filter_from_zeros(m, p, zeros):
    """h_k, k = -p+1..p (mpf list), of m0(z) = sum h_k z^{k+p-1} with a zero
    of order p at z = -1 and the given other zeros, normalised to sum h = sqrt2."""
    Q = [m.mpc(1)]
    for _ in range(p):
        Q = _polymul(Q, [m.mpc(1), m.mpc(1)])
    for z in zeros:
        Q = _polymul(Q, [-z, m.mpc(1)])
    re = [c.real for c in Q]
    s = sum(re)
    return [m.sqrt(2) * c / s for c in re]


ASYM_GRID = 256


def phase_asymmetry(zeros):
    """Asymmetry of the filter whose m0 has zeros of order p at -1 and the
    given other zeros: m0(e^{-iw}) = c (1 + e^{-iw})^p R(e^{-iw}) with
    R(z) = prod (z - z_k).  On (0, pi) the first factor has the exactly linear
    phase -p w / 2, so the deviation of the phase of m0 from a line through
    the origin is that of psi(w) = arg R(e^{-iw}) - arg R(1) (unwrapped); this
    is the mean squared distance of psi from its least-squares line through
    the origin on w_k = pi (k + 1/2) / 256, k < 256.  (Evaluating m0 itself
    there is ill-conditioned near w = pi, where it has a zero of order p.)"""
    z = np.asarray([complex(v) for v in zeros])
    w = np.pi * (np.arange(ASYM_GRID) + 0.5) / ASYM_GRID
    e = np.exp(-1j * w)
    Rw = np.prod(e[:, None] - z[None, :], axis=1) if z.size else np.ones_like(e)
    psi = np.unwrap(np.angle(Rw))
    psi = psi - np.angle(np.prod(1 - z)) if z.size else psi
    # psi(0+) must be near 0 after the shift; take the branch nearest 0
    psi = psi - 2 * np.pi * np.round(psi[0] / (2 * np.pi))
    b = (psi @ w) / (w @ w)
    return float(np.mean((psi - b * w) ** 2))


def _front_loaded(h):
    """True if the energy centre sum n h_n^2 lies in the first half of 0..2p-1."""
    e = [float(v) ** 2 for v in h]
    return sum(i * v for i, v in enumerate(e)) < (len(e) - 1) / 2 * sum(e)


@lru_cache(maxsize=None, typed=True)
def daubechies_mp(p):
    """Daubechies filter h_k, k = -p+1..p, as mpf list.

    Extremal phase (p an int): every zero of m0 other than z = -1 is the
    member of its reciprocal pair outside the unit circle (the classical
    table, h_0 largest first).  Least asymmetric (p a ``Sym``): among the
    choices of one member per pair (a complex pair of P's roots chosen
    together, so that h is real), the one whose phase_asymmetry is smallest;
    a choice and its complement give mirror-image filters with the same
    asymmetry, and the one whose energy lies in the first half is kept (for
    p <= 3 this is the extremal-phase filter again, as Table 1's equal
    DB2/sym2 and DB3/sym3 rows say)."""
    m = _mp()
    pairs = _reciprocal_roots(m, int(p))
    if not isinstance(p, Sym):
        return _filter_from_zeros(m, int(p), [zo for zo, _ in pairs])
    # groups: a real root of P, or a root with positive imaginary part together
    # with its conjugate
    tol = m.mpf(10) ** (-DPS // 2)
    groups, used = [], [False] * len(pairs)
    ys = [(2 - (zo + zi)) / 4 for zo, zi in pairs]      # back to the root y of P
    for i in range(len(pairs)):
        if used[i]:
            continue
        used[i] = True
        if abs(ys[i].imag) < tol:
            groups.append([i])
            continue
        j = min((k for k in range(len(pairs)) if not used[k]), key=lambda k: abs(ys[k] - m.conj(ys[i])))
        used[j] = True
        groups.append([i, j])
    best = None
    for mask in range(1 << max(len(groups) - 1, 0)):     # group 0 fixed: one of each mirror pair
        zeros = []
        for g, idx in enumerate(groups):
            inside = g > 0 and (mask >> (g - 1)) & 1
            zeros += [pairs[i][1] if inside else pairs[i][0] for i in idx]
        a = phase_asymmetry(zeros)
        if best is None or a < best[0]:
            best = (a, zeros)
    h = _filter_from_zeros(m, int(p), best[1])
    return h if _front_loaded(h) else h[::-1]


def _polymul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _h(hl, p, k):
    i = k + p - 1
    return hl[i] if 0 <= i < 2 * p else 0


def daubechies(p):
    """h as float64 array indexed 0..2p-1 <-> k = -p+1..p."""
    return np.array([float(x) for x in daubechies_mp(p)])


def wavelet_filter(p):
    """g_k = (-1)^k h_{1-k}, k = -p+1..p, float64 array like ``daubechies``."""
    h = daubechies_mp(p)
    return np.array([float((-1) ** (k % 2) * _h(h, p, 1 - k)) for k in range(-p + 1, p + 1)])


# ----------------------------------------------------------------------------
# Exact cell integrals of phi.  I_q[t] = int_{t/2^q}^{(t+1)/2^q} phi, the
# "precomputed integrals" behind the taps W phi_{0,-l}(s) of Sec. 4.1.
# ----------------------------------------------------------------------------
@lru_cache(maxsize=None, typed=True)
def _cells_mp(p, q):
    m = _mp()
    h = daubechies_mp(p)
    ts = list(range(-p + 1, p))
    n = len(ts)
    # integer cells: J[t] = (1/sqrt2) sum_k h_k (J[2t-k] + J[2t-k+1]); the
    # eigenvector for eigenvalue 1, normalised by sum J = int phi = 1.
    A = m.matrix(n, n)
    for a, t in enumerate(ts):
        for b, u in enumerate(ts):
            A[a, b] = (_h(h, p, 2 * t - u) + _h(h, p, 2 * t - u + 1)) / m.sqrt(2)
            if a == b:
                A[a, b] -= 1
    rhs = m.matrix(n, 1)
    for b in range(n):
        A[n - 1, b] = 1
    rhs[n - 1] = 1
    J = m.lu_solve(A, rhs)
    cur = {t: J[a] for a, t in enumerate(ts)}
    # finer cells: I_q[t] = (1/sqrt2) sum_k h_k I_{q-1}[t - 2^{q-1} k]
    for qq in range(1, q + 1):
        new = {}
        for t in range((-p + 1) * 2 ** qq, p * 2 ** qq):
            s = 0
            for k in range(-p + 1, p + 1):
                s += _h(h, p, k) * cur.get(t - 2 ** (qq - 1) * k, 0)
            new[t] = s / m.sqrt(2)
        cur = new
    return cur


def cell_integrals(p, q):
    """dict t -> I_q[t] (float64) for t in [(-p+1) 2^q, p 2^q - 1]."""
    return {t: float(v) for t, v in _cells_mp(p, q).items()}


# ----------------------------------------------------------------------------
# Restricted Gram matrix G_{a,b} = int_0^inf phi(x-a) phi(x-b) dx.  Exact
# from the two-scale relation G_{a,b} = sum_{k,l} h_k h_l G_{2a+k, 2b+l},
# with G = delta when a translate lies in [0, inf) and G = 0 when one lies in
# (-inf, 0].
# ----------------------------------------------------------------------------
@lru_cache(maxsize=None, typed=True)
def _gram_left_mp(p):
    m = _mp()
    h = daubechies_mp(p)
    idx = list(range(-p + 1, p - 1))
    pairs = [(a, b) for a in idx for b in idx if a <= b]
    pos = {pr: i for i, pr in enumerate(pairs)}
    n = len(pairs)
    if n == 0:
        return {}
    A = m.eye(n)
    rhs = m.matrix(n, 1)
    for (a, b), r in pos.items():
        for k in range(-p + 1, p + 1):
            for l in range(-p + 1, p + 1):
                c, d = 2 * a + k, 2 * b + l
                if c <= -p or d <= -p:
                    continue
                coef = h[k + p - 1] * h[l + p - 1]
                if c >= p - 1 or d >= p - 1:
                    if c == d:
                        rhs[r] += coef
                    continue
                key = (c, d) if c <= d else (d, c)
                A[r, pos[key]] -= coef
    sol = m.lu_solve(A, rhs)
    return {pr: sol[i] for pr, i in pos.items()}


def gram_left_mp(p, a, b):
    """int_0^inf phi(x-a) phi(x-b) dx (mpf)."""
    if a <= -p or b <= -p:
        return _mp().mpf(0)
    if a >= p - 1 or b >= p - 1:
        return _mp().mpf(1 if a == b else 0)
    g = _gram_left_mp(p)
    return g[(a, b) if a <= b else (b, a)]


def gram_right_mp(p, a, b):
    """int_{-inf}^0 phi(x-a) phi(x-b) dx = delta_ab - int_0^inf (...)."""
    return _mp().mpf(1 if a == b else 0) - gram_left_mp(p, a, b)


# ----------------------------------------------------------------------------
# Boundary scaling functions (Sec. 3.2, Cohen-Daubechies-Vial).  The left edge
# space is { sum_{n=-p+1}^{p-1} c(n) phi(.-n)|_[0,inf) : c a polynomial of
# degree < p }, the part of the polynomials x^k (k < p) on [0, inf) that the
# kept interior translates n >= p do not carry.  phi^left_m is the unit vector
# of the subspace with coefficients vanishing for n > m, orthogonal to the one
# for n > m-1: supp phi^left_m = [0, p+m].  Sign: coefficient of phi(.-m) > 0.
# The right edge is the same construction on (-inf, 0] with translates
# n = -p..p-2, nodes -1, -2, ..: supp phi^right_m = [-m-p, 0].
# ----------------------------------------------------------------------------
def _lagrange(nodes, i, x):
    """Lagrange basis polynomial of nodes[i] at x, in exact rationals (the
    polynomial weights must be exact: rounding them moves the edge space)."""
    v = Fraction(1)
    for k in nodes:
        if k != nodes[i]:
            v = v * Fraction(x - k, nodes[i] - k)
    return v


def _mpq(fr):
    return _mp().mpf(fr.numerator) / fr.denominator


def _gs(vectors, G):
    m = _mp()
    out = []
    for v in vectors:
        w = list(v)
        for _ in range(2):
            for u in out:
                c = sum(u[i] * G[i][j] * w[j] for i in range(len(w)) for j in range(len(w)))
                w = [w[i] - c * u[i] for i in range(len(w))]
        nrm = m.sqrt(sum(w[i] * G[i][j] * w[j] for i in range(len(w)) for j in range(len(w))))
        out.append([x / nrm for x in w])
    return out


@lru_cache(maxsize=None, typed=True)
def _edges_mp(p):
    m = _mp()
    trL = list(range(-p + 1, p))
    GL = [[gram_left_mp(p, a, b) for b in trL] for a in trL]
    nodesL = list(range(0, p))
    A = _gs([[_mpq(_lagrange(nodesL, i, n)) for n in trL] for i in range(p)], GL)
    trR = list(range(-p, p - 1))
    GR = [[gram_right_mp(p, a, b) for b in trR] for a in trR]
    nodesR = [-(i + 1) for i in range(p)]
    B = _gs([[_mpq(_lagrange(nodesR, i, n)) for n in trR] for i in range(p)], GR)
    return A, trL, B, trR


@lru_cache(maxsize=None, typed=True)
def _edge_cells_mp(p, q):
    m = _mp()
    A, trL, B, trR = _edges_mp(p)
    I = _cells_mp(p, q)
    Q = 2 ** q
    n = (2 * p - 1) * Q
    EL = [[sum(A[r][j] * I.get(k - Q * t, 0) for j, t in enumerate(trL)) for k in range(n)] for r in range(p)]
    ER = [[sum(B[r][j] * I.get(-(k + 1) - Q * t, 0) for j, t in enumerate(trR)) for k in range(n)] for r in range(p)]
    return EL, ER


def edge_cells(p, q):
    """(EL, ER), p x (2p-1) 2^q float64: EL[m][k] = int_{k/2^q}^{(k+1)/2^q}
    phi^left_m and ER[m][k] = int_{-(k+1)/2^q}^{-k/2^q} phi^right_m, summed at
    the working precision (the translate coefficients are large exactly where
    the restricted translates are tiny, so a float64 sum would cancel)."""
    EL, ER = _edge_cells_mp(p, q)
    return (np.array([[float(x) for x in r] for r in EL]), np.array([[float(x) for x in r] for r in ER]))


def edge_coefficients(p):
    """(A, trL, B, trR): phi^left_m = sum_j A[m,j] phi(.-trL[j])|[0,inf),
    phi^right_m = sum_j B[m,j] phi(.-trR[j])|(-inf,0], float64."""
    A, trL, B, trR = _edges_mp(p)
    return (np.array([[float(x) for x in r] for r in A]), trL,
            np.array([[float(x) for x in r] for r in B]), trR)


# ----------------------------------------------------------------------------
# Level-independent two-scale blocks at the edges ("DWT matrix W", Sec. 3.2).
# Left coordinates at level 1: index i < p is sqrt2 phi^left_i(2x), index
# i >= p is sqrt2 phi(2x - i).  Right coordinates: index r < p is
# sqrt2 phi^right_r(2x), r >= p is sqrt2 phi(2x + 1 + r).
# Boundary wavelets: the p-dimensional complement, in level-1 edge+interior
# space, of the level-0 space and of the interior wavelets psi(.-n) (n >= p on
# the left, n <= -p-1 on the right).  psi^left_m is its unit vector whose last
# level-1 coordinate is p + 2m (supp [0, p+m]), orthogonal to psi^left_0..m-1;
# sign: that last coordinate is positive.  Mirror rule on the right.
# ----------------------------------------------------------------------------
def _side_rows(p, side):
    """Level-0 rows (edge scaling fns, interior phi, interior psi) expressed
    in level-1 orthonormal side coordinates, plus the coordinate count K."""
    m = _mp()
    h = daubechies_mp(p)
    g = {k: (-1) ** (k % 2) * _h(h, p, 1 - k) for k in range(-p + 1, p + 1)}
    A, trL, B, trR = _edges_mp(p)
    K = 6 * p + 8
    W = 2 * K + 6 * p
    rows_edge, rows_int = [], []
    if side == "L":
        E, tr, gram = A, trL, gram_left_mp
        keep = lambda i: i >= -p + 1           # restricted translate survives
        coord = lambda i: i                      # interior translate -> coord
        interior_n = range(p, (K + p) // 2 + 2)
    else:
        E, tr, gram = B, trR, gram_right_mp
        keep = lambda i: i <= p - 2
        coord = lambda i: -1 - i
        interior_n = range(-p - 1, -(K + p) // 2 - 3, -1)
    for mm in range(p):
        c = {}
        for j, n in enumerate(tr):
            for k in range(-p + 1, p + 1):
                i = 2 * n + k
                if keep(i):
                    c[i] = c.get(i, 0) + E[mm][j] * h[k + p - 1]
        v = [m.mpf(0)] * W
        for mp_ in range(p):
            s = 0
            for i in tr:
                if i in c:
                    for j2, n2 in enumerate(tr):
                        s += c[i] * gram(p, i, n2) * E[mp_][j2]
            v[mp_] = s
        for i, val in c.items():
            if coord(i) >= p:
                v[coord(i)] += val
        rows_edge.append(v)
    for n in interior_n:
        for filt in ({k: h[k + p - 1] for k in range(-p + 1, p + 1)}, g):
            v = [m.mpf(0)] * W
            for k, val in filt.items():
                v[coord(2 * n + k)] = val
            rows_int.append(v)
    return rows_edge, rows_int, K, W


@lru_cache(maxsize=None, typed=True)
def _wavelets_mp(p, side):
    m = _mp()
    h = daubechies_mp(p)
    # sign of the interior wavelet's coefficient at the matching extreme:
    # g_p on the left, g_{-p+1} on the right (g_k = (-1)^k h_{1-k}).
    sgn = (-1) ** (p % 2) * h[0] if side == "L" else (-1) ** ((p + 1) % 2) * h[2 * p - 1]
    rows_edge, rows_int, K, W = _side_rows(p, side)
    rows = rows_edge + rows_int
    us = []
    for mm in range(p):
        c = p + 2 * mm
        live = [r for r in rows if any(r[b] != 0 for b in range(c + 1))]
        # null space of the constraint rows restricted to coordinates 0..c
        R = m.matrix(len(live), c + 1)
        for a, r in enumerate(live):
            for b in range(c + 1):
                R[a, b] = r[b]
        U, S, V = m.svd_r(R, full_matrices=True)
        tol = m.mpf(10) ** (-DPS // 2)
        null = [[V[i, b] for b in range(c + 1)] for i in range(V.rows)
                if i >= len(S) or abs(S[i]) < tol]
        assert len(null) == mm + 1, (p, side, mm, len(null))
        # remove the span of the earlier wavelets, keep the largest remainder
        best, bestn = None, -1
        for v in null:
            w = list(v)
            for u in us:
                cdot = sum(u[i] * w[i] for i in range(len(u)))
                w = [w[i] - cdot * (u[i] if i < len(u) else 0) for i in range(c + 1)]
            nrm = m.sqrt(sum(x * x for x in w))
            if nrm > bestn:
                best, bestn = w, nrm
        w = [x / bestn for x in best]
        if (w[c] < 0) != (sgn < 0):
            w = [-x for x in w]
        us.append(w)
    return rows_edge, us


def edge_blocks(p, side):
    """(P, Q): P[m] = level-1 side coordinates of the level-0 edge scaling
    function m, Q[m] = those of boundary wavelet m (float64, zero-padded to a
    common length).  The same blocks serve every level j -> j+1."""
    rows_edge, us = _wavelets_mp(p, side)
    L = max(max((i for i, x in enumerate(r) if x != 0), default=0) for r in rows_edge) + 1
    L = max(L, 3 * p - 1)
    P = np.array([[float(x) for x in r[:L]] for r in rows_edge])
    Q = np.zeros((p, L))
    for mm, u in enumerate(us):
        Q[mm, :len(u)] = [float(x) for x in u]
    return P, Q


# ----------------------------------------------------------------------------
# Moments and point values (used only by the oracle's own self-checks).
# ----------------------------------------------------------------------------
def phi_dyadic(p, K):
    """Point values phi(i / 2^K) for i in [(-p+1) 2^K, p 2^K], from the
    eigenvector at the integers and the cascade (Sec. 3.2, last paragraph)."""
    m = _mp()
    h = daubechies_mp(p)
    ts = list(range(-p + 1, p + 1))
    n = len(ts)
    A = m.matrix(n, n)
    for a, t in enumerate(ts):
        for b, u in enumerate(ts):
            A[a, b] = m.sqrt(2) * _h(h, p, 2 * t - u) - (1 if a == b else 0)
    rhs = m.matrix(n, 1)
    for b in range(n):
        A[n - 1, b] = 1
    rhs[n - 1] = 1
    v = m.lu_solve(A, rhs)
    cur = {t: float(v[a]) for a, t in enumerate(ts)}
    hf = np.array([float(x) for x in h])
    for lev in range(1, K + 1):
        new = {}
        for num in range((-p + 1) * 2 ** lev, p * 2 ** lev + 1):
            s = 0.0
            for k in range(-p + 1, p + 1):
                s += hf[k + p - 1] * cur.get(num - k * 2 ** (lev - 1), 0.0)
            new[num] = np.sqrt(2.0) * s
        cur = new
    return cur
