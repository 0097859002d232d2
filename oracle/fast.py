"""Algorithm 1 and Algorithm 2 as the paper states them (oracle, test
infrastructure only).  This is the plain O(N log N) CPU version: the interior
by sum_{l=-p+1}^{p-1} D_l H_l (Sec. 4.1) and its adjoint sum_l B_l D_l
(Sec. 4.2), the edges by Prop. 4.4 with pointwise Walsh values, one
zero-padded FWHT per l.  It is slower than one FWHT (2p-1 of them), which is
the point: it follows the paper's own steps so that the dense definition and
the paper's derivation check each other.

Readings taken where the paper is garbled: the right VMP edge formula of
Prop. 4.4 carries 2^{j/2}, read as 2^{-j/2} like every other term; the
adjoint sum runs to N-1 (printed N_1).
"""
import numpy as np

from . import tables, walsh, wavelets


# ----------------------------------------------------------------------------
# FWHT (Sec. 3.1): the N sums sum_k w_n(k/N) x_k, n = 0..N-1.
# ----------------------------------------------------------------------------
def _natural_fwht(v):
    """Textbook radix-2 Walsh-Hadamard butterflies along the last axis
    (natural / Hadamard order: out[r] = sum_k (-1)^{popcount(r & k)} v[k])."""
    v = np.array(v, dtype=np.float64, copy=True)
    N = v.shape[-1]
    h = 1
    while h < N:
        v = v.reshape(v.shape[:-1] + (N // (2 * h), 2, h))
        a = v[..., 0, :].copy()
        b = v[..., 1, :].copy()
        v[..., 0, :] = a + b
        v[..., 1, :] = a - b
        v = v.reshape(v.shape[:-3] + (N,))
        h *= 2
    return v


def sequency_row(N):
    """r(n) with w_n(k/N) = (-1)^{popcount(r(n) & k)}: Def. 3.1 gives the
    exponent sum_j (n^(j) + n^(j+1)) x^(j) with x^(j) = bit L-j of k, so bit
    L-j of r(n) is n^(j) xor n^(j+1)."""
    L = int(N).bit_length() - 1
    n = np.arange(N, dtype=np.int64)
    r = np.zeros(N, dtype=np.int64)
    for j in range(1, L + 1):
        d = ((n >> (j - 1)) & 1) ^ ((n >> j) & 1)
        r |= d << (L - j)
    return r


def fwht(v):
    """Sequency-ordered FWHT along the last axis: out[n] = sum_k w_n(k/N) v[k]."""
    N = v.shape[-1]
    return _natural_fwht(v)[..., sequency_row(N)]


# ----------------------------------------------------------------------------
# Taps (Sec. 4.1): W phi_{0,-l}|[0,1)(s) for s < 2^q, from the cell integrals.
# ----------------------------------------------------------------------------
def _walsh_of_cells(cells, q):
    """sum_c w_s(c/2^q) cells[c] for s < 2^q."""
    Q = 2 ** q
    s = np.arange(Q)[:, None]
    c = np.arange(Q)[None, :]
    return walsh.walsh(s, c, q) @ np.asarray(cells, dtype=np.float64)


def taps(p, q):
    """dict l -> array over s of W phi_{0,-l}|[0,1)(s), l = -p+1..p-1."""
    I = tables.cell_integrals(p, q)
    Q = 2 ** q
    return {l: _walsh_of_cells([I.get(l * Q + c, 0.0) for c in range(Q)], q)
            for l in range(-p + 1, p)}


def _edge_walsh(p, q):
    """W phi^left_m(.+l)|[0,1)(s) and W phi^right_r(.+l)|[0,1)(s)."""
    EL, ER = tables.edge_cells(p, q)
    Q = 2 ** q
    left, right = {}, {}
    for m in range(p):
        for l in range(0, p + m):
            left[(m, l)] = _walsh_of_cells(EL[m, l * Q:(l + 1) * Q], q)
        for l in range(-(m + p), 0):
            # cells [l + c/Q, l + (c+1)/Q) of phi^right_m: ER index -(l Q + c) - 1
            right[(m, l)] = _walsh_of_cells([ER[m, -(l * Q + c) - 1] for c in range(Q)], q)
    return left, right


def edge_inner_products(R, q, p, bd):
    """E[n, c] = <phi^rep_{R,m}, w_n> for the 2p edge columns (Prop. 4.4);
    columns 0..p-1 are m = 0..p-1, columns p..2p-1 are m = M-p..M-1."""
    M, N = 2 ** R, 2 ** (R + q)
    n = np.arange(N)
    s = n >> R                      # floor(n / 2^j)
    sc = 2.0 ** (-R / 2)
    E = np.zeros((N, 2 * p))
    if bd == wavelets.PER:
        tp = taps(p, q)
        for m in range(p):
            for l in range(-p + 1, -m):
                E[:, m] += sc * walsh.walsh(n, M + m + l, R) * tp[l][s]
            for l in range(-m, p):
                E[:, m] += sc * walsh.walsh(n, m + l, R) * tp[l][s]
        for c, m in enumerate(range(M - p, M)):
            for l in range(-p + 1, M - m):
                E[:, p + c] += sc * walsh.walsh(n, l + m, R) * tp[l][s]
            for l in range(M - m, p):
                E[:, p + c] += sc * walsh.walsh(n, l + m - M, R) * tp[l][s]
        return E
    left, right = _edge_walsh(p, q)
    for m in range(p):
        for l in range(0, p + m):
            E[:, m] += sc * walsh.walsh(n, l, R) * left[(m, l)][s]
    for c, m in enumerate(range(M - p, M)):
        r = M - 1 - m
        for l in range(m - M - p + 1, 0):
            E[:, p + c] += sc * walsh.walsh(n, l + M, R) * right[(r, l)][s]
    return E


# ----------------------------------------------------------------------------
# Algorithm 1 on the scaling basis B_{phi,j}.
# ----------------------------------------------------------------------------
def alg1_forward(xi, R, q, p, bd):
    """alpha = P_N U P_M xi for xi (..., M) in the scaling basis."""
    M, N = 2 ** R, 2 ** (R + q)
    xi = np.asarray(xi, dtype=np.float64)
    n = np.arange(N)
    s = n >> R
    tp = taps(p, q)
    E = edge_inner_products(R, q, p, bd)
    beta = xi[..., :p] @ E[:, :p].T + xi[..., M - p:] @ E[:, p:].T
    mids = np.arange(p, M - p)
    for l in range(-p + 1, p):
        z = np.zeros(xi.shape[:-1] + (N,))
        z[..., 2 ** q * (l + mids)] = xi[..., mids]
        beta = beta + 2.0 ** (-R / 2) * tp[l][s] * fwht(z)       # D_l H_l xi
    return beta


def alg1_adjoint(alpha, R, q, p, bd):
    """xi = P_M U^* P_N alpha for alpha (..., N)."""
    M, N = 2 ** R, 2 ** (R + q)
    alpha = np.asarray(alpha, dtype=np.float64)
    n = np.arange(N)
    s = n >> R
    tp = taps(p, q)
    E = edge_inner_products(R, q, p, bd)
    xi = np.zeros(alpha.shape[:-1] + (M,))
    xi[..., :p] = alpha @ E[:, :p]
    xi[..., M - p:] = alpha @ E[:, p:]
    mids = np.arange(p, M - p)
    acc = np.zeros(alpha.shape[:-1] + (M - 2 * p,))
    for l in range(-p + 1, p):
        t = fwht(2.0 ** (-R / 2) * tp[l][s] * alpha)             # B_l D_l alpha
        acc += t[..., 2 ** q * (l + mids)]
    xi[..., p:M - p] = acc
    return xi


# ----------------------------------------------------------------------------
# IDWT / DWT by the cascade (Remark 4.2: O(M)), level by level with filters.
# ----------------------------------------------------------------------------
def _syn_level(lo, hi, p, bd):
    n0 = lo.shape[-1]
    n1 = 2 * n0
    h = tables.daubechies(p)
    g = tables.wavelet_filter(p)
    out = np.zeros(lo.shape[:-1] + (n1,))
    if bd == wavelets.PER:
        for k in range(-p + 1, p + 1):
            idx = (2 * np.arange(n0) + k) % n1
            np.add.at(out, (..., idx), h[k + p - 1] * lo + g[k + p - 1] * hi)
        return out
    PL, QL = tables.edge_blocks(p, "L")
    PR, QR = tables.edge_blocks(p, "R")
    ms = np.arange(p, n0 - p)
    for k in range(-p + 1, p + 1):
        out[..., 2 * ms + k] += h[k + p - 1] * lo[..., ms] + g[k + p - 1] * hi[..., ms]
    L = PL.shape[1]
    out[..., :L] += lo[..., :p] @ PL + hi[..., :p] @ QL
    L = PR.shape[1]
    out[..., n1 - L:] += (lo[..., n0 - 1 - np.arange(p)] @ PR + hi[..., n0 - 1 - np.arange(p)] @ QR)[..., ::-1]
    return out


def _ana_level(s, p, bd):
    n1 = s.shape[-1]
    n0 = n1 // 2
    h = tables.daubechies(p)
    g = tables.wavelet_filter(p)
    lo = np.zeros(s.shape[:-1] + (n0,))
    hi = np.zeros(s.shape[:-1] + (n0,))
    if bd == wavelets.PER:
        for k in range(-p + 1, p + 1):
            idx = (2 * np.arange(n0) + k) % n1
            lo += h[k + p - 1] * s[..., idx]
            hi += g[k + p - 1] * s[..., idx]
        return lo, hi
    PL, QL = tables.edge_blocks(p, "L")
    PR, QR = tables.edge_blocks(p, "R")
    ms = np.arange(p, n0 - p)
    for k in range(-p + 1, p + 1):
        lo[..., ms] += h[k + p - 1] * s[..., 2 * ms + k]
        hi[..., ms] += g[k + p - 1] * s[..., 2 * ms + k]
    L = PL.shape[1]
    lo[..., :p] = s[..., :L] @ PL.T
    hi[..., :p] = s[..., :L] @ QL.T
    L = PR.shape[1]
    rev = s[..., n1 - L:][..., ::-1]
    lo[..., n0 - 1 - np.arange(p)] = rev @ PR.T
    hi[..., n0 - 1 - np.arange(p)] = rev @ QR.T
    return lo, hi


def idwt(x, J0, p, bd):
    x = np.asarray(x, dtype=np.float64)
    R = int(x.shape[-1]).bit_length() - 1
    s = x[..., :2 ** J0]
    for j in range(J0, R):
        s = _syn_level(s, x[..., 2 ** j:2 ** (j + 1)], p, bd)
    return s


def dwt(s, J0, p, bd):
    s = np.asarray(s, dtype=np.float64)
    R = int(s.shape[-1]).bit_length() - 1
    out = np.zeros_like(s)
    for j in range(R - 1, J0 - 1, -1):
        s, d = _ana_level(s, p, bd)
        out[..., 2 ** j:2 ** (j + 1)] = d
    out[..., :2 ** J0] = s
    return out


# ----------------------------------------------------------------------------
# Full products.
# ----------------------------------------------------------------------------
def forward1d(x, R, q, p, bd, J0, omega=None):
    a = alg1_forward(idwt(x, J0, p, bd), R, q, p, bd)
    return a if omega is None else a[..., np.asarray(omega)]


def adjoint1d(y, R, q, p, bd, J0, omega=None):
    N = 2 ** (R + q)
    y = np.asarray(y, dtype=np.float64)
    if omega is None:
        a = y
    else:
        a = np.zeros(y.shape[:-1] + (N,))
        a[..., np.asarray(omega)] = y
    return dwt(alg1_adjoint(a, R, q, p, bd), J0, p, bd)


def idwt2d(X, J0, p, bd):
    X = np.array(X, dtype=np.float64, copy=True)
    R = int(X.shape[-1]).bit_length() - 1
    for j in range(J0, R):
        n0, n1 = 2 ** j, 2 ** (j + 1)
        B = X[..., :n1, :n1]
        B = _syn_level(B[..., :, :n0], B[..., :, n0:], p, bd)                    # rows
        Bt = np.swapaxes(B, -1, -2)
        B = np.swapaxes(_syn_level(Bt[..., :, :n0], Bt[..., :, n0:], p, bd), -1, -2)  # columns
        X[..., :n1, :n1] = B
    return X


def dwt2d(S, J0, p, bd):
    X = np.array(S, dtype=np.float64, copy=True)
    R = int(X.shape[-1]).bit_length() - 1
    for j in range(R - 1, J0 - 1, -1):
        n0, n1 = 2 ** j, 2 ** (j + 1)
        B = X[..., :n1, :n1]
        Bt = np.swapaxes(B, -1, -2)
        lo, hi = _ana_level(Bt, p, bd)
        B = np.swapaxes(np.concatenate([lo, hi], -1), -1, -2)
        lo, hi = _ana_level(B, p, bd)
        X[..., :n1, :n1] = np.concatenate([lo, hi], -1)
    return X


def forward2d(x, R, q, p, bd, J0, omega=None):
    """Algorithm 2: alpha = G xi G^*, xi the Mallat IDWT of x."""
    N = 2 ** (R + q)
    xi = idwt2d(x, J0, p, bd)
    t = alg1_forward(xi, R, q, p, bd)                                  # rows: xi G^T
    a = np.swapaxes(alg1_forward(np.swapaxes(t, -1, -2), R, q, p, bd), -1, -2)
    a = a.reshape(a.shape[:-2] + (N * N,))
    return a if omega is None else a[..., np.asarray(omega)]


def adjoint2d(y, R, q, p, bd, J0, omega=None):
    """Algorithm 2 adjoint: xi = G^* alpha G, then the Mallat DWT."""
    N = 2 ** (R + q)
    y = np.asarray(y, dtype=np.float64)
    if omega is None:
        a = y
    else:
        a = np.zeros(y.shape[:-1] + (N * N,))
        a[..., np.asarray(omega)] = y
    a = a.reshape(a.shape[:-1] + (N, N))
    t = alg1_adjoint(a, R, q, p, bd)                                   # rows
    xi = np.swapaxes(alg1_adjoint(np.swapaxes(t, -1, -2), R, q, p, bd), -1, -2)
    return dwt2d(xi, J0, p, bd)
