"""Dense definition of the product (oracle, test infrastructure only).

U_{n,m} = <r_m, w_n> (Sec. 1.2).  For n < N = 2^L, w_n is constant on the
cells [k/N, (k+1)/N) (Def. 3.1 reads only the first L digits of x), so
<r_m, w_n> = sum_k w_n(k/N) int_{cell k} r_m, i.e. U = H_N C with C the exact
cell integrals of the reconstruction basis.  With r_m from C_{psi,R}
(Remark 4.2), C = T W^{-1}, T the cell integrals of B_{phi,R}:

    P_N U P_M = H_N T W^{-1}          (1D, N x M)

and in 2D (Sec. 5) alpha = G xi G^T with G = H_N T applied to the Mallat
IDWT of the coefficient array.  The sampled rows are P_Omega (Sec. 1.1): y is
the entries of alpha at the sorted linear indices Omega (2D: n1 * N + n2).
"""
import numpy as np

from . import walsh, wavelets


def U1d(R, q, p, bd, J0):
    """Dense N x M section P_N U P_M in the wavelet basis C_{psi,R}."""
    N = 2 ** (R + q)
    return walsh.hadamard(N) @ wavelets.cell_matrix(R, q, p, bd) @ wavelets.idwt_matrix(R, J0, p, bd)


def U1d_scaling(R, q, p, bd):
    """Dense N x M section in the scaling basis B_{phi,R} (the matrix of
    Sec. 4, whose smallest singular value Table 1 reports)."""
    N = 2 ** (R + q)
    return walsh.hadamard(N) @ wavelets.cell_matrix(R, q, p, bd)


def G1d(R, q, p, bd):
    """G = H_N T (N x M), the 1D operator Algorithm 2 applies per dimension."""
    return U1d_scaling(R, q, p, bd)


def forward1d(x, R, q, p, bd, J0, omega=None):
    """y = P_Omega U x for x of shape (..., M)."""
    a = np.asarray(x, dtype=np.float64) @ U1d(R, q, p, bd, J0).T
    return a if omega is None else a[..., np.asarray(omega)]


def adjoint1d(y, R, q, p, bd, J0, omega=None):
    """x = U^T P_Omega^T y for y of shape (..., m)."""
    N = 2 ** (R + q)
    y = np.asarray(y, dtype=np.float64)
    if omega is None:
        a = y
    else:
        a = np.zeros(y.shape[:-1] + (N,))
        a[..., np.asarray(omega)] = y
    return a @ U1d(R, q, p, bd, J0)


def forward2d(x, R, q, p, bd, J0, omega=None, G=None):
    """y = P_Omega vec(G S G^T), S = Mallat IDWT of x (..., M, M)."""
    N = 2 ** (R + q)
    G = G1d(R, q, p, bd) if G is None else G
    S = wavelets.idwt2d(x, J0, p, bd)
    A = G @ S @ G.T
    A = A.reshape(A.shape[:-2] + (N * N,))
    return A if omega is None else A[..., np.asarray(omega)]


def adjoint2d(y, R, q, p, bd, J0, omega=None, G=None):
    """x = DWT2D(G^T A G), A = P_Omega^T y reshaped N x N."""
    N = 2 ** (R + q)
    G = G1d(R, q, p, bd) if G is None else G
    y = np.asarray(y, dtype=np.float64)
    if omega is None:
        A = y
    else:
        A = np.zeros(y.shape[:-1] + (N * N,))
        A[..., np.asarray(omega)] = y
    A = A.reshape(A.shape[:-1] + (N, N))
    return wavelets.dwt2d(G.T @ A @ G, J0, p, bd)
