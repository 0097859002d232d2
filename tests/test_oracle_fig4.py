"""The periodic-versus-boundary comparison of Sec. 3.2 (Wavelets), Fig. 4:
generalised sampling of f(t) = cos(2 pi t) and g(t) = cos(2 pi t) + t from
their first N = 32 Walsh samples in M = 16 DB4 basis functions, with periodic
and with vanishing-moment-preserving (VMP) boundary extensions.  The figure
shows the four reconstructions; its caption states what they show, and that
is what these pins check on the oracle (the GPU solve of the same problems is
in tests/test_solvers_gpu.py):
- the periodic basis reconstructs the periodic f accurately;
- for the non-periodic g it leaves artefacts at the boundaries;
- the VMP basis reconstructs g without them.
A closed-form pin joins the last two: g - f = t is a polynomial of degree 1,
which lies in the VMP reconstruction space (p = 4 vanishing moments, Sec.
3.2), and a least-squares fit reproduces exactly whatever lies in its space,
so with VMP boundaries the reconstruction errors of g and of f are the same
function; t is not in the periodic space, so with periodic boundaries they
differ.

Errors: the fit r = sum_m z_m phi_{R,m} (orthonormal scaling basis of V_R,
R = 4) against f through the cell averages of both on 4096 cells (exact
integrals of f; the oracle's cell integrals of phi_{R,m}), split into the
outer 1/16 of [0, 1] at each end ("boundary") and the rest ("interior"); and
the relative L2 error ||f - r|| / ||f|| from <f, phi_m> by Parseval on the
first 2^12 Walsh functions."""
import numpy as np
import pytest

from oracle import dense, walsh, wavelets as W

scipy_integrate = pytest.importorskip("scipy.integrate")

R, Q, P, NS, NF = 4, 1, 4, 32, 4096
FUNCS = {"f": lambda t: np.cos(2.0 * np.pi * t), "g": lambda t: np.cos(2.0 * np.pi * t) + t}


def cells(name, n):
    """exact integrals over the cells [k/n, (k+1)/n) (closed forms)"""
    a = np.arange(n + 1) / n
    out = np.diff(np.sin(2.0 * np.pi * a)) / (2.0 * np.pi)
    if name in ("g", "t"):
        lin = np.diff(a * a) / 2.0
        out = lin if name == "t" else out + lin
    return out


def samples(name):
    """<fn, w_k>, k < 32 (Def. 3.1: w_k is constant on cells of width 1/32)"""
    return walsh.hadamard(NS) @ cells(name, NS)


_MATS = {}


def mats(bd):
    """(A = P_N U P_M in the scaling basis of V_R, cell integrals of phi_{R,m}
    on 4096 cells)"""
    if bd not in _MATS:
        _MATS[bd] = (dense.U1d_scaling(R, Q, P, bd), W.cell_matrix(R, 12 - R, P, bd))
    return _MATS[bd]


def fit(name, bd):
    """least-squares coefficients in the scaling basis of V_R (Sec. 1.2)"""
    return np.linalg.lstsq(mats(bd)[0], samples(name), rcond=None)[0]


def errors(name, z, bd):
    """(relative L2 error, cell-average error on 4096 cells, boundary rms,
    interior rms).  <fn, phi_m> by Parseval on the first 4096 Walsh
    functions, whose span is the piecewise constants on 4096 cells:
    4096 sum_j cells_fn[j] cells_phi_m[j]."""
    C = mats(bd)[1]
    cf = cells(name, NF)
    d = (C @ z - cf) * NF
    b = NF // 16
    eb = np.sqrt(np.mean(np.r_[d[:b], d[-b:]] ** 2))
    ei = np.sqrt(np.mean(d[b:-b] ** 2))
    fn = FUNCS[name]
    n2 = scipy_integrate.quad(lambda t: fn(t) ** 2, 0.0, 1.0)[0]
    fphi = NF * (cf @ C)
    rel = np.sqrt(max(n2 - 2.0 * fphi @ z + z @ z, 0.0) / n2)
    return rel, d, eb, ei


@pytest.fixture(scope="module")
def table():
    out = {}
    for bd in (W.PER, W.VMP):
        for name in FUNCS:
            out[bd, name] = errors(name, fit(name, bd), bd)
    return out


def test_periodic_basis_reconstructs_the_periodic_function(table):
    rel, _, eb, ei = table[W.PER, "f"]
    assert rel < 2e-3, rel
    assert eb < 2 * ei, (eb, ei)          # no boundary artefact


def test_periodic_basis_leaves_boundary_artefacts_on_the_nonperiodic_function(table):
    rel, _, eb, ei = table[W.PER, "g"]
    assert rel > 20 * table[W.VMP, "g"][0], (rel, table[W.VMP, "g"][0])
    assert eb > 5 * ei, (eb, ei)          # the error sits at the two ends


def test_vmp_basis_reconstructs_the_nonperiodic_function(table):
    rel, _, eb, ei = table[W.VMP, "g"]
    assert rel < 5e-3, rel
    assert eb < 3 * ei, (eb, ei)


def test_vmp_space_holds_the_linear_part(table):
    """g - f = t lies in the VMP space: the two fits differ by exactly its
    coefficients and the two errors are the same function (to rounding); in
    the periodic space they are not."""
    d_vmp = table[W.VMP, "g"][1] - table[W.VMP, "f"][1]
    d_per = table[W.PER, "g"][1] - table[W.PER, "f"][1]
    assert np.max(np.abs(d_vmp)) < 1e-10, np.max(np.abs(d_vmp))
    assert np.max(np.abs(d_per)) > 1e-2, np.max(np.abs(d_per))
    # and t itself is reproduced from its 32 Walsh samples with VMP boundaries
    z = fit("t", W.VMP)
    assert np.max(np.abs(mats(W.VMP)[1] @ z - cells("t", NF))) * NF < 1e-10


def test_closed_form_cells():
    """the closed-form cell integrals against quadrature"""
    quad = scipy_integrate.quad
    for name, fn in FUNCS.items():
        want = np.array([quad(fn, k / 64, (k + 1) / 64)[0] for k in range(64)])
        assert np.max(np.abs(cells(name, 64) - want)) < 1e-14
