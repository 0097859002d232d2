"""Band-by-band GPU parity: the relative L2 error of every Mallat subband of
the adjoint's output and of every dyadic sequency band of the forward's output,
not only of the whole vector.

A whole-vector relative error can hide an error confined to a band that holds
little of the energy: with level-decaying coefficients (alpha = 1.5) the finest
2D detail level carries about 2^{-9} of the amplitude at the benchmark size,
and the forward output's energy sits at low sequency.  So:

* with inputs whose energy is spread over every band (x ~ N(0,1) without
  decay; y ~ N(0,1)) each band must meet the precision's bar on its own;
* with the workloads' own level-decaying inputs each band must meet the bar
  against max(its own norm, the norm it would have if the vector's energy
  were spread evenly over the elements): an error of 1e-5 of the vector's RMS
  per element fails in any band, however small that band's share.

Bands.  Adjoint output x (2D): the J0 scaling block, then the three detail
blocks of each level j = J0 .. R-1 (Mallat layout, Sec. 5).  1D: the J0
scaling block and each detail level.  Forward output y: the samples whose
sequency index n (1D) or max(n1, n2) (2D, linear index n1 N + n2) lies in
[2^(k-1), 2^k), k = 0 .. log2 N (band 0 = {0}).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, fast, wavelets as W
from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, F64, VMP, Plan, build, inputs

TOL = {F64: 1e-12, F32: 1e-5, F32_SPLIT_BF16: 1e-5}


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _dev(a, prec):
    dt = torch.float64 if prec == F64 else torch.float32
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _fwd(plan, x, prec):
    y = plan.forward(_dev(x, prec), precision=prec)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


def _adj(plan, y, prec):
    x = plan.adjoint(_dev(y, prec), precision=prec)
    torch.cuda.synchronize()
    return x.double().cpu().numpy()


def subbands_2d(R, J0):
    """(name, row slice, column slice) of every Mallat subband."""
    out = [("LL%d" % J0, slice(0, 2 ** J0), slice(0, 2 ** J0))]
    for j in range(J0, R):
        lo, hi = slice(0, 2 ** j), slice(2 ** j, 2 ** (j + 1))
        out += [("HL%d" % j, lo, hi), ("LH%d" % j, hi, lo), ("HH%d" % j, hi, hi)]
    return out


def levels_1d(R, J0):
    out = [("L%d" % J0, slice(0, 2 ** J0))]
    out += [("D%d" % j, slice(2 ** j, 2 ** (j + 1))) for j in range(J0, R)]
    return out


def sequency_bands(omega, N, d):
    """Band index of every sample: ceil(log2(s + 1)), s = n (1D) or
    max(n1, n2) (2D)."""
    omega = np.asarray(omega, dtype=np.int64)
    s = omega if d == 1 else np.maximum(omega // N, omega % N)
    band = np.zeros(s.shape, dtype=np.int64)
    nz = s > 0
    band[nz] = np.floor(np.log2(s[nz])).astype(np.int64) + 1
    return band


def check_bands(got, want, groups, tol, floor_rms):
    """groups: list of (name, index) into the flattened arrays.  Each group's
    error norm must be <= tol * max(||want_g||, floor_rms * sqrt(|g|)), with
    floor_rms = 0 for the strict check."""
    got = np.asarray(got, dtype=np.float64).ravel()
    want = np.asarray(want, dtype=np.float64).ravel()
    worst = []
    for name, idx in groups:
        g, w = got[idx], want[idx]
        if w.size == 0:
            continue
        ref = max(np.linalg.norm(w), floor_rms * np.sqrt(w.size))
        err = np.linalg.norm(g - w) / (ref if ref > 0 else 1.0)
        worst.append((err, name))
        assert err <= tol, (name, err, tol)
    return max(worst)


def x_groups_2d(R, J0):
    M = 2 ** R
    flat = np.arange(M * M).reshape(M, M)
    return [(n, flat[r, c].ravel()) for n, r, c in subbands_2d(R, J0)]


def y_groups(omega, N, d):
    b = sequency_bands(omega, N, d)
    return [("band%d" % k, np.nonzero(b == k)[0]) for k in range(int(b.max()) + 1)]


def _rms(a):
    a = np.asarray(a, dtype=np.float64)
    return np.linalg.norm(a) / np.sqrt(a.size)


def _run_2d(R, q, p, frac, seed, prec, alpha):
    rng = np.random.default_rng(seed)
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, frac)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    J0 = plan.J0
    G = dense.G1d(R, q, p, VMP)
    x_flat = rng.standard_normal((2 ** R, 2 ** R))
    x_dec = inputs.coeffs_2d(rng, R, J0, alpha)
    y = rng.standard_normal(omega.size)
    tol = TOL[prec]
    # adjoint: y ~ N(0,1) spreads energy over every subband
    want_x = dense.adjoint2d(y, R, q, p, VMP, J0, omega, G=G)
    check_bands(_adj(plan, y, prec), want_x, x_groups_2d(R, J0), tol, 0.0)
    # forward, flat coefficients: every sequency band on its own
    yg = y_groups(omega, N, 2)
    want = dense.forward2d(x_flat, R, q, p, VMP, J0, omega, G=G)
    check_bands(_fwd(plan, x_flat, prec), want, yg, tol, 0.0)
    # forward, the workload's level-decaying coefficients
    want = dense.forward2d(x_dec, R, q, p, VMP, J0, omega, G=G)
    check_bands(_fwd(plan, x_dec, prec), want, yg, tol, _rms(want))
    # adjoint of the forward's samples: level-decaying x comes back band by band
    want_x = dense.adjoint2d(want, R, q, p, VMP, J0, omega, G=G)
    check_bands(_adj(plan, want, prec), want_x, x_groups_2d(R, J0), tol, _rms(want_x))
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [F32, F32_SPLIT_BF16])
def test_config5_bands(built, prec):
    """The benchmark workload (p = 8, M = 2048^2, q = 1, 12% radial mask,
    seed 4), band by band."""
    _run_2d(11, 1, 8, 0.12, 4, prec, 1.5)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [F64, F32, F32_SPLIT_BF16])
def test_config3_bands(built, prec):
    """p = 4, M = 256^2, q = 1, 25% radial mask, seed 2, band by band."""
    _run_2d(8, 1, 4, 0.25, 2, prec, 1.5)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [F32, F64])
def test_config2_bands(built, prec):
    """1D, p = 4, M = 2^16, q = 2 (N = 2^18), 15% multilevel mask, seed 1:
    two instances of the batch against Algorithm 1, by detail level and by
    dyadic sequency band."""
    rng = np.random.default_rng(1)
    R, q, p = 16, 2, 4
    N = 2 ** (R + q)
    omega = inputs.mask_1d(rng, N, 0.15)
    plan = Plan(1, R, q, p, VMP, omega=omega, max_batch=2)
    J0 = plan.J0
    x_dec = inputs.coeffs_1d(rng, R, J0, 1.5, batch=2)
    x_flat = rng.standard_normal((2, 2 ** R))
    y = rng.standard_normal((2, omega.size))
    tol = TOL[prec]
    xg = [(n, np.arange(2 ** R)[s]) for n, s in levels_1d(R, J0)]
    yg = y_groups(omega, N, 1)
    got_x = _adj(plan, y, prec)
    got_f = _fwd(plan, x_flat, prec)
    got_d = _fwd(plan, x_dec, prec)
    for b in range(2):
        check_bands(got_x[b], fast.adjoint1d(y[b], R, q, p, VMP, J0, omega), xg, tol, 0.0)
        check_bands(got_f[b], fast.forward1d(x_flat[b], R, q, p, VMP, J0, omega), yg, tol, 0.0)
        want = fast.forward1d(x_dec[b], R, q, p, VMP, J0, omega)
        check_bands(got_d[b], want, yg, tol, _rms(want))
    plan.close()


def test_band_check_catches_an_error_confined_to_one_band():
    """The band check itself (host only): an error of 1.5e-5 of the vector's
    RMS per element in the finest diagonal subband, which the whole-vector
    relative error (7.5e-6 here) lets through, fails it."""
    rng = np.random.default_rng(0)
    R, J0 = 8, 4
    want = inputs.coeffs_2d(rng, R, J0, 1.5)
    got = want.copy()
    rms = _rms(want)
    got[128:, 128:] += 1.5e-5 * rms * rng.standard_normal((128, 128))
    whole = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert whole < 1e-5
    with pytest.raises(AssertionError):
        check_bands(got, want, x_groups_2d(R, J0), 1e-5, rms)
