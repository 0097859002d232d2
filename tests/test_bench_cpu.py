"""Host-side pieces of bench.py: the all-core oracle pair that the reference
arm and cpu_baseline time is the oracle's own Algorithm 2 (same result as
oracle.fast.forward2d / adjoint2d), in one process and over a spawned pool."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import fast, wavelets as W  # noqa: E402
from paper_2106_00554_gb300 import inputs  # noqa: E402


def test_pooled_oracle_pair_is_algorithm_2():
    R, q, p = 6, 1, 4
    N = 2 ** (R + q)
    rng = np.random.default_rng(5)
    omega = inputs.mask_2d(rng, N, 0.3)
    J0 = W.default_J0(p)
    x = inputs.coeffs_2d(rng, R, J0, 1.5)
    y = rng.standard_normal(omega.size)
    want_y = fast.forward2d(x, R, q, p, W.VMP, J0, omega)
    want_x = fast.adjoint2d(y, R, q, p, W.VMP, J0, omega)
    got_y, got_x = bench.oracle_pair_2d(None, 1, x, y, R, q, p, J0, omega)
    np.testing.assert_allclose(got_y, want_y, rtol=0, atol=1e-13 * np.abs(want_y).max())
    np.testing.assert_allclose(got_x, want_x, rtol=0, atol=1e-13 * np.abs(want_x).max())
    pool = bench._spawn_pool(2)
    try:
        py, px = bench.oracle_pair_2d(pool, 2, x, y, R, q, p, J0, omega)
    finally:
        pool.close()
        pool.join()
    np.testing.assert_array_equal(py, got_y)
    np.testing.assert_array_equal(px, got_x)


def test_host_cpu_reports_cores_and_model():
    cores, model = bench.host_cpu()
    assert cores >= 1 and isinstance(model, str) and model
