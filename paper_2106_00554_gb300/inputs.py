"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method (no filters, no Walsh
functions, no transforms): it only draws numbers and index sets, so that the
CUDA path and the CPU oracle can be fed the very same inputs.

* Wavelet coefficient vectors / arrays whose magnitude decays with the level
  j of the coefficient: x = g * 2^{-alpha j}, g ~ N(0, 1) (Gaussian signs).
  The J0 scaling block counts as level J0.  2D arrays use the Mallat square
  layout: entry (i1, i2) belongs to level max(j(i1), j(i2)).
* Sampling sets Omega (sorted linear sequency indices):
  - 1D multilevel: every index below 2^8 (or N if smaller), then dyadic bands
    B_k = [2^{8+k}, 2^{9+k}) drawing round(d_k |B_k|) indices uniformly without
    replacement, d_k = min(1, c * 0.5 * 2^{-0.3 k}); c is fitted so that the
    total is exactly round(f N).
  - 2D radial: r = sqrt(n1^2 + n2^2) over sequency pairs; the disc r < N/16
    is fully sampled, annuli [2^k N/16, 2^{k+1} N/16) (clipped to the square)
    take the same density rule with exact total round(f N^2).  The linear
    index is n1 * N + n2.
"""
import numpy as np


def level_of_index(R, J0):
    lev = np.empty(2 ** R, dtype=np.int64)
    lev[:2 ** J0] = J0
    for j in range(J0, R):
        lev[2 ** j:2 ** (j + 1)] = j
    return lev


def coeffs_1d(rng, R, J0, alpha, batch=None):
    lev = level_of_index(R, J0)
    shape = (2 ** R,) if batch is None else (batch, 2 ** R)
    return rng.standard_normal(shape) * 2.0 ** (-alpha * lev)


def coeffs_2d(rng, R, J0, alpha, batch=None):
    lev = level_of_index(R, J0)
    L = np.maximum(lev[:, None], lev[None, :])
    M = 2 ** R
    shape = (M, M) if batch is None else (batch, M, M)
    return rng.standard_normal(shape) * 2.0 ** (-alpha * L)


def _fit_counts(sizes, target, base_full):
    """Counts per band: full bands first, then d_k = min(1, c 0.5 2^-0.3k)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    rest = target - base_full
    if rest <= 0 or len(sizes) == 0:
        return np.zeros(len(sizes), dtype=np.int64)
    if rest >= sizes.sum():
        return sizes.copy()
    k = np.arange(len(sizes))

    def total(c):
        return float(np.sum(np.minimum(1.0, c * 0.5 * 2.0 ** (-0.3 * k)) * sizes))

    lo, hi = 0.0, 1.0
    while total(hi) < rest:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < rest:
            lo = mid
        else:
            hi = mid
    real = np.minimum(1.0, hi * 0.5 * 2.0 ** (-0.3 * k)) * sizes
    cnt = np.floor(real).astype(np.int64)
    frac = real - cnt
    for i in np.argsort(-frac):
        if cnt.sum() >= rest:
            break
        if cnt[i] < sizes[i]:
            cnt[i] += 1
    i = len(sizes) - 1
    while cnt.sum() > rest:
        if cnt[i] > 0:
            cnt[i] -= 1
        i = (i - 1) % len(sizes)
    return cnt


def mask_1d(rng, N, frac):
    """Sorted sequency indices, multilevel 1D pattern, exact size round(f N)."""
    target = int(round(frac * N))
    full = min(256, N)
    if target <= full:
        return np.arange(target, dtype=np.int64)
    bands = []
    lo = full
    while lo < N:
        bands.append((lo, min(2 * lo, N)))
        lo *= 2
    cnt = _fit_counts([b - a for a, b in bands], target, full)
    parts = [np.arange(full, dtype=np.int64)]
    for (a, b), c in zip(bands, cnt):
        parts.append(np.sort(rng.choice(np.arange(a, b, dtype=np.int64), size=int(c), replace=False)))
    return np.concatenate(parts)


def mask_2d(rng, N, frac):
    """Sorted linear indices n1 * N + n2, radial multilevel 2D pattern."""
    target = int(round(frac * N * N))
    n = np.arange(N, dtype=np.float64)
    r = np.sqrt(n[:, None] ** 2 + n[None, :] ** 2).ravel()
    r0 = N / 16.0
    disc = np.flatnonzero(r < r0)
    if target <= disc.size:
        order = np.argsort(r, kind="stable")[:target]
        return np.sort(order).astype(np.int64)
    bands = []
    lo = r0
    while lo <= r.max():
        idx = np.flatnonzero((r >= lo) & (r < 2 * lo))
        bands.append(idx)
        lo *= 2
    cnt = _fit_counts([b.size for b in bands], target, disc.size)
    parts = [disc]
    for b, c in zip(bands, cnt):
        if c:
            parts.append(rng.choice(b, size=int(c), replace=False))
    return np.sort(np.concatenate(parts)).astype(np.int64)


def gaussian(rng, shape):
    return rng.standard_normal(shape)


def sparse_coeffs_2d(rng, R, J0, alpha, density):
    """Level-decaying 2D coefficients with a uniform random support."""
    x = coeffs_2d(rng, R, J0, alpha)
    keep = rng.random(x.shape) < density
    return x * keep
