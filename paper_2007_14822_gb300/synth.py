"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the method: it only draws seeded random
numbers and lays out synthetic sector sizes. Both the GPU library's callers
and the CPU oracle consume exactly these arrays, so neither side duplicates
a random-number generator.

* ``gaussian``        an N(0,1) array of a given shape from one seed.
* ``block_gaussian``  N(0,1) entries for one block of a block-sparse tensor,
                      keyed by (seed, tensor tag, block sector tuple), so the
                      values do not depend on the order blocks are visited.
* ``gaussian_sectors`` sector sizes that follow a discretised Gaussian
                      profile, clipped to [1, maxdim] and rescaled with the
                      largest-remainder rule so that they sum to ``m``.
* ``product_spinors`` one N(0,1) vector per site (a random product state;
                      each consumer normalises it itself).
"""
from __future__ import annotations

import zlib

import numpy as np


def _tag(tag):
    return zlib.crc32(str(tag).encode()) & 0x7FFFFFFF


def gaussian(seed, shape):
    return np.random.default_rng(int(seed)).standard_normal(shape)


def block_gaussian(seed, tag, key, shape):
    ss = [int(seed), _tag(tag)] + [int(k) for k in key]
    return np.random.default_rng(ss).standard_normal(shape)


def _fit_profile(m, sqdist, maxdim):
    """Sizes maxdim * exp(-sqdist / 2 w^2), clipped to [1, maxdim], summing to m.

    The width w is found by bisection so the clipped profile sums to about
    ``m``; the integer sizes then follow the largest-remainder rule, each
    kept within [1, maxdim].
    """
    n = sqdist.size
    if not (n <= m <= n * maxdim):
        raise ValueError("m out of range for the number of sectors and maxdim")

    def prof(w):
        return np.clip(maxdim * np.exp(-sqdist / (2.0 * w * w)), 1.0, maxdim)

    lo, hi = 1e-6, 1e6
    for _ in range(200):
        w = np.sqrt(lo * hi)
        if prof(w).sum() < m:
            lo = w
        else:
            hi = w
    want = prof(np.sqrt(lo * hi))
    base = np.clip(np.floor(want).astype(np.int64), 1, maxdim)
    rem = want - base
    short = int(m - base.sum())
    order = np.argsort(-rem, kind="stable")
    i = 0
    while short != 0:
        k = order[i % n] if short > 0 else order[::-1][i % n]
        if short > 0 and base[k] < maxdim:
            base[k] += 1
            short -= 1
        elif short < 0 and base[k] > 1:
            base[k] -= 1
            short += 1
        i += 1
    return base


def gaussian_sectors(m, nsect, maxdim):
    """Sizes of ``nsect`` sectors summing to ``m``: a discretised Gaussian
    profile centred on the middle sector, peak ``maxdim``, tails clipped at 1.
    """
    x = np.arange(nsect) - (nsect - 1) / 2.0
    return [int(v) for v in _fit_profile(m, x * x, maxdim)]


def gaussian_sectors_2d(m, shape, maxdim):
    """Same recipe on a 2-D grid of sectors (e.g. (N, 2Sz) charges)."""
    n0, n1 = shape
    x0 = np.arange(n0) - (n0 - 1) / 2.0
    x1 = np.arange(n1) - (n1 - 1) / 2.0
    sq = (x0[:, None] ** 2 + x1[None, :] ** 2).ravel()
    return _fit_profile(m, sq, maxdim).reshape(shape)


def product_spinors(seed, N, d):
    g = gaussian(seed, (N, d))
    return [g[j] for j in range(N)]
