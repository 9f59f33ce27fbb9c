"""The seeded input recipe: sector-size profiles, per-block seeding and the
QN links of the block-sparse H_eff workloads (host only, no GPU)."""
import numpy as np
import pytest

import bench
from paper_2007_14822_gb300 import synth


@pytest.mark.parametrize("m,nsect,maxd", [(1024, 40, 128), (2048, 41, 256), (300, 15, 60), (64, 9, 16),
                                          (12, 5, 4)])
def test_gaussian_sectors_sum_clip_and_shape(m, nsect, maxd):
    dims = synth.gaussian_sectors(m, nsect, maxd)
    assert len(dims) == nsect and sum(dims) == m
    assert min(dims) >= 1 and max(dims) <= maxd
    # one peak in the middle, falling off towards both ends (up to the
    # largest-remainder rounding of one unit)
    c = (nsect - 1) // 2
    assert dims[c] >= max(dims) - 1
    for k in range(c):
        assert dims[k] <= dims[k + 1] + 1
    for k in range(c, nsect - 1):
        assert dims[k + 1] <= dims[k] + 1


def test_gaussian_sectors_limits():
    assert synth.gaussian_sectors(7, 7, 5) == [1] * 7
    assert synth.gaussian_sectors(35, 7, 5) == [5] * 7
    with pytest.raises(ValueError):
        synth.gaussian_sectors(6, 7, 5)
    with pytest.raises(ValueError):
        synth.gaussian_sectors(36, 7, 5)


def test_gaussian_sectors_2d():
    dims = synth.gaussian_sectors_2d(4096, (15, 15), 128)
    assert dims.shape == (15, 15) and int(dims.sum()) == 4096
    assert dims.min() >= 1 and dims.max() <= 128
    # the profile depends on the distance from the centre only
    assert abs(int(dims[7, 7]) - int(dims.max())) <= 1
    assert np.all(np.abs(dims - dims.T) <= 1)
    assert np.all(np.abs(dims - dims[::-1, ::-1]) <= 1)


def test_block_gaussian_is_keyed_not_ordered():
    a = synth.block_gaussian(5, "L", (1, 2, 3), (4, 5))
    synth.block_gaussian(5, "L", (0, 0, 0), (7,))          # another block drawn in between
    b = synth.block_gaussian(5, "L", (1, 2, 3), (4, 5))
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, synth.block_gaussian(5, "R", (1, 2, 3), (4, 5)))
    assert not np.array_equal(a, synth.block_gaussian(6, "L", (1, 2, 3), (4, 5)))
    assert not np.array_equal(a, synth.block_gaussian(5, "L", (1, 2, 4), (4, 5)))
    # N(0,1) entries
    big = synth.block_gaussian(1, "x", (0,), (200000,))
    assert abs(big.mean()) < 0.01 and abs(big.std() - 1.0) < 0.01


def test_product_spinors_seeded():
    v1, v2 = synth.product_spinors(1, 20, 2), synth.product_spinors(1, 20, 2)
    assert len(v1) == 20 and all(v.shape == (2,) for v in v1)
    assert all(np.array_equal(x, y) for x, y in zip(v1, v2))
    assert not np.array_equal(v1[0], synth.product_spinors(2, 20, 2)[0])


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bench_qn_links(which):
    _, kind, m, recipe, _ = bench.QN_CONFIGS[which]
    a = bench.qn_link(kind, m, recipe)
    assert a.dim == m
    qns = [q for q, _ in a.sectors]
    assert len(set(qns)) == len(qns)
    if kind == "hub":
        # (N, 2Sz) offsets from half filling: N - 2Sz is even (2 N_down)
        n, maxd = recipe
        assert a.nsect == n * n and all((q[0] - q[1]) % 2 == 0 for q in qns)
        assert (0, 0) in qns
    else:
        nsect, maxd = recipe
        assert a.nsect == nsect and all(q[0] % 2 == 0 for q in qns)
        assert (0,) in qns
    assert max(d for _, d in a.sectors) <= maxd and min(d for _, d in a.sectors) >= 1
