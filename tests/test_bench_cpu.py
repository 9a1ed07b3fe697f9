"""bench.py's model of the sort's traffic (the sort roofline it reports): the number of
prefix-digit passes for a point set, worked out by hand for a few sets, and the bytes
per point of the sort's stages."""
import numpy as np

import bench


def test_active_prefix_passes():
    rng = np.random.default_rng(3)
    x, y = rng.random(1 << 15), rng.random(1 << 15)
    assert bench.active_sort_passes(x, y) == 4  # uniform: every byte of the 32-bit key varies
    # z = j 2^-31 with j < 2^16: the item's largest coordinate is below 2^-15, so its
    # keys step by 2^-47 and z's key is j 2^16 -- the two low bytes never vary
    j = rng.integers(0, 1 << 16, 1 << 16)
    z = j / 2.0 ** 31
    assert bench.active_sort_passes(z[: 1 << 15], z[1 << 15:]) == 2
    # one value, no padding (2 x 4096 points): no digit varies, one pass still writes
    assert bench.active_sort_passes(np.full(4096, 0.25), np.full(4096, 0.25)) == 1
    # one value with padding (5000 points): the padding key 0xFFFFFFFF differs in every byte
    assert bench.active_sort_passes(np.full(2500, 0.25), np.full(2500, 0.25)) == 4


def test_sort_bytes_per_point():
    # range 8 + histogram 8 read, 16 written + 32 per digit pass + detection 12
    assert bench.sort_bytes_per_point(4) == 8 + 24 + 4 * 32 + 12 == 172
    assert bench.sort_bytes_per_point(2) == 108
