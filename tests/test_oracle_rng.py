"""Pins of the SplitMix64 initial-block generator (oracle side)."""
import os

import numpy as np

from oracle import rng


def test_splitmix64_published_seed0_sequence(golden_dir):
    with open(os.path.join(golden_dir, "splitmix64_seed0.txt")) as f:
        want = [int(line, 16) for line in f if line.strip() and not line.startswith("#")]
    got = [int(v) for v in rng.splitmix64(0, len(want))]
    assert got == want


def test_splitmix64_offset_stream_matches_prefix():
    full = rng.splitmix64(12345, 100)
    tail = rng.splitmix64(12345, 40, start=60)
    assert np.array_equal(full[60:], tail)


def test_uniform_block_layout_and_range():
    n, m = 37, 5
    X = rng.uniform_block(2, n, m)
    assert X.shape == (n, m)
    flat = rng.splitmix64(2, n * m)
    # column-major: entry (p, j) is output p + n*j
    p, j = 11, 3
    want = 2.0 * float(int(flat[p + n * j]) >> 11) * 2.0 ** -53 - 1.0
    assert X[p, j] == want
    big = rng.uniform_block(7, 4096, 8)
    assert big.min() >= -1.0 and big.max() < 1.0
    assert abs(big.mean()) < 0.02 and abs(big.var() - 1.0 / 3.0) < 0.02
