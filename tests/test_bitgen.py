"""Pins for the seeded input generator (bitgen): the published SplitMix64
stream, the definition re-evaluated in pure Python, density and thresholds."""
import math
import os

import numpy as np
import pytest

import bitgen
from conftest import GOLDEN


def test_draw_matches_published_splitmix64_stream():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        want = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    got = [bitgen.draw(0, 0, c) for c in range(len(want))]
    assert got == want


def test_c_draw_matches_definition_in_python():
    for seed, mid, c in [(1, 0, 0), (1, 1, 5), (5, 3, 123456789), (2**30, 1, 2**40)]:
        assert bitgen.draw(seed, mid, c) == bitgen.draw_py(seed, mid, c)


def test_dense_fill_layout():
    rows, cols, seed = 5, 192, 7
    M = bitgen.fill_cpu(rows, cols, seed, 1)
    wpr = cols // 64
    for i in range(rows):
        for w in range(wpr):
            assert int(M[i, w]) == bitgen.draw_py(seed, 1, i * wpr + w)
    # row window equals the same rows of the full matrix
    part = bitgen.fill_cpu(rows, cols, seed, 1, row0=2, nrows=2)
    assert (part == M[2:4]).all()


def test_threshold_fill_layout():
    rows, cols, seed = 3, 128, 2
    theta = bitgen.theta_pow2(3)
    M = bitgen.fill_cpu(rows, cols, seed, 0, p="2^-3")
    for i in range(rows):
        for j in range(cols):
            bit = (int(M[i, j // 64]) >> (j % 64)) & 1
            assert bit == int(bitgen.draw_py(seed, 0, i * cols + j) < theta)


def test_thresholds():
    assert bitgen.theta_pow2(6) == 2**58
    t = bitgen.theta_pow2_half(7)
    assert t * t <= 2**113 < (t + 1) ** 2
    assert abs(t / 2.0**64 - 2**-7.5) < 1e-15
    assert bitgen.spec("1/64") == (bitgen.THRESHOLD, 2**58)
    assert bitgen.spec(None) == (bitgen.DENSE, 0)
    tk = bitgen.theta_inv_sqrt(4096)
    assert tk == 2**58


@pytest.mark.parametrize("p,expect", [(None, 0.5), ("1/64", 1 / 64), ("2^-7.5", 2**-7.5)])
def test_density(p, expect):
    M = bitgen.fill_cpu(512, 1024, 3, 0, p=p)
    ones = int(np.unpackbits(M.view(np.uint8)).sum())
    frac = ones / (512 * 1024)
    sd = math.sqrt(expect * (1 - expect) / (512 * 1024))
    assert abs(frac - expect) < 6 * sd


def test_batched_shapes():
    shapes = bitgen.batched_shapes(2048, 5)
    assert len(shapes) == 2048
    for m, k, n, op in shapes:
        for d in (m, k, n):
            assert 256 <= d <= 8192 and d % 64 == 0
    assert sum(op for *_, op in shapes) == 1024
    logs = np.log([s[0] for s in shapes])
    assert abs(logs.mean() - (math.log(256) + math.log(8192)) / 2) < 0.1
