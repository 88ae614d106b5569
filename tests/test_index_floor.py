"""floor_div (bang_device.cuh): floor(n / d) from a float32 reciprocal, which the stencils
use for their spaxel-row and column ranges instead of integer division.  Emulated here in
float32 (reciprocal and product rounded to nearest, truncation at the end) and checked
against integer division over the ranges the kernels use (n < 2^21, d up to 1024), with the
margin the header's argument gives: (n + 1/2) / d lies at least 1 / (2d) from an integer."""
import numpy as np


def floor_div(n, d):
    f32 = np.float32
    inv = f32(1.0) / f32(d)
    return np.trunc((np.asarray(n).astype(f32) + f32(0.5)) * inv).astype(np.int64)


def test_matches_integer_division():
    rng = np.random.default_rng(5)
    n_all = np.concatenate([np.arange(0, 20000), rng.integers(0, 2 ** 21, 200000), np.arange(2 ** 21 - 5000, 2 ** 21)])
    for d in list(range(1, 130)) + [150, 192, 256, 300, 430, 534, 940, 1000, 1024]:
        assert np.array_equal(floor_div(n_all, d), n_all // d), d


def test_margin_exceeds_the_rounding():
    """The product's rounding error, at most (n + 1/2) / d x 2^-23, stays below the distance
    1 / (2d) to the nearest integer for every n < 2^21."""
    n = 2 ** 21
    assert (n + 0.5) * 2.0 ** -23 < 0.5
