"""The add-and-reinterpret float-to-integer rounding used by the spreading
kernel's fixed-point accumulation, checked in IEEE single precision on the
host: for |v| <= 2^22, the bits of float32(v + 1.5 * 2^23) minus those of
1.5 * 2^23 equal v rounded to the nearest integer, ties to even."""
import numpy as np


def _to_fixed(v):
    v = np.asarray(v, dtype=np.float32)
    s = (v + np.float32(12582912.0)).astype(np.float32)
    return s.view(np.int32).astype(np.int64) - 0x4B400000


def test_matches_round_half_even():
    rng = np.random.default_rng(3)
    for scale in (1.0, 1e3, 1e6, 2.0 ** 22):
        v = ((2 * rng.random(200000) - 1) * scale).astype(np.float32)
        v = v[np.abs(v) <= 2.0 ** 22]
        assert np.array_equal(_to_fixed(v), np.rint(v.astype(np.float64)).astype(np.int64))


def test_ties_and_limits():
    v = np.array([0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 2.0 ** 22, -2.0 ** 22, 0.0, -0.0], dtype=np.float32)
    assert list(_to_fixed(v)) == [0, 2, 2, 0, -2, -2, 2 ** 22, -2 ** 22, 0, 0]
