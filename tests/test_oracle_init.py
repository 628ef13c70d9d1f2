"""Pins of the oracle's initial field: the paper's "small random perturbation"
(sections "Example" and "Writing models"), read as a uniform field drawn from
the same counter-based generator as the noise.

phi_x = lo + (hi - lo) u_x with u_x = ((w >> 8) + 0.5) / 2^24, w the first word
of Philox4x32-10(counter = (site, 0, field_id, 1), key = seed).  The affine map,
the counter layout and the distribution are each pinned by something other
than the function itself: the range [lo, hi) and its ends, the first two
moments against the uniform law's closed forms, a chi-square test of 64 equal
bins, the site order against the generator pinned bit for bit elsewhere, and
the orientation (lo at u -> 0, hi at u -> 1) by a single-site map.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _field(shape, seed=77, field_id=0, lo=-0.1, hi=0.3):
    m = O.Model(shape=shape, dt=0.1, seed=seed, field_id=field_id)
    return O.init_uniform(m, lo, hi)


@pytest.mark.parametrize("lo,hi", [(-0.1, 0.1), (-0.05, 0.05), (0.25, 2.0), (-3.0, -1.0)])
def test_range_mean_variance(lo, hi):
    shape = (256, 256)
    x = _field(shape, seed=2405, lo=lo, hi=hi).ravel()
    n = x.size
    assert x.min() >= lo and x.max() < hi
    # the 24-bit lattice reaches within 2^-24 (hi - lo) of both ends
    assert x.min() - lo < 1e-4 * (hi - lo) and hi - x.max() < 1e-4 * (hi - lo)
    w = hi - lo
    mean, var = (lo + hi) / 2, w * w / 12
    # standard errors of the sample mean and variance of U(lo, hi)
    se_mean = math.sqrt(var / n)
    mu4 = w ** 4 / 80
    se_var = math.sqrt((mu4 - var * var) / n)
    assert abs(x.mean() - mean) < 5 * se_mean, (x.mean(), mean)
    assert abs(x.var() - var) < 5 * se_var, (x.var(), var)


def test_chi_square_64_bins():
    lo, hi = -0.1, 0.1
    x = _field((512, 512), seed=11, lo=lo, hi=hi).ravel()
    counts, _ = np.histogram(x, bins=64, range=(lo, hi))
    e = x.size / 64
    chi2 = float(((counts - e) ** 2 / e).sum())
    # 63 degrees of freedom: mean 63, sd sqrt(126) ~ 11.2; 5 sd above the mean
    assert chi2 < 63 + 5 * math.sqrt(126), chi2
    assert counts.sum() == x.size


def test_site_order_and_affine_map_against_the_generator():
    # site s takes word 0 of Philox((s, 0, field_id, 1), (seed_lo, seed_hi)); the generator
    # itself is pinned bit for bit against an independent implementation
    shape, seed, fid, lo, hi = (4, 8), 0x1234_5678_9ABC_DEF0, 2, -0.5, 1.5
    x = _field(shape, seed=seed, field_id=fid, lo=lo, hi=hi).ravel()
    n = x.size
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 2] = fid
    ctr[:, 3] = 1
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    w = O.philox(ctr, key)[:, 0]
    u = ((w >> 8).astype(np.float64) + 0.5) / 2.0 ** 24
    np.testing.assert_array_equal(x, lo + (hi - lo) * u)


def test_orientation_of_the_map():
    # a field with lo > hi is the mirror image: lo + (hi - lo) u with the same u
    a = _field((16, 16), seed=5, lo=0.0, hi=1.0)
    b = _field((16, 16), seed=5, lo=1.0, hi=0.0)
    np.testing.assert_allclose(a + b, 1.0, rtol=0, atol=1e-15)
    # u is strictly inside (0, 1): the smallest value is above lo by at least 2^-25
    assert a.min() >= 2.0 ** -25 and a.max() <= 1.0 - 2.0 ** -25


def test_fields_and_seeds_draw_different_streams():
    a = _field((64, 64), seed=1, field_id=0)
    b = _field((64, 64), seed=1, field_id=1)
    c = _field((64, 64), seed=2, field_id=0)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    # independent streams: correlation within 5 standard errors of 0
    for y in (b, c):
        r = np.corrcoef(a.ravel(), y.ravel())[0, 1]
        assert abs(r) < 5 / math.sqrt(a.size), r
