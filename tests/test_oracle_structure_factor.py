"""Pins of the radially binned structure factor S(q) and coarsening length L(t)."""
import itertools

import numpy as np

from oracle import oracle as O
from tests import inputs


def test_single_mode_structure_factor_and_length():
    n, k0, A = 64, 4, 0.3
    m = O.Model(shape=(n, n), dt=1.0)
    # spectrum of phi(x, y) = A cos(2 pi k0 x / n): two modes of height n^2 A / 2
    phi = np.zeros((n, n), dtype=complex)
    phi[0, k0] = phi[0, n - k0] = n * n * A / 2
    S, cnt, L = O.structure_factor(m, phi, nbins=64)
    # |q0| = 2 pi k0 / n; s = 2 * 64 * k0 / n = 8 -> bin 7 (bins are (b, b+1] in units of pi/64)
    b = 7
    assert np.count_nonzero(S) == 1 and S[b] > 0
    total = 2 * (n * n * A / 2) ** 2 / (n * n)
    assert abs(S[b] * cnt[b] - total) < 1e-10 * total
    # L = 2 pi sum S / sum |q| S = 2 pi / |q0| = n / k0
    assert abs(L - n / k0) < 1e-12


def test_bin_counts_brute_force():
    n, nbins = 32, 16
    m = O.Model(shape=(n, n), dt=1.0)
    phi = np.fft.fft2(inputs.real_field((n, n), seed=51))
    S, cnt, L = O.structure_factor(m, phi, nbins=nbins)
    k = np.fft.fftfreq(n) * n
    ref_cnt = np.zeros(nbins)
    ref_S = np.zeros(nbins)
    for iy, ix in itertools.product(range(n), range(n)):
        kk = np.hypot(k[iy], k[ix])
        if kk == 0:
            continue
        qq = 2 * np.pi * kk / n
        if qq > np.pi + 1e-12:
            continue
        bb = int(np.ceil(qq / (np.pi / nbins) - 1e-9)) - 1
        ref_cnt[bb] += 1
        ref_S[bb] += abs(phi[iy, ix]) ** 2 / n ** 2
    np.testing.assert_array_equal(cnt, ref_cnt)
    np.testing.assert_allclose(S * cnt, ref_S, rtol=1e-12)
