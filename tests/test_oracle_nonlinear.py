"""Pins of the oracle's pseudo-spectral nonlinearity and de-aliasing (section
"De-aliasing", Eq. nonlin_general / cubicexampledealiased) against a brute-force
circular convolution, closed forms and the alias-free property of the order rule."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def _spectrum_of_real(shape, seed):
    x = inputs.real_field(shape, seed)
    return np.fft.fftn(x)


def _brute_cubic(d):
    """(1/N^2) sum_{k,l} d_k d_l d_{q-k-l}, indices modulo the lattice (direct triple sum)."""
    shape = d.shape
    n = d.size
    modes = list(itertools.product(*[range(s) for s in shape]))
    out = np.zeros(shape, dtype=complex)
    flat = {m: d[m] for m in modes if d[m] != 0}
    keys = list(flat)
    for k in keys:
        for l in keys:
            dk_dl = flat[k] * flat[l]
            for q in modes:
                m = tuple((q[j] - k[j] - l[j]) % shape[j] for j in range(len(shape)))
                out[q] += dk_dl * d[m]
    return out / n ** 2


def _model(shape, order):
    return O.Model(shape=shape, dt=0.1, power=3, rhs=[(1.0, 0)], dealias_order=order)


@pytest.mark.parametrize("shape,order", [((8,), 2), ((8,), 0), ((12,), 3), ((4, 4), 2), ((6, 4), 1), ((4, 2, 4), 2)])
def test_cubic_equals_brute_force_convolution(shape, order):
    m = _model(shape, order)
    phi = _spectrum_of_real(shape, seed=31)
    d = phi * O.mask(m)
    got = O.nonlinear(m, phi)
    ref = _brute_cubic(d)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n,order", [(8, 2), (16, 2), (1024, 2), (1024, 3), (64, 3), (12, 2), (7, 2), (256, 1)])
def test_mask_keeps_modes_below_cutoff(n, order):
    # "De-aliasing": zero every mode with |q| > 2 pi / ((n+1) dx); the equality case is zeroed.
    m = O.Model(shape=(n,), dt=1.0, dealias_order=order)
    mk = O.mask(m)
    k = np.fft.fftfreq(n) * n
    q = 2 * np.pi * k / n
    cutoff = 2 * np.pi / (order + 1)
    expect = (np.abs(q) < cutoff - 1e-12).astype(int)
    np.testing.assert_array_equal(mk, expect)
    # 2/3 rule at N = 1024 keeps |k| <= 341: 683 modes, 342 of them in the half spectrum
    if (n, order) == (1024, 2):
        assert mk.sum() == 683 and mk[: n // 2 + 1].sum() == 342


def test_mask_is_tensor_product_in_2d():
    m = O.Model(shape=(12, 8), dt=1.0, dealias_order=2)
    mk = O.mask(m)
    my = O.mask(O.Model(shape=(12,), dt=1.0, dealias_order=2))
    mx = O.mask(O.Model(shape=(8,), dt=1.0, dealias_order=2))
    np.testing.assert_array_equal(mk, np.outer(my, mx))


def test_cos_cubed_closed_form():
    # u = (A cos th)^3 = A^3 (3 cos th + cos 3 th) / 4
    n, k0, A = 32, 2, 0.7
    x = np.arange(n)
    phi = np.fft.fft(A * np.cos(2 * np.pi * k0 * x / n))
    m = _model((n,), 2)
    P = O.nonlinear(m, phi)
    ref = np.zeros(n, dtype=complex)
    ref[k0] = ref[-k0] = n * A ** 3 * 3 / 8
    ref[3 * k0] = ref[-3 * k0] = n * A ** 3 / 8
    assert np.max(np.abs(P - ref)) < 1e-12 * n


def test_uniform_field_cube():
    m = _model((4, 8), 2)
    c = 0.37
    phi = np.zeros((4, 8), dtype=complex)
    phi[0, 0] = 32 * c
    P = O.nonlinear(m, phi)
    ref = np.zeros_like(phi)
    ref[0, 0] = 32 * c ** 3
    assert np.max(np.abs(P - ref)) < 1e-13


def _linear_cubic_1d(d, n):
    """Non-circular (linear) convolution over signed wavenumbers, returned on the lattice."""
    ks = [k if k < n // 2 else k - n for k in range(n)]
    out = {}
    for i, j, l in itertools.product(range(n), repeat=3):
        if d[i] == 0 or d[j] == 0 or d[l] == 0:
            continue
        s = ks[i] + ks[j] + ks[l]
        out[s] = out.get(s, 0) + d[i] * d[j] * d[l]
    return {s: v / n ** 2 for s, v in out.items()}


def test_order_rule_is_alias_free_in_band():
    # With the order rule for a cubic (n_d = 3, cutoff 2 pi / 4), every kept output
    # mode equals the linear (non-wrapping) convolution: no aliasing lands in band.
    n = 16
    m = _model((n,), 3)
    phi = _spectrum_of_real((n,), seed=33)
    d = phi * O.mask(m)
    P = O.nonlinear(m, phi)
    lin = _linear_cubic_1d(d, n)
    for k in range(-3, 4):
        assert abs(P[k % n] - lin.get(k, 0)) < 1e-12
    # the 2/3 rule does alias a cubic: some kept mode differs from the linear convolution
    m2 = _model((n,), 2)
    d2 = phi * O.mask(m2)
    P2 = O.nonlinear(m2, phi)
    lin2 = _linear_cubic_1d(d2, n)
    kept = [k for k in range(-n // 2, n // 2) if 3 * abs(k) < n]
    assert max(abs(P2[k % n] - lin2.get(k, 0)) for k in kept) > 1e-3
