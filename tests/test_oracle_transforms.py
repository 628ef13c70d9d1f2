"""Pins of the oracle's transforms (the F, F^-1 of Eq. cubicexample) against
numpy.fft (a library routine), Parseval and the inverse/forward identity."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


@pytest.mark.parametrize("shape", [(1,), (2,), (3,), (5,), (8,), (12,), (16,), (4, 8), (6, 5), (3, 4, 4)])
@pytest.mark.parametrize("sign", [-1, +1])
def test_naive_dft_matches_numpy(shape, sign):
    x = inputs.complex_array(shape, seed=11)
    got = O.dft(x, sign, method=1)
    ref = np.fft.fftn(x) if sign < 0 else np.fft.ifftn(x) * x.size
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(2,), (4,), (64,), (1024,), (8, 4), (64, 32), (16, 8, 4), (8, 8, 8)])
@pytest.mark.parametrize("sign", [-1, +1])
def test_radix2_matches_numpy(shape, sign):
    x = inputs.complex_array(shape, seed=12)
    got = O.dft(x, sign, method=2)
    ref = np.fft.fftn(x) if sign < 0 else np.fft.ifftn(x) * x.size
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(16,), (8, 8), (4, 4, 4), (32, 16)])
def test_radix2_equals_naive(shape):
    x = inputs.complex_array(shape, seed=13)
    a = O.dft(x, -1, method=1)
    b = O.dft(x, -1, method=2)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_radix2_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        O.dft(np.ones(6, dtype=complex), -1, method=2)


@pytest.mark.parametrize("shape", [(64,), (16, 32), (8, 8, 16)])
def test_parseval_and_roundtrip(shape):
    x = inputs.real_field(shape, seed=14)
    X = O.dft(x.astype(complex), -1, method=2)
    n = x.size
    # sum |x|^2 = (1/N) sum |X|^2 for the unnormalised forward transform
    assert abs(np.sum(x * x) - np.sum(np.abs(X) ** 2) / n) <= 1e-13 * np.sum(x * x)
    back = O.dft(X, +1, method=2) / n
    assert np.max(np.abs(back - x)) <= 1e-14 * n


@pytest.mark.parametrize("shape", [(16,), (8, 12), (4, 8, 8)])
def test_real_input_is_hermitian(shape):
    x = inputs.real_field(shape, seed=15)
    X = O.dft(x.astype(complex), -1, method=1)
    # X(-q) = conj X(q): reverse every axis modulo its length
    idx = tuple((-np.arange(s)) % s for s in shape)
    Xm = X[np.ix_(*idx)]
    assert np.max(np.abs(Xm - np.conj(X))) <= 1e-12 * np.max(np.abs(X))
