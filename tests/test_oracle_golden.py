"""The oracle against the numbers the paper prints (tests/golden/paper_values.json)."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("case", GOLDEN["dealias_cutoff"]["cases"])
def test_dealias_cutoff(case):
    n = 96
    mk = O.mask(O.Model(shape=(n,), dt=1.0, dealias_order=case["order"]))
    q = np.abs(2 * np.pi * np.fft.fftfreq(n))
    cut = case["cutoff_over_pi"] * np.pi
    assert np.all(mk[q < cut - 1e-12] == 1)
    assert np.all(mk[q > cut + 1e-12] == 0)


def test_model_b_example_phases_and_interface():
    g = GOLDEN["model_b_example"]
    a, b, k = g["a"], g["b"], g["k"]
    n, dx = 128, 0.5
    m = O.Model(shape=(n,), dt=0.05, lhs=[(a, 1), (k, 2)], rhs=[(-b, 1)], power=3, dx=(dx, 1, 1), transform=2)
    x = (np.arange(n) + 0.5) * dx
    init = 0.9 * np.sign(np.sin(2 * np.pi * x / (n * dx)))
    r = O.to_real(m, O.run(m, np.fft.fft(init), 0, 8000))
    for p in g["phases"]:
        assert np.min(np.abs(r - p)) < 1e-3
    # thickness: distance over which phi goes from -tanh(1) to tanh(1) around one interface
    i = np.argmin(np.abs(r[n // 4: 3 * n // 4] - 0.0)) + n // 4
    xi = np.interp([-np.tanh(1), np.tanh(1)], -r[i - 20:i + 20], x[i - 20:i + 20])
    width = abs(xi[1] - xi[0]) / 2
    assert 0.7 * g["interface_thickness_approx"] < width < 1.6 * g["interface_thickness_approx"]


def test_noisy_diffusion_linear_operator():
    D = GOLDEN["noisy_diffusion"]["D"]
    m = O.Model(shape=(16, 16), dt=0.01, lhs=[(D, 1)])
    phi0 = np.fft.fft2(np.random.default_rng(3).uniform(-1, 1, (16, 16)))
    got = O.run(m, phi0, 0, 25)
    np.testing.assert_allclose(got, phi0 / (1 + 0.01 * D * O.q2(m)) ** 25, rtol=1e-12, atol=1e-12)


def test_conserved_noise_leaves_mass():
    g = GOLDEN["conserved_noise"]
    m = O.Model(shape=(16, 16), dt=0.1, noise_D=g["D"], noise_pow=g["q2_power"], noisy=True)
    for step in range(5):
        xi = O.noise(m, step)
        assert xi[0, 0] == 0 and np.any(xi != 0)
