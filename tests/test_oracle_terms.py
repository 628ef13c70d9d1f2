"""General product terms of the oracle (Eq. basefourier; section "Writing
models": N = M prod_k psi_k^n_k with psi_k the fields acted on by differential
operators), pinned by the C oracle's own step, closed forms of cosine modes,
the sign of the first derivative, and the exact rotation of two linearly
coupled uniform fields."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _cos(shape, axis, k, amp, phase=0.0):
    idx = np.indices(shape)
    n = shape[len(shape) - 1 - axis]
    return amp * np.cos(2 * np.pi * k * idx[len(shape) - 1 - axis] / n + phase)


def test_single_power_term_is_the_c_oracle_step():
    # Model B written as one general term: the same numbers as orc_run
    for shape in [(16, 16), (32,), (8, 8, 16)]:
        m = O.model_b(shape, dt=0.01, seed=3)
        phi = O.to_spectrum(m, O.init_uniform(m, -0.3, 0.3))
        a = O.run(m, phi, 0, 5)
        b = O.run_coupled([m], [O.Term(0, [(-1.0, 1)], [O.Factor(0, 3)])], [phi], 0, 5)[0]
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_kpz_as_derivative_terms_is_the_c_oracle_step():
    for shape in [(16, 16), (8, 8, 16)]:
        m = O.kpz(shape, dt=0.02, lam=0.6, seed=4)
        phi = O.to_spectrum(m, O.init_uniform(m, -0.5, 0.5))
        terms = [O.Term(0, [(0.6, 0)], [O.Factor(0, 2, deriv=j)]) for j in range(len(shape))]
        a = O.run(m, phi, 0, 5)
        b = O.run_coupled([m], terms, [phi], 0, 5)[0]
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_product_of_two_fields():
    # A cos(q_a x) B cos(q_b y) = AB/4 sum of the four (+-q_a, +-q_b) modes
    ny, nx, ka, kb, A, B = 16, 32, 3, 2, 0.5, 0.8
    ms = [O.model_a((ny, nx), field_id=i, noisy=False) for i in range(2)]
    phis = [O.to_spectrum(ms[0], _cos((ny, nx), 0, ka, A)), O.to_spectrum(ms[1], _cos((ny, nx), 1, kb, B))]
    P = O.term_products(ms, [O.Term(0, [(1.0, 0)], [O.Factor(0), O.Factor(1)])], phis)
    want = np.zeros((ny, nx), dtype=complex)
    for sy in (1, -1):
        for sx in (1, -1):
            want[(sy * kb) % ny, (sx * ka) % nx] = nx * ny * A * B / 4
    np.testing.assert_allclose(P[0], want, atol=1e-9)
    assert np.max(np.abs(P[1])) == 0


def test_laplacian_factor_and_operator():
    # phi lap(phi) for A cos(q x) is -q^2 A^2 cos^2; with M = q^2 on top
    n, k, A = 64, 5, 0.9
    m = O.model_a((n,), noisy=False)
    phi = O.to_spectrum(m, _cos((n,), 0, k, A))
    q = 2 * np.pi * k / n
    P = O.term_products([m], [O.Term(0, [(2.0, 1)], [O.Factor(0), O.Factor(0, lap=1)])], [phi])[0]
    want = np.zeros(n, dtype=complex)
    # M(0) = 0 removes the mean -q^2 A^2 n / 2
    want[2 * k] = want[n - 2 * k] = 2.0 * (2 * q) ** 2 * (-q * q * A * A * n / 4)
    np.testing.assert_allclose(P, want, atol=1e-9)


def test_the_sign_of_the_first_derivative():
    # d/dx sin(q x) = q cos(q x); sin(q x) d/dx sin(q x) = (q/2) sin(2 q x)
    n, k = 32, 3
    m = O.model_a((n,), noisy=False)
    s = O.to_spectrum(m, _cos((n,), 0, k, 1.0, -np.pi / 2))
    q = 2 * np.pi * k / n
    d = O.term_products([m], [O.Term(0, [(1.0, 0)], [O.Factor(0, deriv=0)])], [s])[0]
    want = np.zeros(n, dtype=complex)
    want[k] = want[n - k] = n * q / 2
    np.testing.assert_allclose(d, want, atol=1e-10)
    ps = O.term_products([m], [O.Term(0, [(1.0, 0)], [O.Factor(0), O.Factor(0, deriv=0)])], [s])[0]
    want = np.zeros(n, dtype=complex)
    want[2 * k] = -1j * n * q / 4
    want[n - 2 * k] = 1j * n * q / 4
    np.testing.assert_allclose(ps, want, atol=1e-10)


def test_linear_coupling_rotates_uniform_fields():
    # dt phi = -c psi, dt psi = c phi, explicit: each step multiplies the uniform
    # pair by sqrt(1 + dt^2 c^2) and turns it by atan(dt c)
    shape, dt, c, n = (8, 8), 0.05, 1.3, 40
    ms = [O.Model(shape=shape, dt=dt, field_id=i) for i in range(2)]
    terms = [O.Term(0, [(-c, 0)], [O.Factor(1)]), O.Term(1, [(c, 0)], [O.Factor(0)])]
    u0, v0 = 0.4, -0.1
    phis = [O.to_spectrum(ms[0], np.full(shape, u0)), O.to_spectrum(ms[1], np.full(shape, v0))]
    out = O.run_coupled(ms, terms, phis, 0, n)
    g, th = (1 + dt * dt * c * c) ** (n / 2), n * math.atan(dt * c)
    u = g * (u0 * math.cos(th) - v0 * math.sin(th))
    v = g * (u0 * math.sin(th) + v0 * math.cos(th))
    N = 64
    assert abs(out[0][0, 0] - N * u) < 1e-10 and abs(out[1][0, 0] - N * v) < 1e-10
    assert np.max(np.abs(out[0].ravel()[1:])) < 1e-10
