"""Pins of the oracle's time step, Eq. (timeupdate), by closed forms of the
scheme and by invariants of the models (conservation, Lyapunov decrease, the
exact stationary variance of linear noisy modes, the 1D Cahn-Hilliard kink)."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def _poly(coefs, q2):
    return sum(c * q2 ** p for c, p in coefs)


def test_linear_decay_closed_form():
    # b = 0, D = 0: phi_q(n) = phi_q(0) / (1 + dt O(q))^n
    m = O.Model(shape=(16, 16), dt=0.05, lhs=[(0.3, 0), (-0.2, 1), (0.5, 2)])
    phi0 = np.fft.fftn(inputs.real_field((16, 16), seed=41))
    n = 40
    got = O.run(m, phi0, 0, n)
    q2 = O.q2(m)
    ref = phi0 / (1 + m.dt * _poly(m.lhs, q2)) ** n
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_q2_is_continuum_symbol():
    m = O.Model(shape=(4, 8), dt=1.0, dx=(0.5, 2.0, 1.0))
    ky = np.fft.fftfreq(4) * 4
    kx = np.fft.fftfreq(8) * 8
    qy = 2 * np.pi * ky / (4 * 2.0)
    qx = 2 * np.pi * kx / (8 * 0.5)
    ref = qy[:, None] ** 2 + qx[None, :] ** 2
    np.testing.assert_allclose(O.q2(m), ref, rtol=1e-15, atol=0)


def test_uniform_field_follows_scalar_recursion():
    # Model A with K = 0 on a uniform field reduces to the ODE dphi/dt = -(a phi + b phi^3);
    # the scheme gives c' = (c - dt b c^3) / (1 + dt a), converging to sqrt(-a/b) ("Example": phi = +-1).
    a, b, dt = -1.0, 1.0, 0.05
    # no de-aliasing: with K = 0 a masked mode would grow like (1 + dt a)^-n without bound
    m = O.Model(shape=(8, 8), dt=dt, lhs=[(a, 0)], rhs=[(-b, 0)], power=3, dealias_order=0)
    c = 0.2
    phi = np.zeros((8, 8), dtype=complex)
    phi[0, 0] = 64 * c
    for s in range(30):
        phi = O.run(m, phi, s, 1)
        c = (c - dt * b * c ** 3) / (1 + dt * a)
        assert abs(phi[0, 0].real / 64 - c) < 1e-14
    assert np.max(np.abs(phi.ravel()[1:])) < 1e-12
    phi = O.run(m, phi, 30, 2000)
    assert abs(phi[0, 0].real / 64 - np.sqrt(-a / b)) < 1e-10


def test_model_b_conserves_mass_exactly():
    m = O.model_b((32, 32), D=0.05)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.1, 0.3))
    phi = O.run(m, phi0, 0, 50)
    assert phi[0, 0] == phi0[0, 0]
    real = O.to_real(m, phi)
    assert abs(real.sum() - O.init_uniform(m, -0.1, 0.3).sum()) < 1e-11


def _free_energy(m, phi, a, b, K):
    # G = sum_x [a/2 phi^2 + b/4 phi^4] + K/2 sum_x |grad phi|^2 (gradient spectrally)
    r = O.to_real(m, phi)
    grad2 = np.sum(O.q2(m) * np.abs(phi) ** 2) / m.n_sites
    return np.sum(a / 2 * r ** 2 + b / 4 * r ** 4) + K / 2 * grad2


@pytest.mark.parametrize("which", ["A", "B"])
def test_free_energy_decreases(which):
    # Models A and B are gradient flows of G; without de-aliasing and noise the
    # discrete scheme must lower G every step at small dt.
    a, b, K = -1.0, 1.0, 1.0
    mk = O.model_a if which == "A" else O.model_b
    m = mk((32, 32), dt=0.02, a=a, b=b, K=K, noisy=False, dealias_order=0)
    phi = O.to_spectrum(m, O.init_uniform(m, -0.5, 0.5))
    G = _free_energy(m, phi, a, b, K)
    for s in range(40):
        phi = O.run(m, phi, s, 1)
        G2 = _free_energy(m, phi, a, b, K)
        assert G2 < G
        G = G2


def test_step_is_resumable():
    m = O.model_b((16, 16), D=0.1)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1))
    full = O.run(m, phi0, 0, 10)
    half = O.run(O.model_b((16, 16), D=0.1), O.run(m, phi0, 0, 4), 4, 6)
    np.testing.assert_array_equal(full, half)


def test_noise_reality_and_real_space_variance():
    # Model A noise: a real field with per-site variance 2 D dt / dV per step
    D, dt = 0.3, 0.2
    m = O.model_a((64, 64), dt=dt, D=D, dx=(0.5, 0.5, 1.0))
    var = []
    for step in range(4):
        xi = O.noise(m, step)
        r = O.dft(xi, +1, 2) / m.n_sites
        assert np.max(np.abs(r.imag)) < 1e-12 * np.max(np.abs(r.real))
        var.append(np.var(r.real))
    n = 4 * m.n_sites
    expect = 2 * D * dt / 0.25
    assert abs(np.mean(var) / expect - 1) < 5 * np.sqrt(2 / n)


def test_conserved_noise_spectrum():
    # D~ = D q^2: the q = 0 mode gets no noise; E|xi_q|^2 = N 2 D q^2 dt / dV
    D, dt = 0.2, 0.1
    m = O.model_b((64, 64), dt=dt, D=D)
    q2 = O.q2(m)
    acc = np.zeros((64, 64))
    nsamp = 6
    for step in range(nsamp):
        xi = O.noise(m, step)
        assert xi[0, 0] == 0
        acc += np.abs(xi) ** 2
    ratio = acc[q2 > 0] / (nsamp * m.n_sites * 2 * D * q2[q2 > 0] * dt)
    assert abs(ratio.mean() - 1) < 5 / np.sqrt(ratio.size * nsamp / 2)


def test_noise_draws_once_per_pair():
    m = O.model_a((8, 6), dt=1.0, D=1.0, seed=5)
    xi = O.noise(m, 3)
    idx = tuple((-np.arange(s)) % s for s in (8, 6))
    np.testing.assert_array_equal(xi[np.ix_(*idx)], np.conj(xi))
    # self-conjugate modes are real
    for ky in (0, 4):
        for kx in (0, 3):
            assert xi[ky, kx].imag == 0


@pytest.mark.parametrize("which", ["A", "B"])
def test_stationary_variance_of_linear_modes(which):
    # b = 0, a > 0: each mode is an AR(1) process phi' = g (phi + xi), g = 1/(1 + dt O(q)),
    # E|xi|^2 = s = N 2 D~ dt / dV.  From phi = 0: E|phi(n)|^2 = s g^2 (1 - g^{2n}) / (1 - g^2).
    a, K, D, dt = 0.5, 1.0, 0.1, 0.1
    shape = (32, 32)
    if which == "A":
        m = O.Model(shape=shape, dt=dt, lhs=[(a, 0), (K, 1)], noise_D=D, noise_pow=0, noisy=True, seed=7)
    else:
        m = O.Model(shape=shape, dt=dt, lhs=[(a, 1), (K, 2)], noise_D=D, noise_pow=1, noisy=True, seed=7)
    q2 = O.q2(m)
    O_q = _poly(m.lhs, q2)
    g = 1 / (1 + dt * O_q)
    s = m.n_sites * 2 * D * (q2 ** m.noise_pow) * dt
    phi = np.zeros(shape, dtype=complex)
    ratios = []
    step = 0
    for block in range(4):
        phi = O.run(m, phi, step, 60)
        step += 60
        pred = s * g ** 2 * (1 - g ** (2 * step)) / (1 - g ** 2)
        sel = pred > 0
        ratios.append(np.abs(phi[sel]) ** 2 / pred[sel])
    r = np.concatenate(ratios)
    # each ratio is ~Exp(1) (chi^2_2 / 2; chi^2_1 on self-conjugate modes); allow 5 sigma
    assert abs(r.mean() - 1) < 5 * np.sqrt(2.0 / r.size) * 1.5


def test_model_b_kink_matches_tanh_profile():
    # 1D Cahn-Hilliard, -a = b = 1, K = k: the stationary kink is tanh(x / w), w = sqrt(2K/(-a)),
    # between the phases phi = +-sqrt(-a/b) ("Example" section: phases at +-1).
    a, b, K, n, dx = -1.0, 1.0, 4.0, 256, 0.5
    m = O.Model(shape=(n,), dt=0.05, lhs=[(a, 1), (K, 2)], rhs=[(-b, 1)], power=3,
                dealias_order=2, dx=(dx, 1.0, 1.0), transform=2)
    x = (np.arange(n) + 0.5) * dx
    Lbox = n * dx
    w_exact = np.sqrt(2 * K / -a)
    # start from two kinks of the wrong width and let the profile relax
    init = np.tanh((x - Lbox / 4) / 1.5) * np.tanh((3 * Lbox / 4 - x) / 1.5)
    phi = O.run(m, np.fft.fft(init), 0, 16000)
    r = O.to_real(m, phi)
    ref = np.tanh((x - Lbox / 4) / w_exact) * np.tanh((3 * Lbox / 4 - x) / w_exact)
    assert np.max(np.abs(r - ref)) < 5e-4
    assert abs(np.max(r) - 1) < 5e-4 and abs(np.min(r) + 1) < 5e-4
