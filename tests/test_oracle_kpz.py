"""The KPZ nonlinearity of the oracle (section "Writing models": lambda psi^2
with psi = grad phi), pinned by closed forms of single modes, by what the
de-alias mask and the Nyquist index must give, and by the step's q = 0 mode."""
import numpy as np
import pytest

from oracle import oracle as O


def _spectrum_of(m, real):
    return O.to_spectrum(m, real)


def _cos_mode(shape, axis, k, amp):
    # amp cos(2 pi k x_axis / N_axis) on the lattice (axis 0 = x, the last array axis)
    idx = np.indices(shape)
    coord = idx[len(shape) - 1 - axis]
    n = shape[len(shape) - 1 - axis]
    return amp * np.cos(2 * np.pi * k * coord / n)


@pytest.mark.parametrize("shape,axis,k", [((64,), 0, 5), ((16, 32), 1, 3), ((16, 32), 0, 7), ((8, 8, 16), 2, 1), ((16, 8, 8), 2, 5)])
def test_one_cosine_mode(shape, axis, k):
    # (d/dx_j [A cos(q x_j)])^2 = A^2 q^2 (1 - cos(2 q x_j)) / 2: the transform has
    # N A^2 q^2 / 2 at q = 0 and -N A^2 q^2 / 4 at +-2q along that axis, nothing else
    amp = 0.7
    m = O.kpz(shape, noisy=False)
    P = O.nonlinear(m, _spectrum_of(m, _cos_mode(shape, axis, k, amp)))
    n_ax = shape[len(shape) - 1 - axis]
    q = 2 * np.pi * k / n_ax
    N = int(np.prod(shape))
    want = np.zeros(shape, dtype=complex)
    zero = (0,) * len(shape)
    want[zero] = N * amp ** 2 * q ** 2 / 2
    for s in (1, -1):
        ix = [0] * len(shape)
        ix[len(shape) - 1 - axis] = (s * 2 * k) % n_ax
        want[tuple(ix)] = -N * amp ** 2 * q ** 2 / 4
    np.testing.assert_allclose(P, want, atol=1e-9 * N)


def test_two_axes_add_without_cross_terms():
    # A cos(q_a x) + B cos(q_b y): the squares of the two partial derivatives add;
    # a cross term d_x phi d_y phi would put weight at (+-q_a, +-q_b)
    ny, nx, ka, kb, A, B = 16, 32, 3, 2, 0.5, 0.8
    m = O.kpz((ny, nx), noisy=False)
    r = _cos_mode((ny, nx), 0, ka, A) + _cos_mode((ny, nx), 1, kb, B)
    P = O.nonlinear(m, O.to_spectrum(m, r))
    qa, qb, N = 2 * np.pi * ka / nx, 2 * np.pi * kb / ny, nx * ny
    assert abs(P[0, 0] - N * (A ** 2 * qa ** 2 + B ** 2 * qb ** 2) / 2) < 1e-9 * N
    assert abs(P[0, 2 * ka] + N * A ** 2 * qa ** 2 / 4) < 1e-9 * N
    assert abs(P[2 * kb, 0] + N * B ** 2 * qb ** 2 / 4) < 1e-9 * N
    P2 = P.copy()
    for ix in [(0, 0), (0, 2 * ka), (0, nx - 2 * ka), (2 * kb, 0), (ny - 2 * kb, 0)]:
        P2[ix] = 0
    assert np.max(np.abs(P2)) < 1e-9 * N


def test_masked_and_nyquist_modes_do_not_enter():
    n = 48
    # k = 20: 3 * 20 >= 48, outside the two-thirds band
    m = O.kpz((n,), noisy=False)
    assert np.max(np.abs(O.nonlinear(m, O.to_spectrum(m, _cos_mode((n,), 0, 20, 1.0))))) < 1e-9
    # the Nyquist mode (-1)^x, with every mode kept: its derivative is 0
    m0 = O.kpz((n,), noisy=False, dealias_order=0)
    assert np.max(np.abs(O.nonlinear(m0, O.to_spectrum(m0, _cos_mode((n,), 0, n // 2, 1.0))))) < 1e-9


def test_matches_a_brute_force_gradient_on_a_small_lattice():
    # direct sums: psi_j(x) = (1/N) sum_q m_q i q_j phi_q e^{i q.x}, P_q = sum_x |psi|^2 e^{-i q.x}
    ny, nx = 6, 8
    g = np.random.default_rng(3)
    m = O.kpz((ny, nx), noisy=False, dealias_order=1)
    phi = O.to_spectrum(m, g.standard_normal((ny, nx)))
    ky = np.fft.fftfreq(ny, 1.0 / ny)
    kx = np.fft.fftfreq(nx, 1.0 / nx)
    keep = (2 * np.abs(ky)[:, None] < ny) & (2 * np.abs(kx)[None, :] < nx)
    qy = np.where(np.abs(ky) == ny / 2, 0.0, 2 * np.pi * ky / ny)
    qx = np.where(np.abs(kx) == nx / 2, 0.0, 2 * np.pi * kx / nx)
    y, x = np.indices((ny, nx))
    N = nx * ny
    grad2 = np.zeros((ny, nx))
    for qj in (qx[None, :] * np.ones((ny, 1)), qy[:, None] * np.ones((1, nx))):
        psi = np.zeros((ny, nx), dtype=complex)
        for a in range(ny):
            for b in range(nx):
                if keep[a, b]:
                    psi += 1j * qj[a, b] * phi[a, b] * np.exp(2j * np.pi * (ky[a] * y / ny + kx[b] * x / nx))
        grad2 += (psi.real / N) ** 2
    want = np.zeros((ny, nx), dtype=complex)
    for a in range(ny):
        for b in range(nx):
            want[a, b] = np.sum(grad2 * np.exp(-2j * np.pi * (ky[a] * y / ny + kx[b] * x / nx)))
    np.testing.assert_allclose(O.nonlinear(m, phi), want, atol=1e-10)


def test_the_mean_grows_by_lambda_times_the_mean_square_gradient():
    # q = 0: O(0) = 0 and M(0) = lambda, so one noiseless step adds dt lambda P_0
    shape, dt, lam = (32, 32), 0.05, 0.8
    m = O.kpz(shape, dt=dt, sigma=1.0, lam=lam, noisy=False)
    phi = O.to_spectrum(m, O.init_uniform(m, -0.5, 0.5))
    P0 = O.nonlinear(m, phi)[0, 0]
    after = O.run(m, phi, 0, 1)
    assert abs(after[0, 0] - (phi[0, 0] + dt * lam * P0)) < 1e-10 * abs(P0)
    assert P0.real > 0


def test_lambda_zero_is_edwards_wilkinson():
    shape, dt, sigma = (16, 16), 0.1, 0.7
    m = O.kpz(shape, dt=dt, sigma=sigma, lam=0.0, noisy=False)
    phi = O.to_spectrum(m, O.init_uniform(m, -1, 1))
    ky = np.fft.fftfreq(16, 1 / 16)
    q2 = (2 * np.pi / 16) ** 2 * (ky[:, None] ** 2 + ky[None, :] ** 2)
    np.testing.assert_allclose(O.run(m, phi, 0, 3), phi / (1 + dt * sigma * q2) ** 3, atol=1e-11)
