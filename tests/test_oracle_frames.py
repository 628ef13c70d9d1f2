"""Boundary frames (section "Callback functions") in the oracle: the frame
sits where the paper's example puts it, comes after the step, and the
heat-bath example relaxes to the straight line the paper states."""
import numpy as np

from oracle import oracle as O


def _diffusion(n, dt):
    # dt T = d_x^2 T: O(q) = q^2, no explicit term, no noise
    return O.Model(shape=(n,), dt=dt, lhs=[(1.0, 1)], rhs=[], power=0, noisy=False)


def test_first_step_from_zero_is_the_transform_of_the_frame():
    # phi = 0 stays 0 under the step; the frame then leaves the two boxes,
    # whose transform is a geometric sum per box
    n, w, lo, hi = 48, 5, 3.0, -2.0
    m = _diffusion(n, 0.1)
    got = O.run_framed(m, np.zeros(n, dtype=complex), 0, 1, w, lo, hi)
    q = 2 * np.pi * np.arange(n) / n
    z = np.exp(-1j * q)
    box = np.where(np.arange(n) == 0, w, (1 - z ** w) / np.where(np.arange(n) == 0, 1, 1 - z))
    want = lo * box + hi * z ** (n - w) * box
    np.testing.assert_allclose(got, want, atol=1e-11)


def test_the_frame_follows_the_step():
    # one step of diffusion from a framed field, then the frame: inside the
    # frames the values are exact, elsewhere they are the diffused ones
    n, w, dt = 32, 3, 0.7
    m = _diffusion(n, dt)
    r0 = np.cos(2 * np.pi * 3 * np.arange(n) / n)
    got = O.to_real(m, O.run_framed(m, O.to_spectrum(m, r0), 0, 1, w, 1.5, -0.5))
    diffused = r0 / (1 + dt * (2 * np.pi * 3 / n) ** 2)     # the cosine is one mode pair, q = 2 pi 3 / n
    np.testing.assert_allclose(got[:w], 1.5, atol=1e-12)
    np.testing.assert_allclose(got[n - w:], -0.5, atol=1e-12)
    np.testing.assert_allclose(got[w:n - w], diffused[w:n - w], atol=1e-12)


def test_width_zero_is_the_plain_run():
    m = O.model_b((16, 16), dt=0.01, seed=4)
    phi = O.to_spectrum(m, O.init_uniform(m, -0.2, 0.2))
    np.testing.assert_array_equal(O.run_framed(m, phi, 0, 5, 0, 1.0, 2.0), O.run(m, phi, 0, 5))


def test_heat_bath_relaxes_to_the_straight_line():
    # the paper's heat-bath example with a frame of several sites: the steady
    # state between the baths is the line from T1 to T2
    n, w, t1, t2, dt = 64, 6, 10.0, 0.0, 0.5
    m = _diffusion(n, dt)
    phi = O.run_framed(m, O.to_spectrum(m, np.full(n, 5.0)), 0, 3000, w, t1, t2)
    r = O.to_real(m, phi)
    xl, xr = w - 1, n - w
    x = np.arange(xl, xr + 1)
    line = t1 + (t2 - t1) * (x - xl) / (xr - xl)
    assert np.max(np.abs(r[xl:xr + 1] - line)) < 0.01 * abs(t1 - t2)
    # and one more step changes nothing (steady)
    r2 = O.to_real(m, O.run_framed(m, phi, 3000, 1, w, t1, t2))
    assert np.max(np.abs(r2 - r)) < 1e-6


def test_one_site_baths_leave_the_artifact():
    # with the baths on single sites (the paper's first callback) the periodic
    # jump between them dominates: far from the straight line
    n, t1, t2, dt = 64, 10.0, 0.0, 0.5
    m = _diffusion(n, dt)
    r = O.to_real(m, O.run_framed(m, O.to_spectrum(m, np.full(n, 5.0)), 0, 3000, 1, t1, t2))
    line = t1 + (t2 - t1) * np.arange(n) / (n - 1)
    assert np.max(np.abs(r - line)) > 0.2 * abs(t1 - t2)
