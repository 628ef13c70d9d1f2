"""Pins of the oracle's adjoint (orc_adjoint) by central finite differences of
the oracle's own forward map, in FP64: the gradient with respect to the
initial field along random Hermitian directions, and with respect to every
operator coefficient and the noise strength."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def _setup(shape, order, seed=3):
    m = O.model_b(shape, dt=0.02, a=-1.0, b=1.0, K=1.0, D=0.05, seed=seed, dealias_order=order)
    phi0 = O.to_spectrum(m, O.init_uniform(m, -0.4, 0.4))
    return m, phi0


def _quad_loss(m, phi, c):
    # J = sum_q c_q |phi_q|^2 / N with c even in q: dJ/dphi = 2 c phi / N
    return float(np.sum(c * np.abs(phi) ** 2) / m.n_sites), 2.0 * c * phi / m.n_sites


def _weights(shape, seed):
    # a smooth positive weight that depends on |k| only (even under q -> -q)
    k = np.meshgrid(*[np.fft.fftfreq(n) * n for n in shape], indexing="ij")
    kk = np.sqrt(sum(x ** 2 for x in k))
    r = inputs.rng(seed).uniform(0.5, 1.5, size=8)
    return r[0] + r[1] * np.cos(0.3 * kk * r[2]) ** 2


def _inner(a, b):
    return float(np.real(np.vdot(a, b)))


@pytest.mark.parametrize("shape,order", [((16,), 2), ((8, 8), 2), ((8, 12), 3), ((4, 4, 8), 2)])
def test_adjoint_initial_field_matches_finite_differences(shape, order):
    m, phi0 = _setup(shape, order)
    nsteps = 12
    c = _weights(shape, 5)
    J0, lamT = _quad_loss(m, O.run(m, phi0, 0, nsteps), c)
    lam0, _ = O.adjoint(m, phi0, 0, nsteps, lamT)
    for trial in range(3):
        d = O.to_spectrum(m, inputs.real_field(shape, seed=40 + trial))
        h = 1e-4
        Jp, _ = _quad_loss(m, O.run(m, phi0 + h * d, 0, nsteps), c)
        Jm, _ = _quad_loss(m, O.run(m, phi0 - h * d, 0, nsteps), c)
        fd = (Jp - Jm) / (2 * h)
        assert abs(_inner(lam0, d) - fd) <= 1e-6 * max(abs(fd), 1e-12), (_inner(lam0, d), fd)


def _with(m, **kw):
    p = dict(a=-1.0, b=1.0, K=1.0, D=0.05)
    p.update(kw)
    return O.model_b(m.shape, dt=m.dt, seed=m.seed, dealias_order=m.dealias_order, **p)


@pytest.mark.parametrize("shape", [(16,), (8, 8)])
def test_adjoint_coefficients_match_finite_differences(shape):
    m, phi0 = _setup(shape, 2)
    nsteps = 10
    c = _weights(shape, 7)
    _, lamT = _quad_loss(m, O.run(m, phi0, 0, nsteps), c)
    _, g = O.adjoint(m, phi0, 0, nsteps, lamT)
    # Model B: O = a q^2 + K q^4, M = -b q^2, D~ = D q^2
    analytic = {"a": g[1], "K": g[2], "b": -g[6], "D": g[10]}
    base = dict(a=-1.0, b=1.0, K=1.0, D=0.05)
    for name, val in analytic.items():
        h = 1e-5
        Jp, _ = _quad_loss(m, O.run(_with(m, **{name: base[name] + h}), phi0, 0, nsteps), c)
        Jm, _ = _quad_loss(m, O.run(_with(m, **{name: base[name] - h}), phi0, 0, nsteps), c)
        fd = (Jp - Jm) / (2 * h)
        assert abs(val - fd) <= 1e-6 * max(abs(fd), 1e-10), (name, val, fd)


def test_adjoint_of_binned_structure_factor_loss():
    shape = (16, 16)
    m, phi0 = _setup(shape, 2)
    nsteps = 8
    target = np.linspace(0.5, 2.0, 16) * 1e-2
    bins = O.sq_bin_index(m, 16)

    def loss(phi):
        J, coef = O.binned_sq_loss(m, phi, target, 16)
        lam = np.where(bins >= 0, coef[np.clip(bins, 0, None)], 0.0) * phi
        return J, lam

    J0, lamT = loss(O.run(m, phi0, 0, nsteps))
    lam0, g = O.adjoint(m, phi0, 0, nsteps, lamT)
    d = O.to_spectrum(m, inputs.real_field(shape, seed=77))
    h = 1e-4
    fd = (loss(O.run(m, phi0 + h * d, 0, nsteps))[0] - loss(O.run(m, phi0 - h * d, 0, nsteps))[0]) / (2 * h)
    assert abs(_inner(lam0, d) - fd) <= 1e-6 * abs(fd)
    hb = 1e-5
    fdb = (loss(O.run(_with(m, b=1.0 + hb), phi0, 0, nsteps))[0]
           - loss(O.run(_with(m, b=1.0 - hb), phi0, 0, nsteps))[0]) / (2 * hb)
    assert abs(-g[6] - fdb) <= 1e-6 * abs(fdb)


def test_bin_index_matches_structure_factor_counts():
    m = O.Model(shape=(32, 16), dt=1.0)
    b = O.sq_bin_index(m, 24)
    _, cnt, _ = O.structure_factor(m, np.ones((32, 16), dtype=complex), 24)
    np.testing.assert_array_equal(np.bincount(b[b >= 0], minlength=24), cnt)
