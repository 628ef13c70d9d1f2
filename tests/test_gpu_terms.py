"""General product terms (Eq. basefourier; section "Writing models") on the
GPU against the oracle's coupled-field step: cross-field products, derivative
and Laplacian factors, several operators per field, batched parameters."""
import math

import numpy as np
import pytest

from oracle import oracle as O

from tests.parity import check_spectrum  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2405_02410_gb300 import build
    build.build()


def pss():
    from paper_2405_02410_gb300 import pss as m
    return m


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


# A conserved field phi and a non-conserved field psi, coupled (a Model C-like pair):
#   dt phi + (a q^2 + K q^4) phi = -b q^2 F[phi^3] - g q^2 F[phi psi^2]   (two operators)
#   dt psi + (c + L q^2) psi     = -h F[phi^2 psi]                          (one operator)
P0 = dict(a=-1.0, K=1.0, b=1.0, g=0.5, c=0.3, L=1.0, h=0.7, D0=0.02, D1=0.05)


def _pair_gpu(shape, prec, dt, seed, batch=1, seeds=None, p=P0):
    P = pss()
    s = P.System(shape, dt=dt, seed=seed, precision=prec, batch=batch, seeds=seeds)
    f0, f1 = s.add_field("phi"), s.add_field("psi")
    ids = {k: s.add_param(k, v) for k, v in p.items()}
    s.add_term(f0, True, [(ids["a"], 1.0, 1), (ids["K"], 1.0, 2)], [(f0, 1)])
    s.add_term(f0, False, [(ids["b"], -1.0, 1)], [(f0, 3)])
    s.add_product_term(f0, [(ids["g"], -1.0, 1)], [(f0, 1), (f1, 2)])
    s.add_term(f1, True, [(ids["c"], 1.0, 0), (ids["L"], 1.0, 1)], [(f1, 1)])
    s.add_product_term(f1, [(ids["h"], -1.0, 0)], [(f0, 2), (f1, 1)])
    s.set_noise(f0, ids["D0"], 1)
    s.set_noise(f1, ids["D1"], 0)
    return s, ids


def _pair_oracle(shape, dt, seed, p=P0):
    m0 = O.Model(shape=shape, dt=dt, lhs=[(p["a"], 1), (p["K"], 2)], noise_D=p["D0"], noise_pow=1, noisy=True,
                 seed=seed, field_id=0)
    m1 = O.Model(shape=shape, dt=dt, lhs=[(p["c"], 0), (p["L"], 1)], noise_D=p["D1"], noise_pow=0, noisy=True,
                 seed=seed, field_id=1)
    terms = [O.Term(0, [(-p["b"], 1)], [O.Factor(0, 3)]),
             O.Term(0, [(-p["g"], 1)], [O.Factor(0), O.Factor(1, 2)]),
             O.Term(1, [(-p["h"], 0)], [O.Factor(0, 2), O.Factor(1)])]
    return [m0, m1], terms


def _init_oracle(ms, lo=(-0.2, -0.2), hi=(0.2, 0.2)):
    return [O.to_spectrum(m, O.init_uniform(m, lo[i], hi[i])) for i, m in enumerate(ms)]


@pytest.mark.parametrize("shape,prec,tol,steps", [((64, 64), "f64", 1e-10, 30), ((128,), "f64", 1e-10, 40),
                                                  ((8, 16, 32), "f64", 1e-10, 15), ((128, 128), "f32", 1e-4, 30),
                                                  ((16, 16, 32), "f32", 1e-4, 15)])
def test_coupled_pair_matches_oracle(shape, prec, tol, steps):
    dt, seed = 0.01, 77
    s, _ = _pair_gpu(shape, prec, dt, seed)
    assert s.step_path in ("generic", "fast3d_rows")
    s.init_uniform(0, -0.2, 0.2)
    s.init_uniform(1, -0.2, 0.2)
    s.step(steps)
    ms, terms = _pair_oracle(shape, dt, seed)
    ref = O.run_coupled(ms, terms, _init_oracle(ms), 0, steps)
    for fid in (0, 1):
        check_spectrum(s.get_spectrum(fid), O.half(ref[fid]), tol, what=str(fid))


def test_batched_coupling_parameters():
    # per-instance operators of a two-operator field reach the combine launch
    shape, dt, seeds = (32, 32), 0.01, [5, 6]
    s, ids = _pair_gpu(shape, "f64", dt, 5, batch=2, seeds=seeds)
    s.set_param_batch(ids["g"], np.array([0.2, 0.9]))
    for i in range(2):
        s.select_instance(i)
        s.init_uniform(0, -0.2, 0.2)
        s.init_uniform(1, -0.2, 0.2)
    s.step(20)
    for i, g in enumerate((0.2, 0.9)):
        ms, terms = _pair_oracle(shape, dt, seeds[i], p={**P0, "g": g})
        ref = O.run_coupled(ms, terms, _init_oracle(ms), 0, 20)
        s.select_instance(i)
        for fid in (0, 1):
            check_spectrum(s.get_spectrum(fid), O.half(ref[fid]), 1e-10, what=str((i, fid)))


def test_changing_a_coupling_between_runs():
    shape, dt = (32, 32), 0.01
    s, ids = _pair_gpu(shape, "f64", dt, 9)
    s.init_uniform(0, -0.2, 0.2)
    s.init_uniform(1, -0.2, 0.2)
    s.step(17)                          # one captured graph and a tail
    s.set_param(ids["g"], 1.4)
    s.set_param(ids["h"], 0.1)
    s.step(17)
    ms, terms = _pair_oracle(shape, dt, 9)
    mid = O.run_coupled(ms, terms, _init_oracle(ms), 0, 17)
    ms2, terms2 = _pair_oracle(shape, dt, 9, p={**P0, "g": 1.4, "h": 0.1})
    ref = O.run_coupled(ms2, terms2, mid, 17, 17)
    for fid in (0, 1):
        check_spectrum(s.get_spectrum(fid), O.half(ref[fid]), 1e-10, what=str(fid))


def test_linear_coupling_rotates_uniform_fields():
    shape, dt, c, n = (16, 16), 0.05, 1.3, 40
    P = pss()
    s = P.System(shape, dt=dt, seed=1, precision="f64")
    f0, f1 = s.add_field("u"), s.add_field("v")
    s.add_product_term(f0, [(-1, -c, 0)], [(f1, 1)])
    s.add_product_term(f1, [(-1, c, 0)], [(f0, 1)])
    u0, v0 = 0.4, -0.1
    s.set_field(0, np.full(shape, u0))
    s.set_field(1, np.full(shape, v0))
    s.step(n)
    g, th = (1 + dt * dt * c * c) ** (n / 2), n * math.atan(dt * c)
    u = g * (u0 * math.cos(th) - v0 * math.sin(th))
    v = g * (u0 * math.sin(th) + v0 * math.cos(th))
    np.testing.assert_allclose(s.get_field(0), u, atol=1e-12)
    np.testing.assert_allclose(s.get_field(1), v, atol=1e-12)


@pytest.mark.parametrize("shape,prec,tol", [((256,), "f64", 1e-10), ((64, 64), "f64", 1e-10), ((128, 128), "f32", 1e-4)])
def test_burgers_and_a_laplacian_factor(shape, prec, tol):
    # dt u = nu lap u - u d_x u + 0.1 u lap u: derivative and Laplacian factors;
    # the two terms have different operators (two groups, summed in Fourier space)
    dt, seed, steps, nu = 0.01, 3, 30, 0.5
    P = pss()
    s = P.System(shape, dt=dt, seed=seed, precision=prec)
    f = s.add_field("u")
    s.add_term(f, True, [(-1, nu, 1)], [(f, 1)])
    s.add_product_term(f, [(-1, -1.0, 0)], [(f, 1), (f, 1, 0)])
    s.add_product_term(f, [(-1, 0.1, 0)], [(f, 1, -1, 0), (f, 1, -1, 1)])
    s.init_uniform(0, -0.5, 0.5)
    s.step(steps)
    m = O.Model(shape=shape, dt=dt, lhs=[(nu, 1)], seed=seed)
    terms = [O.Term(0, [(-1.0, 0)], [O.Factor(0), O.Factor(0, deriv=0)]),
             O.Term(0, [(0.1, 0)], [O.Factor(0), O.Factor(0, lap=1)])]
    ref = O.run_coupled([m], terms, [O.to_spectrum(m, O.init_uniform(m, -0.5, 0.5))], 0, steps)[0]
    check_spectrum(s.get_spectrum(0), O.half(ref), tol)


def test_product_terms_with_a_frame_and_argument_checks():
    P = pss()
    shape, dt = (64,), 0.01
    s, ids = _pair_gpu(shape, "f64", dt, 4)
    s.init_uniform(0, -0.2, 0.2)
    s.init_uniform(1, -0.2, 0.2)
    s.set_frame(1, 3, 0.2, -0.2)
    s.step(12)
    ms, terms = _pair_oracle(shape, dt, 4)
    phis = _init_oracle(ms)
    for k in range(12):
        phis = O.run_coupled(ms, terms, phis, k, 1)
        r = O.to_real(ms[1], phis[1])
        r[:3], r[-3:] = 0.2, -0.2
        phis[1] = O.to_spectrum(ms[1], r)
    for fid in (0, 1):
        check_spectrum(s.get_spectrum(fid), O.half(phis[fid]), 1e-10, what=str(fid))
    for bad in ([(5, 1)], [(0, 0)], [(0, 1, 3)], [(0, 1, -1, 3)]):
        with pytest.raises(P.PssError) as ei:
            s.add_product_term(0, [(-1, 1.0, 0)], bad)
        assert ei.value.code == P.PSS_EINVAL
    with pytest.raises(P.PssError) as ei:
        s.adjoint_forward(3)
    assert ei.value.code == P.PSS_EUNSUPPORTED
