"""The KPZ workload (section "Writing models": lambda (grad phi)^2 written as
lambda psi^2 with psi = grad phi) on the GPU against the oracle."""
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


KW = dict(dt=0.02, sigma=1.0, lam=0.6, D=0.02)


def _oracle(shape, steps, seed, field_id=0, order=2, **kw):
    m = O.kpz(shape, seed=seed, field_id=field_id, dealias_order=order, **{**KW, **kw})
    return m, O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.5, 0.5)), 0, steps)


@pytest.mark.parametrize("shape,prec,tol,steps", [
    ((256,), "f64", 1e-10, 60), ((64, 64), "f64", 1e-10, 40), ((8, 16, 32), "f64", 1e-10, 20),
    ((128, 256), "f32", 1e-4, 40), ((256, 256), "f32", 1e-4, 30), ((16, 16, 64), "f32", 1e-4, 20),
])
def test_kpz_matches_oracle(shape, prec, tol, steps):
    s = pss().kpz(shape, seed=41, precision=prec, **KW)
    square_fp32 = prec == "f32" and len(shape) == 2 and shape[0] == shape[1] and shape[0] >= 256
    assert s.step_path == ("persist2d" if square_fp32 else "generic")
    s.init_uniform(0, -0.5, 0.5)
    s.step(steps)
    _, ref = _oracle(shape, steps, 41)
    check_spectrum(s.get_spectrum(0), O.half(ref), tol)


def test_kpz_order_zero_and_three():
    for order in (0, 3):
        s = pss().kpz((64, 64), seed=9, precision="f64", dealias_order=order, **KW)
        s.init_uniform(0, -0.5, 0.5)
        s.step(25)
        _, ref = _oracle((64, 64), 25, 9, order=order)
        check_spectrum(s.get_spectrum(0), O.half(ref), 1e-10, what=str(order))


def test_kpz_beside_a_model_b_field():
    # field 0 takes the gradient product, field 1 the power product of the fused kernels
    P = pss()
    shape, steps = (64, 64), 30
    s = P.System(shape, dt=0.02, seed=13, precision="f64")
    P.add_kpz_field(s, sigma=1.0, lam=0.6, D=0.02, name="h")
    P.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi")
    s.init_uniform(0, -0.5, 0.5)
    s.init_uniform(1, -0.1, 0.1)
    s.step(steps)
    _, ref_h = _oracle(shape, steps, 13, field_id=0)
    mb = O.model_b(shape, dt=0.02, a=-1, b=1, K=1, D=0.05, seed=13, field_id=1)
    ref_b = O.run(mb, O.to_spectrum(mb, O.init_uniform(mb, -0.1, 0.1)), 0, steps)
    check_spectrum(s.get_spectrum(0), O.half(ref_h), 1e-10)
    check_spectrum(s.get_spectrum(1), O.half(ref_b), 1e-10)


def test_kpz_batched_instances():
    P = pss()
    shape, seeds = (64, 64), [3, 4, 5]
    s = P.System(shape, dt=0.02, batch=3, seeds=seeds, precision="f64")
    P.add_kpz_field(s, **{k: v for k, v in KW.items() if k != "dt"})
    for i in range(3):
        s.select_instance(i)
        s.init_uniform(0, -0.5, 0.5)
    s.step(20)
    for i in range(3):
        _, ref = _oracle(shape, 20, seeds[i])
        s.select_instance(i)
        check_spectrum(s.get_spectrum(0), O.half(ref), 1e-10, what=str(i))


def test_kpz_with_a_frame():
    n, steps = 128, 40
    s = pss().kpz((n,), seed=2, precision="f64", **KW)
    s.init_uniform(0, -0.5, 0.5)
    s.set_frame(0, 5, 1.0, -1.0)
    s.step(steps)
    m = O.kpz((n,), seed=2, **KW)
    ref = O.run_framed(m, O.to_spectrum(m, O.init_uniform(m, -0.5, 0.5)), 0, steps, 5, 1.0, -1.0)
    check_spectrum(s.get_spectrum(0), O.half(ref), 1e-10)


def test_kpz_launches_and_limits():
    P = pss()
    s = P.kpz((64, 64), seed=1, precision="f64", **KW)
    s.init_uniform(0, -0.5, 0.5)
    s.step(1)
    l0 = s.launch_count
    s.step(40)
    # column + row kernels (2), then per axis the column inverse of i q_j m h
    # and the row inverse that adds its square (2 x 2), and the row transform
    # of the sum (1)
    assert s.launch_count - l0 == 40 * 7
    with pytest.raises(P.PssError) as ei:
        s.adjoint_forward(4)
    assert ei.value.code == P.PSS_EUNSUPPORTED



def test_kpz_with_a_cubic_term():
    # a power product beside the gradient square: both go through real space,
    # in two operator groups
    shape, steps = (64, 64), 25
    s = pss().kpz(shape, seed=8, precision="f64", **KW)
    s.add_term(0, False, [(-1, -0.3, 0)], [(0, 3)])
    s.init_uniform(0, -0.5, 0.5)
    s.step(steps)
    m = O.kpz(shape, seed=8, **KW)
    terms = [O.Term(0, [(KW["lam"], 0)], [O.Factor(0, 2, deriv=j)]) for j in (0, 1)]
    terms.append(O.Term(0, [(-0.3, 0)], [O.Factor(0, 3)]))
    ref = O.run_coupled([m], terms, [O.to_spectrum(m, O.init_uniform(m, -0.5, 0.5))], 0, steps)[0]
    check_spectrum(s.get_spectrum(0), O.half(ref), 1e-10)
