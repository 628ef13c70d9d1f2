"""Boundary frames (section "Callback functions") and the real-space round
trip of the state on the GPU, against the oracle's framed run."""
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


def _diffusion_gpu(n, dt, prec):
    P = pss()
    s = P.System((n,), dt=dt, seed=1, precision=prec)
    f = s.add_field("T")
    s.add_term(f, True, [(-1, 1.0, 1)], [(f, 1)])     # O(q) = q^2: dt T = d_x^2 T
    return s


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_heat_bath(prec, tol):
    n, w, t1, t2, dt, steps = 256, 10, 10.0, 0.0, 0.5, 300
    m = O.Model(shape=(n,), dt=dt, lhs=[(1.0, 1)], rhs=[], power=0, noisy=False)
    ref = O.run_framed(m, O.to_spectrum(m, np.full(n, 5.0)), 0, steps, w, t1, t2)
    s = _diffusion_gpu(n, dt, prec)
    s.set_field(0, np.full(n, 5.0))
    s.set_frame(0, w, t1, t2)
    s.step(steps)
    check_spectrum(s.get_spectrum(0), O.half(ref), tol)
    r = s.get_field(0)
    np.testing.assert_allclose(r[:w], t1, atol=1e-9 if prec == "f64" else 1e-4)
    np.testing.assert_allclose(r[n - w:], t2, atol=1e-9 if prec == "f64" else 1e-4)


@pytest.mark.parametrize("shape,prec,tol,steps", [((64, 64), "f64", 1e-10, 30), ((256, 256), "f32", 1e-4, 20),
                                                  ((64, 128), "f32", 1e-4, 20)])
def test_model_b_with_a_frame(shape, prec, tol, steps):
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=31)
    m = O.model_b(shape, **kw)
    ref = O.run_framed(m, O.to_spectrum(m, O.init_uniform(m, -0.2, 0.2)), 0, steps, 4, 0.3, -0.3)
    s = pss().model_b(shape, precision=prec, **kw)
    s.init_uniform(0, -0.2, 0.2)
    s.set_frame(0, 4, 0.3, -0.3)
    s.step(steps)
    check_spectrum(s.get_spectrum(0), O.half(ref), tol)


def test_3d_pair_with_a_frame_on_one_field():
    shape, steps = (8, 16, 32), 12
    P = pss()
    s = P.System(shape, dt=0.005, seed=21, precision="f64")
    P.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
    P.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi")
    s.init_uniform(0, -0.05, 0.05)
    s.init_uniform(1, -0.05, 0.05)
    s.set_frame(1, 3, 0.1, -0.2)
    s.step(steps)
    ma = O.model_a(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=21, field_id=0)
    mb = O.model_b(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=21, field_id=1)
    refs = [O.run(ma, O.to_spectrum(ma, O.init_uniform(ma, -0.05, 0.05)), 0, steps),
            O.run_framed(mb, O.to_spectrum(mb, O.init_uniform(mb, -0.05, 0.05)), 0, steps, 3, 0.1, -0.2)]
    for fid in (0, 1):
        check_spectrum(s.get_spectrum(fid), O.half(refs[fid]), 1e-10, what=str(fid))


@pytest.mark.parametrize("shape,prec,tol", [((128, 128), "f64", 1e-12), ((256, 256), "f32", 1e-5),
                                            ((16, 16, 32), "f64", 1e-12), ((512,), "f64", 1e-12)])
def test_real_space_round_trip_changes_only_rounding(shape, prec, tol):
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=5)
    runs = []
    for rt in (0, 1):
        s = pss().model_b(shape, precision=prec, **kw)
        s.set_tuning("real_state", rt)
        s.init_uniform(0, -0.1, 0.1)
        s.step(40)
        runs.append(s.get_spectrum(0))
    assert rel(runs[1], runs[0]) < tol


def test_batched_instances_each_take_the_frame():
    P = pss()
    shape, seeds = (64, 64), [7, 8]
    s = P.System(shape, dt=0.01, batch=2, seeds=seeds, precision="f64")
    P.add_model_b_field(s, a=-1.0, b=1.0, K=1.0, D=0.05)
    for i in range(2):
        s.select_instance(i)
        s.init_uniform(0, -0.1, 0.1)
    s.set_frame(0, 2, 0.25, -0.25)
    s.step(10)
    for i in range(2):
        m = O.model_b(shape, dt=0.01, a=-1.0, b=1.0, K=1.0, D=0.05, seed=seeds[i])
        ref = O.run_framed(m, O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1)), 0, 10, 2, 0.25, -0.25)
        s.select_instance(i)
        check_spectrum(s.get_spectrum(0), O.half(ref), 1e-10, what=str(i))


def test_launches_per_framed_step_and_graph_bookkeeping():
    # one slot of a 2D generic-path system: step (2) + full inverse (2) + frame
    # (1) + forward (2) + the next product (2); 40 steps = two 16-step graphs
    # and 8 steps launched one by one
    s = pss().model_b((64, 64), precision="f64", dt=0.01, seed=3)
    s.init_uniform(0, -0.1, 0.1)
    s.set_frame(0, 3, 0.0, 0.0)
    s.step(1)
    l0 = s.launch_count
    s.step(40)
    assert s.launch_count - l0 == 40 * 9


def test_frame_arguments_and_the_adjoint():
    P = pss()
    s = P.model_b((32, 32), precision="f64", dt=0.01, seed=3)
    for bad in (-1, 17):
        with pytest.raises(P.PssError) as ei:
            s.set_frame(0, bad, 0.0, 0.0)
        assert ei.value.code == P.PSS_EINVAL
    with pytest.raises(P.PssError) as ei:
        s.set_frame(0, 2, float("nan"), 0.0)
    assert ei.value.code == P.PSS_EINVAL
    s.set_frame(0, 16, 1.0, -1.0)       # the whole lattice is frame: allowed
    s.set_frame(0, 2, 1.0, -1.0)
    with pytest.raises(P.PssError) as ei:
        s.adjoint_forward(4)
    assert ei.value.code == P.PSS_EUNSUPPORTED
    s.set_frame(0, 0, 0.0, 0.0)         # removed: the adjoint runs again
    s.init_uniform(0, -0.1, 0.1)
    s.adjoint_forward(4)
