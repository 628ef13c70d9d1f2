"""The persistent FP32 2D step (k2p_step: a run of steps in one cooperative
launch, grid barriers between the column and row phases) against the FP64
oracle and against the two-kernel step it replaces.

The persistent step performs the same arithmetic as k2_col / k2_row, so at
the same FFT radix the two give the same bits, whatever the step count per
launch, the number of CTAs, or how runs alternate between the paths.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests.parity import check_spectrum

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


def _model_b(shape, knobs=None, **kw):
    s = pss().model_b(shape, precision="f32", **kw)
    for k, v in (knobs or {}).items():
        s.set_tuning(k, v)
    s.init_uniform(0, -0.1, 0.1)
    return s


def _oracle_b(shape, steps, **kw):
    m = O.model_b(shape, **kw)
    return O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1)), 0, steps))


@pytest.mark.parametrize("shape,order,noisy,steps", [
    ((256, 256), 2, True, 100), ((512, 512), 2, True, 40), ((256, 256), 3, True, 60),
    ((256, 256), 0, True, 60), ((512, 512), 2, False, 30), ((1024, 1024), 3, True, 20),
])
def test_matches_oracle(shape, order, noisy, steps):
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=17, dealias_order=order, noisy=noisy)
    s = _model_b(shape, **kw)
    assert s.step_path == "persist2d"
    s.step(steps)
    check_spectrum(s.get_spectrum(0), _oracle_b(shape, steps, **kw), 1e-4, order=order)


@pytest.mark.parametrize("radix", [8, 16])
@pytest.mark.parametrize("shape,order,noisy", [
    ((256, 256), 2, True), ((512, 512), 3, True), ((1024, 1024), 2, True), ((1024, 1024), 0, False),
])
def test_same_bits_as_the_two_kernel_step(shape, order, noisy, radix):
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=29, dealias_order=order, noisy=noisy)
    knobs = dict(col2_radix=radix, row2_radix=radix)
    p = _model_b(shape, knobs=knobs, **kw)
    q = _model_b(shape, knobs=dict(knobs, persist=0), **kw)
    assert p.step_path == "persist2d" and q.step_path == "fast2d"
    for n in (1, 6, 33):
        p.step(n)
        q.step(n)
        assert p.get_spectrum(0).tobytes() == q.get_spectrum(0).tobytes(), n
    assert p.get_step() == q.get_step() == 40


@pytest.mark.parametrize("blocks", [129, 140, 151])
def test_number_of_ctas_changes_no_bit(blocks):
    # the columns and rows cut into other contiguous blocks (at most 2 column
    # pairs and 4 row pairs per CTA: at least 129 CTAs at 1024^2)
    shape = (1024, 1024)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.01, seed=2405)
    ref = _model_b(shape, **kw)
    s = _model_b(shape, knobs=dict(persist_blocks=blocks), **kw)
    ref.step(12)
    s.step(12)
    assert s.get_spectrum(0).tobytes() == ref.get_spectrum(0).tobytes()


def test_paths_alternate_mid_run():
    # persistent runs, two-kernel runs and generic-kernel runs in turn: the work
    # arrays and the drawn-ahead noise stay consistent across the switches
    shape = (256, 256)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=5)
    s = _model_b(shape, **kw)
    ref = _model_b(shape, knobs=dict(persist=0), **kw)
    for persist in (1, 0, 1, 0, 1):
        s.set_tuning("persist", persist)
        s.step(9)
        ref.step(9)
    assert s.get_spectrum(0).tobytes() == ref.get_spectrum(0).tobytes()
    s.set_tuning("fast2d", 0)
    s.step(10)
    s.set_tuning("fast2d", 1)
    s.step(11)
    check_spectrum(s.get_spectrum(0), _oracle_b(shape, 66, **kw), 1e-4)


def test_mass_is_conserved_bitwise():
    s = _model_b((1024, 1024), dt=0.01, a=-1, b=1, K=1, D=0.1, seed=3)
    m0 = s.get_spectrum(0)[0, 0]
    s.step(300)
    assert s.get_spectrum(0)[0, 0] == m0


def test_parameter_change_between_runs():
    shape = (512, 512)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=8)
    s = _model_b(shape, **kw)
    s.step(10)
    s.set_param(0, -0.7)      # a
    s.set_param(3, 0.02)      # D
    s.step(10)
    m1 = O.model_b(shape, **kw)
    phi = O.run(m1, O.to_spectrum(m1, O.init_uniform(m1, -0.1, 0.1)), 0, 10)
    m2 = O.model_b(shape, **dict(kw, a=-0.7, D=0.02))
    check_spectrum(s.get_spectrum(0), O.half(O.run(m2, phi, 10, 10)), 1e-4)


def test_grid_barrier_timeout_is_reported_and_the_handle_recovers():
    # the check of the bounded waits: one CTA never arrives at the first grid
    # barrier, every wait gives up after 1024 polls, the launch records the
    # timeout and leaves; the next synchronising call reports it and clears the
    # barrier words, and the handle keeps working
    import time
    P = pss()
    shape = (256, 256)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=41)
    s = _model_b(shape, **kw)
    assert s.step_path == "persist2d"
    s.sync()
    s.set_tuning("test_timeout", 1)
    t0 = time.perf_counter()
    s.step(3)
    with pytest.raises(P.PssError) as ei:
        s.sync()
    assert ei.value.code == P.PSS_ETIMEOUT
    assert time.perf_counter() - t0 < 1.0
    s.set_tuning("test_timeout", 0)
    s.init_uniform(0, -0.1, 0.1)
    s.set_step(0)
    s.step(20)
    check_spectrum(s.get_spectrum(0), _oracle_b(shape, 20, **kw), 1e-4)


def test_launches_per_run():
    s = _model_b((1024, 1024), dt=0.01, a=-1, b=1, K=1, D=0.01, seed=1)
    s.step(1)
    n0 = s.launch_count
    s.step(1000)
    assert s.launch_count - n0 == 1


# ---------------------------------------------------------------------------
# KPZ (the gradient-square term) on the persistent step
# ---------------------------------------------------------------------------
KPZ = dict(dt=0.02, sigma=1.0, lam=0.6, D=0.02)


def _kpz(shape, knobs=None, order=2, seed=41):
    s = pss().kpz(shape, seed=seed, precision="f32", dealias_order=order, **KPZ)
    for k, v in (knobs or {}).items():
        s.set_tuning(k, v)
    s.init_uniform(0, -0.5, 0.5)
    return s


def _oracle_kpz(shape, steps, order=2, seed=41):
    m = O.kpz(shape, seed=seed, dealias_order=order, **KPZ)
    return O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.5, 0.5)), 0, steps))


@pytest.mark.parametrize("shape,order,steps", [((256, 256), 2, 40), ((512, 512), 2, 20), ((256, 256), 0, 30),
                                               ((256, 256), 3, 30), ((1024, 1024), 2, 8)])
def test_kpz_matches_oracle(shape, order, steps):
    s = _kpz(shape, order=order)
    assert s.step_path == "persist2d"
    s.step(steps)
    check_spectrum(s.get_spectrum(0), _oracle_kpz(shape, steps, order), 1e-4, order=order)


@pytest.mark.parametrize("radix", [8, 16])
def test_kpz_matches_the_generic_kernels_and_takes_one_launch(radix):
    shape = (512, 512)
    p = _kpz(shape, knobs=dict(col2_radix=radix, row2_radix=radix))
    q = _kpz(shape, knobs=dict(persist=0))
    assert q.step_path == "generic"
    p.step(3)
    q.step(3)
    n0 = p.launch_count
    p.step(30)
    assert p.launch_count - n0 == 1
    q.step(30)
    check_spectrum(p.get_spectrum(0), q.get_spectrum(0), 1e-5)
    # switching between the paths mid-run recomputes the product in each layout
    p.set_tuning("persist", 0)
    p.step(5)
    p.set_tuning("persist", 1)
    p.step(5)
    q.step(10)
    check_spectrum(p.get_spectrum(0), q.get_spectrum(0), 1e-5)


def test_kpz_parameter_change_and_resume():
    shape = (256, 256)
    s = _kpz(shape)
    s.step(10)
    blob = s.save_state()
    s.set_param(1, 0.3)        # lambda (parameters: sigma, lambda, D)
    s.step(10)
    m1 = O.kpz(shape, seed=41, **KPZ)
    phi = O.run(m1, O.to_spectrum(m1, O.init_uniform(m1, -0.5, 0.5)), 0, 10)
    m2 = O.kpz(shape, seed=41, **dict(KPZ, lam=0.3))
    check_spectrum(s.get_spectrum(0), O.half(O.run(m2, phi, 10, 10)), 1e-4)
    r = _kpz(shape, seed=99)
    r.load_state(blob)
    r.set_param(1, 0.3)
    r.step(10)
    assert r.get_spectrum(0).tobytes() == s.get_spectrum(0).tobytes()
