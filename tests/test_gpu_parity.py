"""Parity of the sm_103a path (through the C ABI) with the FP64 CPU oracle.

Bars: FP32 rel-L2 <= 1e-4 and FP64 rel-L2 <= 1e-10 over <= 200 steps (sizes the
oracle finishes in seconds, spanning several tiles and a ragged last tile),
bit-identical results for replays, resumes and graph vs. eager launches.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs
from tests.parity import check_real, check_spectrum, rel

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2405_02410_gb300 import build
    build.build()


def pss():
    from paper_2405_02410_gb300 import pss as m
    return m


SHAPES = [(4,), (64,), (1024,), (4, 4), (8, 16), (64, 64), (32, 128), (128, 32), (4, 8, 4), (8, 16, 32), (16, 16, 16)]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("shape", SHAPES)
def test_transform_roundtrip_and_spectrum(shape, prec):
    s = pss().System(shape, dt=0.1, precision=prec)
    f = s.add_field("phi")
    x = inputs.real_field(shape, seed=101)
    s.set_field(f, x)
    spec = s.get_spectrum(f)
    ref = np.fft.rfftn(x)
    check_spectrum(spec, ref, 2e-6 if prec == "f32" else 1e-13, order=0)
    back = s.get_field(f)
    check_real(back, x, 2e-6 if prec == "f32" else 1e-13)


@pytest.mark.parametrize("shape", [(64, 64), (8, 8, 8), (64,)])
def test_init_uniform_matches_oracle(shape):
    s = pss().System(shape, dt=0.1, seed=77, precision="f64")
    f = s.add_field("phi")
    s.init_uniform(f, -0.1, 0.3)
    m = O.Model(shape=shape, dt=0.1, seed=77)
    assert rel(s.get_field(f), O.init_uniform(m, -0.1, 0.3)) < 1e-13


def _oracle_b(shape, steps, **kw):
    m = O.model_b(shape, **kw)
    phi = O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1))
    return O.half(O.run(m, phi, 0, steps))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_model_b_64x64_100_steps(prec):
    # the 64 x 64 Model B parity workload: a=-1, b=1, K=1, D=0.01, dt=0.01, 2/3 rule
    shape, steps = (64, 64), 100
    s = pss().model_b(shape, dt=0.01, a=-1, b=1, K=1, D=0.01, seed=2405, precision=prec)
    s.init_uniform(0, -0.1, 0.1)
    s.step(steps)
    ref = _oracle_b(shape, steps, dt=0.01, a=-1, b=1, K=1, D=0.01, seed=2405)
    check_spectrum(s.get_spectrum(0), ref, TOL[prec])
    check_real(s.get_field(0), np.fft.irfftn(ref, s=shape), TOL[prec] * 10)


def _full_from_half(half, shape):
    """Hermitian completion of a half spectrum (numpy helper, no method arithmetic)."""
    return np.fft.fftn(np.fft.irfftn(half, s=shape))


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("shape,order,noisy", [
    ((64,), 2, True), ((256,), 3, True), ((8, 16), 2, True), ((32, 128), 0, True), ((128, 32), 3, False),
    ((4, 4), 2, True), ((8, 8, 8), 2, True), ((8, 16, 32), 3, True), ((16, 16, 16), 0, False),
])
def test_model_b_shapes_and_dealias_orders(shape, order, noisy, prec):
    steps = 50
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=11, dealias_order=order, noisy=noisy)
    s = pss().model_b(shape, precision=prec, **kw)
    s.init_uniform(0, -0.1, 0.1)
    s.step(steps)
    ref = _oracle_b(shape, steps, **kw)
    check_spectrum(s.get_spectrum(0), ref, TOL[prec], order=order)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_model_a_and_b_pair_3d(prec):
    # two uncoupled fields in one system (Model A field 0, Model B field 1), sharing the seed
    shape, steps = (8, 16, 16), 40
    P = pss()
    s = P.System(shape, dt=0.005, seed=5, precision=prec)
    P.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
    P.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi")
    s.init_uniform(0, -0.05, 0.05)
    s.init_uniform(1, -0.05, 0.05)
    s.step(steps)
    ma = O.model_a(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=5, field_id=0)
    mb = O.model_b(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=5, field_id=1)
    for fid, m in ((0, ma), (1, mb)):
        ref = O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.05, 0.05)), 0, steps))
        check_spectrum(s.get_spectrum(fid), ref, TOL[prec], what=f"field {fid}")


def test_noise_only_linear_model_every_step():
    # b = 0: phi' = (phi + xi) / (1 + dt O); checks the noise of every mode, step by step
    shape = (16, 32)
    P = pss()
    s = P.System(shape, dt=0.1, seed=9, precision="f64")
    f = s.add_field("phi")
    pa, pD = s.add_param("a", 0.5), s.add_param("D", 0.3)
    s.add_term(f, True, [(pa, 1.0, 0), (-1, 1.0, 1)], [(f, 1)])
    s.set_noise(f, pD, 0)
    m = O.Model(shape=shape, dt=0.1, lhs=[(0.5, 0), (1.0, 1)], noise_D=0.3, noise_pow=0, noisy=True, seed=9)
    phi = np.zeros(shape, dtype=complex)
    for k in range(3):
        s.step(1)
        phi = O.run(m, phi, k, 1)
        check_spectrum(s.get_spectrum(f), O.half(phi), 1e-12, what=f"step {k}")


def test_mass_is_conserved_bitwise_in_the_spectrum():
    s = pss().model_b((64, 64), D=0.1, seed=3, precision="f32")
    s.init_uniform(0, -0.2, 0.4)
    m0 = s.get_spectrum(0)[0, 0]
    s.step(200)
    assert s.get_spectrum(0)[0, 0] == m0


def test_graph_replay_resume_and_determinism():
    P = pss()

    def run(chunks):
        s = P.model_b((64, 64), D=0.05, seed=21, precision="f32")
        s.init_uniform(0, -0.1, 0.1)
        for c in chunks:
            s.step(c)
        return s.get_spectrum(0), s.get_step()

    a, na = run([40])          # 2 graphs of 16 steps + one graph of 8
    b, nb = run([1] * 40)      # 40 replays of the one-step graph
    c, nc = run([17, 3, 20])
    assert na == nb == nc == 40
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)


def test_structure_factor_matches_oracle():
    shape, steps = (64, 64), 60
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=13)
    s = pss().model_b(shape, precision="f64", **kw)
    s.init_uniform(0, -0.1, 0.1)
    s.step(steps)
    S, cnt, L = s.structure_factor(0, 64)
    m = O.model_b(shape, **kw)
    full = O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1)), 0, steps)
    So, co, Lo = O.structure_factor(m, full, 64)
    np.testing.assert_array_equal(cnt, co)
    assert rel(S, So) < 1e-10 and abs(L - Lo) < 1e-10 * Lo


def test_structure_factor_many_bins():
    # 4096 bins need more than 48 KB of shared memory per block
    shape = (256, 256)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=21)
    s = pss().model_b(shape, precision="f64", **kw)
    s.init_uniform(0, -0.1, 0.1)
    s.step(3)
    S, cnt, L = s.structure_factor(0, 4096)
    m = O.model_b(shape, **kw)
    full = O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1)), 0, 3)
    So, co, Lo = O.structure_factor(m, full, 4096)
    np.testing.assert_array_equal(cnt, co)
    assert rel(S, So) < 1e-10 and abs(L - Lo) < 1e-10 * Lo


def test_set_spectrum_roundtrip_and_param_change():
    P = pss()
    s = P.model_b((32, 32), D=0.0, noisy=False, seed=1, precision="f64")
    half = np.fft.rfftn(inputs.real_field((32, 32), seed=5, lo=-0.2, hi=0.2))
    s.set_spectrum(0, half)
    assert rel(s.get_spectrum(0), half) == 0
    s.set_param(0, -0.5)   # a
    s.step(20)
    m = O.model_b((32, 32), a=-0.5, D=0.0, noisy=False)
    ref = O.half(O.run(m, _full_from_half(half, (32, 32)), 0, 20))
    check_spectrum(s.get_spectrum(0), ref, 1e-10)


def test_nonfinite_is_reported():
    P = pss()
    s = P.model_b((16, 16), noisy=False, precision="f32")
    x = np.zeros((16, 16))
    x[3, 4] = np.inf
    s.set_field(0, x)
    s.step(2)
    with pytest.raises(P.PssError) as ei:
        s.sync()
    assert ei.value.code == P.PSS_ENONFINITE


def test_bounded_wait_timeout_is_reported_and_the_handle_recovers():
    # the check of the bounded waits: the first CTA of the column kernel expects
    # 16 bytes more than its bulk copies deliver (every copy is issued and lands)
    # and gives up after 1024 polls; the kernel records the timeout and returns,
    # and the next synchronising call reports it
    import time
    P = pss()
    shape, steps = (64, 64), 20
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.01, seed=2405)
    s = P.model_b(shape, precision="f32", **kw)
    assert s.step_path == "generic"
    s.init_uniform(0, -0.1, 0.1)
    s.sync()
    s.set_tuning("test_timeout", 1)
    t0 = time.perf_counter()
    s.step(1)
    with pytest.raises(P.PssError) as ei:
        s.sync()
    assert ei.value.code == P.PSS_ETIMEOUT
    assert time.perf_counter() - t0 < 1.0
    # the status is cleared, the handle keeps working
    s.set_tuning("test_timeout", 0)
    s.sync()
    s.init_uniform(0, -0.1, 0.1)
    s.set_step(0)
    s.step(steps)
    check_spectrum(s.get_spectrum(0), _oracle_b(shape, steps, **kw), 1e-4)


def test_model_b_1024_against_oracle_100_steps():
    # the 1024 x 1024 workload in its timed launch configuration, 100 steps, every
    # mode checked (the oracle's radix-2 transforms take about 0.25 s a step)
    shape, steps = (1024, 1024), 100
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.01, seed=2405)
    s = pss().model_b(shape, precision="f32", **kw)
    s.init_uniform(0, -0.1, 0.1)
    s.step(steps)
    ref = _oracle_b(shape, steps, **kw)
    check_spectrum(s.get_spectrum(0), ref, 1e-4)


def _oracle_3d_field(args):
    # one field of the 256^3 pair on the oracle, in a spawned process
    fid, steps = args
    from oracle import oracle as Om
    kw = dict(dt=0.005, a=-1, b=1, K=1, D=0.05, seed=2405, field_id=fid)
    m = Om.model_a((256, 256, 256), **kw) if fid == 0 else Om.model_b((256, 256, 256), **kw)
    return Om.half(Om.run(m, Om.to_spectrum(m, Om.init_uniform(m, -0.05, 0.05)), 0, steps))


def test_model_ab_256cubed_against_oracle():
    # the 256^3 Model A + B pair in its timed launch configuration (FFT-group x
    # pass), ten steps, every mode of both fields checked; the two oracle fields
    # run in two spawned processes (about 4 s a step each)
    import multiprocessing as mp
    shape, steps = (256, 256, 256), 10
    P = pss()
    s = P.System(shape, dt=0.005, seed=2405, precision="f32")
    P.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
    P.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi")
    assert s.step_path == "fast3d_rows"
    s.init_uniform(0, -0.05, 0.05)
    s.init_uniform(1, -0.05, 0.05)
    s.step(steps)
    got = [s.get_spectrum(f) for f in (0, 1)]
    s.close()
    with mp.get_context("spawn").Pool(2) as pool:
        refs = pool.map(_oracle_3d_field, [(0, steps), (1, steps)])
    for fid in (0, 1):
        check_spectrum(got[fid], refs[fid], 1e-4, what=f"field {fid}")


@pytest.mark.parametrize("knobs", [
    dict(row_pairs=1), dict(row_pairs=2), dict(row_pairs=4), dict(row_pairs=8),
    dict(mid_planes=1), dict(mid_planes=2), dict(mid_planes=4), dict(col_tiles=2), dict(col_tiles=4),
    dict(pdl=1), dict(row_pairs=2, mid_planes=4, pdl=1),
    dict(col_radix=8, row_radix=8, mid_radix=8), dict(col_radix=16, row_radix=16, mid_radix=16),
    dict(col_radix=8, row_radix=16, mid_radix=8, row_pairs=2),
])
@pytest.mark.parametrize("shape", [(16, 32, 32), (8, 64, 16), (64, 128), (1024, 32), (32, 1024)])
def test_launch_shapes_do_not_change_results(shape, knobs):
    # every launch-shape knob must give the oracle's result (Model A + B pair)
    steps = 12
    P = pss()
    s = P.System(shape, dt=0.005, seed=8, precision="f32")
    P.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
    P.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi")
    for k, v in knobs.items():
        s.set_tuning(k, v)
    s.init_uniform(0, -0.05, 0.05)
    s.init_uniform(1, -0.05, 0.05)
    s.step(steps)
    ma = O.model_a(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=8, field_id=0)
    mb = O.model_b(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=8, field_id=1)
    for fid, m in ((0, ma), (1, mb)):
        ref = O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.05, 0.05)), 0, steps))
        check_spectrum(s.get_spectrum(fid), ref, 1e-4, what=f"field {fid} {knobs}")


def test_stream_switch_keeps_order():
    # initialise on the default stream, then step on a non-blocking torch stream
    import torch
    P = pss()
    ref_sys = P.model_b((256, 256), seed=31, precision="f32")
    ref_sys.init_uniform(0, -0.1, 0.1)
    ref_sys.step(30)
    ref = ref_sys.get_spectrum(0)
    s = P.model_b((256, 256), seed=31, precision="f32")
    s.init_uniform(0, -0.1, 0.1)
    st = torch.cuda.Stream()
    s.set_stream(st)
    s.step(30)
    np.testing.assert_array_equal(s.get_spectrum(0), ref)
