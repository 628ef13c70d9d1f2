"""The FP32 2D path with one warp per transform (sides of 256, 512 and 1024
points) against the FP64 oracle and against the generic kernels.

Bars: rel-L2 <= 1e-4 against the oracle over <= 200 steps; the generic FP32
kernels agree with it to FP32 rounding (rel-L2 <= 1e-5 over 100 steps); its
launch-shape knobs change no bit of the result.
"""
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


def _model_b(shape, fast=True, knobs=None, **kw):
    s = pss().model_b(shape, precision="f32", **kw)
    s.set_tuning("fast2d", 1 if fast else 0)
    for k, v in (knobs or {}).items():
        s.set_tuning(k, v)
    s.init_uniform(0, -0.1, 0.1)
    return s


def _oracle_b(shape, steps, **kw):
    m = O.model_b(shape, **kw)
    phi = O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1))
    return O.half(O.run(m, phi, 0, steps))


@pytest.mark.parametrize("shape,order,noisy,steps", [
    ((256, 256), 2, True, 100), ((512, 256), 2, True, 40), ((256, 512), 3, True, 40),
    ((256, 256), 0, True, 60), ((256, 256), 2, False, 60), ((256, 1024), 2, True, 20),
])
def test_matches_oracle(shape, order, noisy, steps):
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=17, dealias_order=order, noisy=noisy)
    s = _model_b(shape, **kw)
    s.step(steps)
    check_spectrum(s.get_spectrum(0), _oracle_b(shape, steps, **kw), 1e-4)
    # the real field too (generic inverse of the state the fast path wrote)
    assert rel(s.get_field(0), np.fft.irfftn(_oracle_b(shape, steps, **kw), s=shape, axes=(0, 1))) < 1e-3


@pytest.mark.parametrize("shape", [(1024, 1024), (1024, 256), (256, 1024), (512, 512)])
def test_matches_generic_kernels(shape):
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.01, seed=2405)
    fast, gen = _model_b(shape, True, **kw), _model_b(shape, False, **kw)
    for s in (fast, gen):
        s.step(100)
    a, b = fast.get_spectrum(0), gen.get_spectrum(0)
    assert rel(a, b) < 1e-5, rel(a, b)
    # the conserved mode is never touched by the update: bit-identical
    assert a[0, 0] == b[0, 0]


@pytest.mark.parametrize("knobs", [dict(col2_warps=1), dict(col2_warps=4), dict(col2_warps=16),
                                   dict(row2_pairs=1), dict(row2_pairs=4), dict(row2_pairs=8),
                                   dict(pdl=1), dict(pdl=0), dict(graph_steps=3, row2_pairs=1, col2_warps=2),
                                   dict(row2_share=0), dict(row2_share=100), dict(row2_share=30, row2_noise=2)])
def test_launch_shapes_do_not_change_bits(knobs):
    shape = (512, 256)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=3)
    ref, s = _model_b(shape, **kw), _model_b(shape, knobs=knobs, **kw)
    ref.step(37)
    s.step(37)
    np.testing.assert_array_equal(s.get_spectrum(0), ref.get_spectrum(0))


@pytest.mark.parametrize("shape", [(1024, 1024), (512, 1024), (1024, 512)])
def test_fft_radix_changes_only_rounding(shape):
    # radix-8, -16 and -32 passes order the sums differently: FP32 rounding apart
    # (radix 32 serves sides of 1024; other sides fall back to 16)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.01, seed=9)
    runs = []
    for radix in (8, 16, 32):
        s = _model_b(shape, knobs=dict(col2_radix=radix, row2_radix=radix), **kw)
        s.step(50)
        runs.append(s.get_spectrum(0))
    assert rel(runs[1], runs[0]) < 1e-5
    assert rel(runs[2], runs[0]) < 1e-5


def test_switching_paths_mid_run():
    # the work arrays change layout with the path: a switch must redo the product
    shape = (256, 256)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=5)
    s = _model_b(shape, **kw)
    s.step(20)
    s.set_tuning("fast2d", 0)
    s.step(20)
    s.set_tuning("fast2d", 1)
    s.step(20)
    check_spectrum(s.get_spectrum(0), _oracle_b(shape, 60, **kw), 1e-4)


def test_model_a_and_b_pair():
    shape, steps = (256, 512), 40
    P = pss()
    s = P.System(shape, dt=0.005, seed=21, precision="f32")
    P.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
    P.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi", dealias_order=3)
    s.init_uniform(0, -0.05, 0.05)
    s.init_uniform(1, -0.05, 0.05)
    s.step(steps)
    ma = O.model_a(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=21, field_id=0)
    mb = O.model_b(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=21, field_id=1, dealias_order=3)
    for fid, m in ((0, ma), (1, mb)):
        ref = O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.05, 0.05)), 0, steps))
        check_spectrum(s.get_spectrum(fid), ref, 1e-4, what=f"field {fid}")


def test_batched_instances_match_single_runs():
    P = pss()
    shape, seeds, a_vals = (256, 256), [101, 102, 103], [-1.2, -0.8, -1.0]
    s = P.System(shape, dt=0.01, batch=3, seeds=seeds, precision="f32")
    P.add_model_b_field(s, a=-1.0, b=1.0, K=1.0, D=0.01)
    s.set_param_batch(0, np.asarray(a_vals))
    for i in range(3):
        s.select_instance(i)
        s.init_uniform(0, -0.1, 0.1)
    s.step(25)
    for i in range(3):
        one = P.model_b(shape, dt=0.01, a=a_vals[i], b=1.0, K=1.0, D=0.01, seed=seeds[i], precision="f32")
        one.init_uniform(0, -0.1, 0.1)
        one.step(25)
        s.select_instance(i)
        np.testing.assert_array_equal(s.get_spectrum(0), one.get_spectrum(0))
        if i == 1:
            ref = _oracle_b(shape, 25, dt=0.01, a=a_vals[i], b=1.0, K=1.0, D=0.01, seed=seeds[i])
            check_spectrum(s.get_spectrum(0), ref, 1e-4)


def test_nonfinite_is_reported_on_the_fast_path():
    P = pss()
    s = P.model_b((256, 256), noisy=False, precision="f32")
    x = np.zeros((256, 256))
    x[3, 7] = np.inf
    s.set_field(0, x)
    s.step(2)
    with pytest.raises(P.PssError) as ei:
        s.sync()
    assert ei.value.code == P.PSS_ENONFINITE


# ---------------------------------------------------------------------------
# the 3D x pass on FFT groups (tiled arrays, tuning key "fast3d")
# ---------------------------------------------------------------------------
def _pair_3d(shape, fast, order=2, seed=8):
    P = pss()
    s = P.System(shape, dt=0.005, seed=seed, precision="f32")
    P.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi", dealias_order=order)
    P.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi", dealias_order=order)
    s.set_tuning("fast3d", 1 if fast else 0)
    s.init_uniform(0, -0.05, 0.05)
    s.init_uniform(1, -0.05, 0.05)
    return s


@pytest.mark.parametrize("shape,order", [((8, 16, 256), 2), ((4, 8, 256), 0), ((4, 4, 512), 3)])
def test_3d_x_pass_matches_oracle(shape, order):
    steps = 16
    s = _pair_3d(shape, True, order)
    assert s.step_path == "fast3d_rows"
    s.step(steps)
    ma = O.model_a(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=8, field_id=0, dealias_order=order)
    mb = O.model_b(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=8, field_id=1, dealias_order=order)
    for fid, m in ((0, ma), (1, mb)):
        ref = O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.05, 0.05)), 0, steps))
        check_spectrum(s.get_spectrum(fid), ref, 1e-4, what=f"field {fid}")


@pytest.mark.parametrize("shape", [(16, 32, 512), (32, 32, 1024), (64, 64, 256)])
def test_3d_x_pass_matches_generic_kernels(shape):
    fast, gen = _pair_3d(shape, True), _pair_3d(shape, False)
    assert gen.step_path == "generic"
    for s in (fast, gen):
        s.step(30)
    for fid in (0, 1):
        check_spectrum(fast.get_spectrum(fid), gen.get_spectrum(fid), 1e-5, what=f"field {fid}")
