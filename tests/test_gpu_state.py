"""Checkpoint and resume through the C ABI (pss_save_state / pss_load_state).

A run saved in the middle and loaded into a fresh handle takes the same steps,
bit for bit, as the run that was never interrupted: on the FP32 2D path with
the noise drawn a step ahead, on the generic kernels (1D, 3D, FP64), on a
batched system with per-instance parameters, and across parameter changes.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2405_02410_gb300 import build
    build.build()


def P():
    from paper_2405_02410_gb300 import pss
    return pss


def _spectra(s, nfields):
    out = []
    for b in range(s.batch):
        s.select_instance(b)
        out.extend(s.get_spectrum(f) for f in range(nfields))
    s.select_instance(0)
    return out


def _model_b(shape, prec="f32", batch=1, seed=2405):
    pss = P()
    s = pss.System(shape, dt=0.01, seed=seed, precision=prec, batch=batch)
    pss.add_model_b_field(s, a=-1, b=1, K=1, D=0.01)
    return s


@pytest.mark.parametrize("shape,prec,path", [
    ((256, 256), "f32", "persist2d"),
    ((512, 256), "f32", "fast2d"),
    ((64, 64), "f32", "generic"),
    ((8, 16, 32), "f64", "generic"),
    ((1024,), "f32", "generic"),
])
def test_resume_is_bit_identical(shape, prec, path):
    a = _model_b(shape, prec)
    assert a.step_path == path, a.step_path
    a.init_uniform(0, -0.1, 0.1)
    a.step(7)
    blob = a.save_state()
    a.step(13)
    ref = a.get_spectrum(0)
    b = _model_b(shape, prec, seed=99)        # a different seed: the state carries the saved one
    b.load_state(blob)
    assert b.get_step() == 7
    b.step(13)
    got = b.get_spectrum(0)
    assert got.tobytes() == ref.tobytes()
    a.close()
    b.close()


def test_resume_of_a_batch_with_per_instance_parameters():
    shape, batch = (256, 256), 3
    a = _model_b(shape, batch=batch)
    a.set_param_batch(0, np.array([-1.2, -0.9, -0.6]))        # "phi.a" per instance
    for i in range(batch):
        a.select_instance(i)
        a.init_uniform(0, -0.1, 0.1)
    a.select_instance(0)
    a.step(5)
    blob = a.save_state()
    a.step(11)
    ref = _spectra(a, 1)
    b = _model_b(shape, batch=batch, seed=7)                   # default parameters and other seeds
    b.load_state(blob)
    assert abs(b.get_param(0) - (-1.2)) == 0.0
    b.step(11)
    got = _spectra(b, 1)
    for x, y in zip(got, ref):
        assert x.tobytes() == y.tobytes()


def test_two_fields_3d_and_the_step_counter():
    pss = P()
    shape = (8, 16, 16)

    def build(seed):
        s = pss.System(shape, dt=0.005, seed=seed, precision="f32")
        pss.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
        pss.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi")
        return s

    a = build(5)
    a.init_uniform(0, -0.05, 0.05)
    a.init_uniform(1, -0.05, 0.05)
    a.step(4)
    blob = a.save_state()
    a.step(9)
    b = build(6)
    b.load_state(blob)
    b.step(9)
    assert b.get_step() == a.get_step() == 13
    for f in (0, 1):
        assert b.get_spectrum(f).tobytes() == a.get_spectrum(f).tobytes()


def test_load_rejects_another_system_and_leaves_it_unchanged():
    pss = P()
    a = _model_b((64, 64))
    a.init_uniform(0, -0.1, 0.1)
    blob = a.save_state()
    b = _model_b((64, 128))
    b.init_uniform(0, -0.2, 0.2)
    before = b.get_spectrum(0)
    with pytest.raises(pss.PssError) as ei:
        b.load_state(blob)
    assert ei.value.code == pss.PSS_EINVAL
    assert b.get_spectrum(0).tobytes() == before.tobytes()
    with pytest.raises(pss.PssError):
        a.load_state(blob[:-8])                                 # truncated
    with pytest.raises(pss.PssError):
        a.load_state(b"not a state" + blob[11:])                # wrong tag
    c = _model_b((64, 64), prec="f64")
    with pytest.raises(pss.PssError):
        c.load_state(blob)                                      # other precision
