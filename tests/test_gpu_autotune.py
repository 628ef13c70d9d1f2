"""pss_autotune: the launch-shape autotuner.

It times the knobs of a system's step path on the GPU and keeps the fastest
settings.  Checked here: the call leaves the state and the step counter as
they were (bit for bit), the run that follows still matches the FP64 oracle
(rel-L2 <= 1e-4) and the untuned run to FP32 rounding (the radix changes only
the rounding order: rel-L2 <= 1e-5), the chosen settings are never slower
than the starting ones in the tuner's own back-to-back timing, and the
report names every knob of the path, on all three step paths and a batch.
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


KNOBS = {
    "fast2d": {"col2_radix", "row2_radix", "row2_pairs", "col2_warps", "row2_noise", "pdl", "graph_steps"},
    "fast3d_rows": {"col_radix", "row2_radix", "mid_radix", "mid_planes", "col_tiles", "pdl", "graph_steps"},
    "generic": {"col_radix", "row_radix", "row_pairs", "col_tiles", "pdl", "graph_steps"},   # 3D: also mid_radix, mid_planes
}
# a system that qualifies for the persistent step also times it against the two-kernel step
KNOBS["persist2d"] = KNOBS["fast2d"] | {"persist"}


def _pair(shape, seed=8):
    P = pss()
    s = P.System(shape, dt=0.005, seed=seed, precision="f32")
    P.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
    P.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi")
    s.init_uniform(0, -0.05, 0.05)
    s.init_uniform(1, -0.05, 0.05)
    return s


def _oracle_pair(shape, steps, seed=8):
    out = []
    ma = O.model_a(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=seed, field_id=0)
    mb = O.model_b(shape, dt=0.005, a=-1, b=1, K=1, D=0.05, seed=seed, field_id=1)
    for m in (ma, mb):
        out.append(O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.05, 0.05)), 0, steps)))
    return out


def _check_report(rep, path, dim=2):
    if path == "persist2d":
        assert rep["path"] in (3, 1) and rep["persist"] == (1 if rep["path"] == 3 else 0)   # either step may win
    else:
        assert rep["path"] == {"generic": 0, "fast2d": 1, "fast3d_rows": 2}[path]
    knobs = set(rep) - {"path", "trials", "skipped", "initial_ms", "tuned_ms"}
    want = KNOBS[path] | ({"mid_radix", "mid_planes"} if path == "generic" and dim == 3 else set())
    assert knobs == want, knobs
    assert rep["trials"] >= 5
    assert 0 < rep["tuned_ms"] <= rep["initial_ms"]


@pytest.mark.parametrize("shape,path", [((256, 256), "persist2d"), ((512, 256), "fast2d"), ((64, 64), "generic"),
                                        ((8, 16, 256), "fast3d_rows"),
                                        ((16, 32, 32), "generic")])
def test_autotune_keeps_the_run(shape, path):
    steps0, steps1 = 10, 20
    if len(shape) == 2:
        kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=17)
        tuned, plain = (pss().model_b(shape, precision="f32", **kw) for _ in range(2))
        for s in (tuned, plain):
            s.init_uniform(0, -0.1, 0.1)
        m = O.model_b(shape, **kw)
        ref = [O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1)), 0, steps0 + steps1))]
    else:
        tuned, plain = _pair(shape), _pair(shape)
        ref = _oracle_pair(shape, steps0 + steps1)
    nf = len(ref)
    assert tuned.step_path == path
    for s in (tuned, plain):
        s.step(steps0)
    before = [tuned.get_spectrum(f) for f in range(nf)]
    rep = tuned.autotune(steps_per_trial=16)
    _check_report(rep, path, len(shape))
    assert tuned.get_step() == steps0
    for f in range(nf):
        np.testing.assert_array_equal(tuned.get_spectrum(f), before[f])
    for s in (tuned, plain):
        s.step(steps1)
    for f in range(nf):
        a, b = tuned.get_spectrum(f), plain.get_spectrum(f)
        assert rel(a, b) < 1e-5, (f, rel(a, b))
        assert rel(a, ref[f]) < 1e-4, (f, rel(a, ref[f]))


def test_autotune_settings_are_pss_set_tuning_values():
    # the report's settings, given to an untuned twin, reproduce the tuned run bit for bit
    shape = (512, 256)
    kw = dict(dt=0.01, a=-1, b=1, K=1, D=0.05, seed=3)
    tuned, twin = (pss().model_b(shape, precision="f32", **kw) for _ in range(2))
    for s in (tuned, twin):
        s.init_uniform(0, -0.1, 0.1)
    rep = tuned.autotune(steps_per_trial=16)
    twin.set_tunings(rep)
    for s in (tuned, twin):
        s.step(33)
    np.testing.assert_array_equal(tuned.get_spectrum(0), twin.get_spectrum(0))


def test_autotune_batch_and_step_many():
    # a batched system tuned on its own, then stepped beside another system from one graph
    P = pss()
    shape, seeds = (256, 256), [101, 102]
    s = P.System(shape, dt=0.01, batch=2, seeds=seeds, precision="f32")
    P.add_model_b_field(s, a=-1.0, b=1.0, K=1.0, D=0.01)
    for i in range(2):
        s.select_instance(i)
        s.init_uniform(0, -0.1, 0.1)
    other = P.model_b((64, 64), dt=0.01, a=-1.0, b=1.0, K=1.0, D=0.01, seed=7, precision="f32")
    other.init_uniform(0, -0.1, 0.1)
    _check_report(s.autotune(steps_per_trial=16), "fast2d")
    _check_report(other.autotune(steps_per_trial=16), "generic")
    P.step_many([s, other], 40)
    for i in range(2):
        one = P.model_b(shape, dt=0.01, a=-1.0, b=1.0, K=1.0, D=0.01, seed=seeds[i], precision="f32")
        one.init_uniform(0, -0.1, 0.1)
        one.step(40)
        s.select_instance(i)
        check_spectrum(s.get_spectrum(0), one.get_spectrum(0), 1e-5)
    ref = O.model_b((64, 64), dt=0.01, a=-1.0, b=1.0, K=1.0, D=0.01, seed=7)
    want = O.half(O.run(ref, O.to_spectrum(ref, O.init_uniform(ref, -0.1, 0.1)), 0, 40))
    check_spectrum(other.get_spectrum(0), want, 1e-4)


def test_autotune_rejects_bad_arguments():
    P = pss()
    s = P.System((64, 64), dt=0.01, precision="f32")
    with pytest.raises(P.PssError):
        s.autotune()          # no fields yet
    P.add_model_b_field(s, a=-1.0, b=1.0, K=1.0, D=0.01)
    with pytest.raises(P.PssError):
        s.autotune(steps_per_trial=0)
