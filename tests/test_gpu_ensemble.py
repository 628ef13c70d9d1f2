"""Batched ensembles on the GPU: independent instances (own seed, own
parameter values) in one system, and several systems stepped from one graph.
Each instance must equal a single-system run bit for bit, and the oracle."""
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


def _batch(shape, seeds, a_values, precision="f32"):
    P = pss()
    s = P.System(shape, dt=0.01, batch=len(seeds), seeds=seeds, precision=precision)
    f = P.add_model_b_field(s, a=-1.0, b=1.0, K=1.0, D=0.01)
    s.set_param_batch(0, np.asarray(a_values, dtype=float))    # parameter 0 is "phi.a"
    for i in range(len(seeds)):
        s.select_instance(i)
        s.init_uniform(f, -0.1, 0.1)
    return s


@pytest.mark.parametrize("shape", [(64, 64), (32, 128), (16, 16, 16)])
def test_batch_instances_equal_single_runs(shape):
    seeds = [11, 12, 13, 1 << 40]
    a_values = [-1.5, -1.0, -0.75, -0.5]
    s = _batch(shape, seeds, a_values)
    s.step(40)
    P = pss()
    for i, (sd, av) in enumerate(zip(seeds, a_values)):
        one = P.model_b(shape, dt=0.01, a=av, b=1.0, K=1.0, D=0.01, seed=sd)
        one.init_uniform(0, -0.1, 0.1)
        one.step(40)
        s.select_instance(i)
        np.testing.assert_array_equal(s.get_spectrum(0), one.get_spectrum(0))


@pytest.mark.parametrize("prec,tol", [("f32", 1e-4), ("f64", 1e-10)])
def test_batch_matches_oracle(prec, tol):
    shape, steps = (64, 64), 50
    seeds = [5, 6, 7]
    a_values = [-1.4, -0.9, -0.6]
    s = _batch(shape, seeds, a_values, precision=prec)
    s.step(steps)
    for i, (sd, av) in enumerate(zip(seeds, a_values)):
        m = O.model_b(shape, dt=0.01, a=av, b=1.0, K=1.0, D=0.01, seed=sd)
        ref = O.half(O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1)), 0, steps))
        s.select_instance(i)
        check_spectrum(s.get_spectrum(0), ref, tol)


def test_step_many_mixed_sizes_equal_separate_runs():
    P = pss()
    shapes = [(64, 64), (128, 128), (256, 256)]
    systems = [_batch(sh, [100 + j, 200 + j], [-1.2, -0.8]) for j, sh in enumerate(shapes)]
    P.step_many(systems, 37)          # two graph replays of 16 + 5 eager steps
    for j, sh in enumerate(shapes):
        ref = _batch(sh, [100 + j, 200 + j], [-1.2, -0.8])
        ref.step(37)
        for i in range(2):
            systems[j].select_instance(i)
            ref.select_instance(i)
            np.testing.assert_array_equal(systems[j].get_spectrum(0), ref.get_spectrum(0))
        assert systems[j].get_step() == 37


def test_step_many_runs_a_system_listed_twice_in_order():
    # distinct systems run as parallel branches of the captured graph; a system
    # listed twice keeps the serial order: two steps per step of the call
    P = pss()
    a = _batch((64, 64), [5, 6], [-1.0, -0.9])
    b = _batch((64, 64), [5, 6], [-1.0, -0.9])
    P.step_many([a, a], 20)           # one graph replay of 16 (32 steps) + 4 eager (8 steps)
    b.step(40)
    assert a.get_step() == 40
    for i in range(2):
        a.select_instance(i)
        b.select_instance(i)
        np.testing.assert_array_equal(a.get_spectrum(0), b.get_spectrum(0))


def test_param_change_between_graph_replays():
    # parameters live on the device: a change between runs applies without re-capture
    P = pss()
    s = _batch((64, 64), [1, 2], [-1.0, -1.0])
    s.step(32)
    s.set_param_batch(0, np.array([-0.7, -1.3]))
    s.step(32)
    for i, (first, second) in enumerate([(-1.0, -0.7), (-1.0, -1.3)]):
        one = P.model_b((64, 64), dt=0.01, a=first, b=1.0, K=1.0, D=0.01, seed=i + 1)
        one.init_uniform(0, -0.1, 0.1)
        one.step(32)
        one.set_param(0, second)
        one.step(32)
        s.select_instance(i)
        np.testing.assert_array_equal(s.get_spectrum(0), one.get_spectrum(0))
