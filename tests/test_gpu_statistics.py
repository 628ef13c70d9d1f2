"""Long-run statistics of the FP32 GPU path against the FP64 oracle.

Over long runs the FP32 and FP64 trajectories drift apart, so the check is on
what the method is run for: the radially binned structure factor S(q) and the
coarsening length L = 2 pi sum S / sum |q| S, averaged over seeds, must agree
within 2 %.  The oracle runs in a pool of spawned worker processes (safe after
CUDA has been initialised in this process).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

NBINS = 64
TOL = 0.02


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2405_02410_gb300 import build
    build.build()


def pss():
    from paper_2405_02410_gb300 import pss as m
    return m


def _oracle_sq(args):
    """S(q), mode counts and L of one oracle run (worker process)."""
    shape, a, seed, steps = args
    m = O.model_b(shape, dt=0.01, a=a, b=1.0, K=1.0, D=0.01, seed=seed)
    phi = O.run(m, O.to_spectrum(m, O.init_uniform(m, -0.1, 0.1)), 0, steps)
    return O.structure_factor(m, phi, NBINS)


def _oracle_pool(jobs):
    O.build()                      # compile once, before the workers load it
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        return pool.map(_oracle_sq, jobs)


def _gpu_batch(shape, seeds, a_values, steps):
    P = pss()
    s = P.System(shape, dt=0.01, batch=len(seeds), seeds=seeds, precision="f32")
    f = P.add_model_b_field(s, a=-1.0, b=1.0, K=1.0, D=0.01)
    s.set_param_batch(0, np.asarray(a_values, dtype=float))     # parameter 0 is "phi.a"
    for i in range(len(seeds)):
        s.select_instance(i)
        s.init_uniform(f, -0.1, 0.1)
    return s


def _gpu_sq(s, n):
    out = []
    for i in range(n):
        s.select_instance(i)
        out.append(s.structure_factor(0, NBINS))
    return out


def _compare(gpu, ref):
    Sg = np.mean([g[0] for g in gpu], axis=0)
    So = np.mean([r[0] for r in ref], axis=0)
    np.testing.assert_array_equal(gpu[0][1], ref[0][1])          # the same modes in every bin
    filled = ref[0][1] > 0
    dev = np.abs(Sg[filled] - So[filled]) / So[filled]
    assert dev.max() <= TOL, (dev.max(), int(np.argmax(dev)))
    Lg = np.mean([g[2] for g in gpu])
    Lo = np.mean([r[2] for r in ref])
    assert abs(Lg - Lo) <= TOL * Lo, (Lg, Lo)


def test_model_b_256_long_run_structure_factor_8_seeds():
    # Model B at 256 x 256 (the 1024 x 1024 workload's parameters), 2000 steps, 8 seeds
    shape, steps = (256, 256), 2000
    seeds = [2405 + i for i in range(8)]
    s = _gpu_batch(shape, seeds, [-1.0] * 8, steps)
    s.step(steps)
    gpu = _gpu_sq(s, len(seeds))
    ref = _oracle_pool([(shape, -1.0, sd, steps) for sd in seeds])
    _compare(gpu, ref)


def test_ensemble_of_mixed_sizes_structure_factor_by_size():
    # an ensemble of instances with their own seed and a in [-1.5, -0.5], stepped
    # together from one graph; S(q) averaged over the instances of each size
    P = pss()
    rng = np.random.default_rng(512)
    steps, per_size = 1000, 6
    groups = []
    for j, shape in enumerate([(64, 64), (128, 128)]):
        seeds = [7000 + 100 * j + i for i in range(per_size)]
        a_values = list(rng.uniform(-1.5, -0.5, size=per_size))
        groups.append((shape, seeds, a_values, _gpu_batch(shape, seeds, a_values, steps)))
    P.step_many([g[3] for g in groups], steps)
    jobs = [(shape, a, sd, steps) for shape, seeds, a_values, _ in groups for sd, a in zip(seeds, a_values)]
    ref = _oracle_pool(jobs)
    k = 0
    for shape, seeds, a_values, s in groups:
        _compare(_gpu_sq(s, per_size), ref[k:k + per_size])
        k += per_size


def test_ensemble_recipe_structure_factor_all_four_sides():
    # instances of the 512-instance ensemble recipe (their own side, seed and a), built
    # and stepped through the ensemble module (one batched system per side, one graph);
    # the S(q) averaged over the instances of each side of 64, 128, 256 and 512 points
    # against the oracle's (4 instances of the small sides, 2 of the large ones)
    from paper_2405_02410_gb300 import ensemble as E
    P = pss()
    steps = 300
    full = E.recipe(n=512, steps=steps)
    want = {64: 4, 128: 4, 256: 2, 512: 2}
    pick = []
    for i in range(len(full)):
        if want.get(full.side[i], 0) > 0:
            pick.append(i)
            want[full.side[i]] -= 1
    spec = E.Spec(side=[full.side[i] for i in pick], seed=[full.seed[i] for i in pick],
                  a=[full.a[i] for i in pick], steps=steps, nbins=NBINS)
    groups = E.build_systems(P, spec, list(range(len(spec))))
    P.step_many([g[1] for g in groups], steps)
    per = E.structure_factors(groups, NBINS)
    ref = _oracle_pool([((spec.side[i],) * 2, spec.a[i], spec.seed[i], steps) for i in range(len(spec))])
    got_by_side = E.merge(spec, per)
    ref_by_side = E.merge(spec, {i: r[0] for i, r in enumerate(ref)})
    assert set(got_by_side) == {64, 128, 256, 512}
    for side in got_by_side:
        counts = ref[spec.side.index(side)][1]
        filled = counts > 0
        dev = np.abs(got_by_side[side][filled] - ref_by_side[side][filled]) / ref_by_side[side][filled]
        assert dev.max() <= TOL, (side, dev.max())
