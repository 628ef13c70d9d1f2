"""Sharding an ensemble over ranks (paper_2405_02410_gb300.ensemble), on CPU.

The instances are split by cost (sites x steps); each rank runs its share,
and the per-instance FP64 S(q) are gathered and averaged per lattice size in
instance order.  The per-instance S(q) here come from the FP64 oracle (the
host logic under test does not care where they come from), so a run on two
gloo ranks must give the single-rank result bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _spec():
    from paper_2405_02410_gb300 import ensemble as E
    sp = E.recipe(n=10, gen_seed=7, base_seed=300, steps=6, sizes=(8, 16))
    sp.nbins = 8
    sp.D = 0.05
    return sp


def oracle_runner(spec, indices):
    """Per-instance S(q) bin means from the FP64 oracle (Model B, the instance's side, seed and a)."""
    from oracle import oracle as O
    out = {}
    for i in indices:
        n = spec.side[i]
        m = O.model_b((n, n), dt=spec.dt, a=spec.a[i], b=spec.b, K=spec.K, D=spec.D, seed=spec.seed[i])
        phi = O.run(m, O.to_spectrum(m, O.init_uniform(m, spec.lo, spec.hi)), 0, spec.steps)
        S, _, _ = O.structure_factor(m, phi, spec.nbins)
        out[i] = S
    return out


def test_partition_covers_every_instance_once_and_balances_cost():
    from paper_2405_02410_gb300 import ensemble as E
    sp = E.recipe(n=512)
    costs = [sp.cost(i) for i in range(len(sp))]
    for world in (1, 2, 3, 8):
        parts = E.partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(512))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)          # greedy longest-first bound
        assert parts == E.partition(costs, world)              # deterministic
        assert all(p == sorted(p) for p in parts)
    # the 512-instance recipe: every side occurs, seeds base + i, a in [-1.5, -0.5)
    assert set(sp.side) == {64, 128, 256, 512}
    assert sp.seed[:3] == [10000, 10001, 10002]
    assert all(-1.5 <= a < -0.5 for a in sp.a)


def test_merge_averages_in_instance_order():
    from paper_2405_02410_gb300 import ensemble as E
    sp = E.Spec(side=[8, 16, 8, 8], seed=[1, 2, 3, 4], a=[-1.0] * 4, nbins=2)
    per = {0: np.array([1.0, 2.0]), 1: np.array([5.0, 5.0]), 2: np.array([3.0, 4.0]), 3: np.array([2.0, 0.0])}
    m = E.merge(sp, per)
    np.testing.assert_array_equal(m[8], (np.array([1.0, 2.0]) + np.array([3.0, 4.0]) + np.array([2.0, 0.0])) / 3)
    np.testing.assert_array_equal(m[16], np.array([5.0, 5.0]))
    with pytest.raises(KeyError):
        E.merge(sp, {0: per[0]})


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    try:
        import torch.distributed as dist
        from paper_2405_02410_gb300 import ensemble as E
        from tests.test_ensemble_shard_gloo import _spec, oracle_runner
        dist.init_process_group("gloo", rank=rank, world_size=world)
        merged, idx = E.run_sharded(_spec(), rank, world, oracle_runner)
        dist.destroy_process_group()
        q.put((rank, idx, {k: v.tolist() for k, v in merged.items()}))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, "error", repr(e)))


def test_two_ranks_give_the_single_rank_result_bit_for_bit():
    import torch.multiprocessing as mp
    from paper_2405_02410_gb300 import ensemble as E
    sp = _spec()
    single, idx1 = E.run_sharded(sp, 0, 1, oracle_runner)
    assert idx1 == list(range(len(sp)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted((q.get(timeout=240) for _ in range(2)), key=lambda x: x[0])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(r[1] != "error" for r in res), res
    (_, idx_a, m_a), (_, idx_b, m_b) = res
    assert sorted(idx_a + idx_b) == list(range(len(sp))) and not set(idx_a) & set(idx_b)
    assert idx_a and idx_b
    for merged in (m_a, m_b):
        assert set(merged) == set(single)
        for side, S in merged.items():
            assert np.array_equal(np.asarray(S), single[side]), side
