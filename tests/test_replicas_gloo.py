"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

A single system does not shard (a distributed FFT would need an all-to-all
transpose per pass), so N GPUs run N independent replicas: the only
collectives are a barrier and the max of the ranks' timed durations, and the
job's throughput is all ranks' units over the slowest rank's time.  The
reference arm runs on rank 0 alone; the other ranks exit without work.
"""
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, mode, q):
    os.environ["CUDA_VISIBLE_DEVICES"] = ""          # gloo on CPU, whatever machine runs this
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), PSS_REF_BUDGET_S="0.2")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    try:
        if mode == "rate":
            w, r, _ = bench.dist_setup(world)
            bench.barrier(w)
            value, t_max = bench.whole_job_rate(1000, 10.0 * (r + 1), w)
            q.put((r, w, dist.get_backend(), value, t_max))
            dist.destroy_process_group()
        else:
            out = io.StringIO()
            old, sys.stdout = sys.stdout, out
            try:
                rc = bench.main(["--impl", "reference", "--gpus", str(world), "--steps", "1", "--warmup", "3"])
            finally:
                sys.stdout = old
            if dist.is_initialized():
                dist.destroy_process_group()
            q.put((rank, rc, out.getvalue()))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, "error", repr(e)))


def _run(world, mode):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda x: x[0])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    return res


def test_two_replicas_take_the_slowest_rank():
    res = _run(2, "rate")
    assert all(r[1] != "error" for r in res), res
    for rank, world, backend, value, t_max in res:
        assert world == 2 and backend == "gloo"
        assert t_max == 20.0                       # rank 1's 20 ms, on both ranks
        assert value == pytest.approx(2 * 1000 / 0.020)


def test_reference_arm_runs_on_rank_0_only():
    import json
    res = _run(2, "reference")
    assert all(r[1] != "error" for r in res), res
    (r0, rc0, out0), (r1, rc1, out1) = res
    assert rc0 == 0 and rc1 == 0
    assert out1.strip() == ""
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
