"""The multi-process path of bench.py on CPU (gloo, world size 2).

Registrations shard by problem: every rank registers its own pair and no
collective touches the data path.  The only cross-rank steps are the timing
barrier, the max over ranks of the timed seconds and the sum of the units,
which these tests exercise with two spawned gloo ranks on 127.0.0.1.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_info()
    d = bench.Dist(w)
    d.barrier()
    seconds = d.max(1.5 + rank)          # the slowest rank sets the job time
    units = d.sum(100.0 * (rank + 1))     # every rank's work counts
    d.barrier()
    d.close()
    out.put((r, w, local, seconds, units))


def test_two_gloo_ranks_aggregate_max_time_and_total_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    for _, _, _, seconds, units in res:
        assert seconds == 2.5 and units == 300.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload, warmup, steps, gpus, cpu_sample_particles = "mask64", 0, 1, 2, 1
    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(1)
    assert d.max(3.0) == 3.0 and d.sum(4.0) == 4.0
    d.barrier()
    d.close()
