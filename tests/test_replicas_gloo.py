"""The multi-GPU mode of bench.py is replicas only: every rank runs its own
independent searches and the ranks exchange nothing on the data path, only a
barrier and the max / sum of timing scalars.  That host-side plumbing runs here
as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    d = bench.Dist()
    d.init(torch, backend="gloo")
    d.barrier()
    mx = d.max(torch, float(10 + rank), "cpu")
    sm = d.sum(torch, float(1 + rank), "cpu")
    q.put((rank, mx, sm, bench.replica_seeds(rank, 4)))
    d.pg.destroy_process_group()


def test_two_gloo_ranks_reduce_timings_and_split_seeds():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [11.0, 11.0]  # max over ranks, on every rank
    assert [o[2] for o in out] == [3.0, 3.0]    # sum over ranks
    seeds = [o[3] for o in out]
    assert seeds == [[0, 1, 2, 3], [4, 5, 6, 7]]  # disjoint starts: replicas of one workload
