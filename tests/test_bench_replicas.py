"""Multi-GPU path of bench.py (replicas, no collective on the data path):
the host logic run as two gloo ranks on the CPU.  Each rank draws its own
pairs, the job time is the slowest rank's, and the whole-job rate counts
every rank's pairs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    import bench
    from paper_1802_07210_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = [120.0, 80.0][rank]
    t = bench.max_over_ranks(torch, dist, ws, local_ms, torch.device("cpu"))
    L, _, _ = synth.workload_pair(synth.SMALL_320, bench.replica_seed(rank, 0), 1)
    q.put((rank, t, int(L.astype(np.int64).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [120.0, 120.0]  # max over ranks
    assert out[0][2] != out[1][2]  # disjoint pair seeds
    import bench
    # two replicas, 10 steps of 307200 px each, slowest 120 ms
    assert bench.replica_throughput(2, 10, 307200, 120.0) == pytest.approx(2 * 10 * 307200 / 0.120)


def test_replica_seeds_are_disjoint():
    import bench
    seeds = {bench.replica_seed(r, i) for r in range(8) for i in range(64)}
    assert len(seeds) == 8 * 64
