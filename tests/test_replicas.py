"""Multi-GPU replicas (one process per GPU, independent instances, no data-path
collective): the sharding of instances over ranks and the whole-job timing, run as
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from synth.problems import Workload
    B = 4
    off = bench.replica_offset(rank, B)
    wl = Workload("q4_16")
    xis = wl.query_thetas(B, offset=off)
    ms_local = 10.0 + 5.0 * rank  # rank 1 is the slowest
    dist.barrier()
    ms = bench.max_over_ranks(ms_local, dist, device="cpu")
    q.put((rank, off, xis.tolist(), ms, bench.job_value(ms, world, B)))
    dist.destroy_process_group()


def test_two_replicas_shard_instances_and_time_the_slowest():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, off0, x0, ms0, v0), (r1, off1, x1, ms1, v1) = out
    assert (off0, off1) == (0, 4)
    # distinct instances per rank, identical to the global seeded sequence
    from synth.problems import Workload
    allx = Workload("q4_16").query_thetas(8).tolist()
    assert x0 == allx[:4] and x1 == allx[4:]
    assert ms0 == ms1 == 15.0
    assert abs(v0 - 2 * 4 / 0.015) < 1e-9 and v0 == v1
