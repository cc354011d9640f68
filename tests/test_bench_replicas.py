"""The benchmark's replicas path on CPU: two gloo ranks (spawned processes, 127.0.0.1).

Under torchrun each rank compresses its own copy of the workload on its own GPU; the only
collectives are the barriers around the timed regions and the maximum of the ranks' times. Here
the ranks report different times and must agree on the slowest; the whole-job rate counts every
replica's bytes over that time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist

    bench.dist_init(world, backend="gloo")  # host-side test, with or without a GPU
    try:
        assert dist.get_backend() == "gloo"
        bench.barrier()
        slowest = bench.replica_max(10.0 + 3.0 * rank)  # ranks' own ms: 10, 13
        bench.barrier()
        out.put((rank, slowest, bench.whole_job_gbs(8e9, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_replicas_agree_on_slowest_time_and_whole_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(world))
    for r, slowest, gbs in got:
        assert slowest == 13.0
        assert gbs == pytest.approx(2 * 8e9 / 13e-3 / 1e9)


def test_single_process_needs_no_group():
    import bench

    assert bench.replica_max(7.5) == 7.5
    bench.barrier()  # no process group: nothing to wait for
    assert bench.whole_job_gbs(8e9, 1, 16.0) == pytest.approx(500.0)

