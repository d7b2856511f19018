"""The multi-GPU form is replicas only: each rank solves its own copy of the
workload and the job's time per step is the slowest rank's. This checks the
rank logic of bench.py with two gloo processes on the CPU (no GPU, no
collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        os.environ["RANK"], os.environ["WORLD_SIZE"], os.environ["LOCAL_RANK"] = str(rank), str(world), str(rank)
        ws, r, local = bench.dist_env()
        mine = 10.0 * (rank + 1)                     # rank 1 is the slow one
        dist.barrier()
        got = bench.max_over_ranks(mine, dist, "cpu")
        out.put((rank, ws, r, local, got))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    mp = torch.multiprocessing.get_context("spawn")
    out = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2, 2]
    assert [(r[2], r[3]) for r in res] == [(0, 0), (1, 1)]
    assert all(r[4] == 20.0 for r in res)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
