"""The benchmark's multi-rank plumbing on CPU ranks (gloo, world size 2):
replicas time their own work and the job's time is the maximum over ranks;
each rank's integrand parameters are the same seeded draw."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import sg_inputs as si
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench._dist()
    t = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))
    params = si.cfg2()["params"]
    q.put((r, ws, local, t, float(params.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_take_max_time_and_same_inputs():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == world for o in out)
    assert all(o[3] == 11.0 for o in out)        # maximum over the two ranks
    assert out[0][4] == out[1][4]                 # identical seeded draw on every replica


def test_single_process_time_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
