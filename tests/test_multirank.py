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


# ---------------------------------------------------------------------------
# sharded batches: each rank holds the long-accumulator limbs of its part of
# the chunk queue; the ranks exchange them (all_gather) and combine
# ---------------------------------------------------------------------------

def _chunk_values(n_items, n_chunks, seed):
    """Chunk sums of a synthetic batch: heavy cancellation and 40 binades,
    so that a rounding anywhere in the combine would show."""
    import numpy as np
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n_items, n_chunks)) * 10.0 ** rng.uniform(-20, 20, (n_items, n_chunks))
    v[:, 1::2] = -v[:, 0::2] * (1 + 1e-12 * rng.standard_normal(v[:, 1::2].shape))  # near-cancelling pairs
    return v


def _shard_parts(vals, lo, hi):
    import numpy as np
    import index_check
    parts = np.zeros((vals.shape[0], 64), dtype=np.int64)
    for k in range(vals.shape[0]):
        parts[k, :32] = index_check.lacc_limbs(vals[k, lo:hi])
        parts[k, 32:] = index_check.lacc_limbs(np.abs(vals[k, lo:hi]))
    return parts


def _info(n):
    import paper_2210_14313_gb300 as sg
    info = (sg.sg_shard_info * n)()
    for k in range(n):
        info[k].mult, info[k].base_rel, info[k].scale_m = 1.0 + k / 7.0, 0.5, 1.0
        info[k].scale_e2, info[k].unit_roundoff, info[k].points, info[k].evals = -k, 2.0 ** -53, 100, 90
    return info


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import paper_2210_14313_gb300 as sg
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vals = _chunk_values(6, 300, 17)
    lo, hi = vals.shape[1] * rank // world, vals.shape[1] * (rank + 1) // world
    mine = torch.from_numpy(_shard_parts(vals, lo, hi))
    gathered = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine)
    res = sg.shard_combine([g.numpy() for g in gathered], _info(vals.shape[0]))
    q.put((rank, [(r.mant, r.exp2, r.cond) for r in res]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_combine_shards_bitwise_like_one():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import paper_2210_14313_gb300 as sg
    vals = _chunk_values(6, 300, 17)
    one = [(r.mant, r.exp2, r.cond) for r in sg.shard_combine([_shard_parts(vals, 0, 300)], _info(6))]
    three = [(r.mant, r.exp2, r.cond) for r in
             sg.shard_combine([_shard_parts(vals, a, b) for a, b in ((0, 77), (77, 200), (200, 300))], _info(6))]
    assert out[0] == out[1] == one == three
    # and the combine is the exact sum, rounded: item value = mult (base_rel + sum) 2^-k
    from fractions import Fraction
    for k, (mant, e, _) in enumerate(one):
        tot = sum((Fraction(float(x)) for x in vals[k]), Fraction(0))
        ref = (1 + k / 7.0) * (0.5 + float(tot)) * 2.0 ** -k
        assert abs(mant * 2.0 ** e - ref) <= 2e-16 * abs(ref)
