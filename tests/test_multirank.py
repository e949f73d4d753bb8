"""Host logic of the multi-GPU benchmark path, on CPU with two gloo ranks: rays are
sharded (each rank draws disjoint seeded batches, no data-path collective) and the
timing aggregates the maximum step time and the total ray count over ranks."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_2210_04847_gb300 import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        batches = bench.rank_batches(r)
        o, d, t = synth.bounded_rays(0, 64, batch=batches[0])
        step_ms = 1.0 + r  # rank-dependent step time
        mx = bench.max_over_ranks(step_ms, w, "cpu")
        tot = bench.sum_over_ranks(64.0, w, "cpu")
        q.put((r, batches, o[:2].tolist(), mx, tot))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, o0, mx0, t0), (r1, b1, o1, mx1, t1) = out
    assert set(b0).isdisjoint(b1)  # disjoint ray batches: no shared work, no exchange
    assert o0 != o1
    assert mx0 == mx1 == 2.0  # max over ranks of the step time
    assert t0 == t1 == 128.0  # rays of all ranks


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5 and bench.sum_over_ranks(7.0, 1) == 7.0
    assert bench.rank_batches(0) != bench.rank_batches(1)
