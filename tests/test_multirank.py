"""The N > 1 bench path on CPU with gloo: ranks solve independent problems and
only their timings are combined (max of elapsed time, sum of iterations)."""
import os
import socket



def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed, units = bench.reduce_over_ranks(torch, 10.0 + rank, 200 * (rank + 1), world, "cpu")
    q.put((rank, elapsed, units))
    dist.destroy_process_group()


def test_timing_reduction_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time and the total units of the job
    assert res == [(0, 11.0, 600.0), (1, 11.0, 600.0)]


def test_single_rank_is_identity():
    import torch
    import bench
    assert bench.reduce_over_ranks(torch, 3.5, 7, 1, "cpu") == (3.5, 7.0)
