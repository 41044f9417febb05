"""The replica driver of bench.py (one process per GPU, no collective on the data
path) on two gloo ranks on the CPU: process-group set-up from the torchrun
environment, the barrier around the timed region, the maximum of the ranks' times and
the sum of their units, and the reference arm doing its work on rank 0 only."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist
    r, ws = bench.dist_setup()
    bench.barrier(ws)
    t_max = bench.allreduce_max(0.5 + rank, ws)        # per-rank seconds
    units = bench.allreduce_sum(1000.0 * (rank + 1), ws)  # per-rank units processed
    bench.barrier(ws)
    # the reference arm returns at once on every rank but 0 (checked without running it)
    skipped = bench.run_reference(None, r, ws) is None if r != 0 else True
    dist.destroy_process_group()
    q.put((r, ws, t_max, units, skipped))


def test_replica_reductions_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, ws, t_max, units, skipped in out:
        assert ws == 2 and t_max == 1.5 and units == 3000.0 and skipped
