"""Host logic of bench.py's multi-GPU mode on CPU ranks (gloo, world size 2): each rank
times its own batch (weak scaling, distinct seeds) and the job's time is the maximum over
ranks.  No GPU and no collective on the data path are involved."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 1.5 + rank * 2.0                       # rank 1 is the slow one
    mx = bench.combine_max(local, dist, "cpu")
    seed = bench.rank_batch_seed(2, rank)
    out.put((rank, mx, seed))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_distinct_batches():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [3.5, 3.5]
    assert res[0][2] != res[1][2]


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_max(2.25, None, "cpu") == 2.25
