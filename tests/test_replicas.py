"""The benchmark's N > 1 path, on CPU with the gloo backend (world size 2): one process per
replica, each with its own seeded workload and no collective on the data path; the step time
is the maximum over ranks and the units are summed.  Under torchrun the reference arm runs on
rank 0 alone."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                          WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
        sys.path.insert(0, ROOT)
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import bench
        r, w, local = bench.dist_env()
        ms, units = bench.combine_ranks(10.0 + rank, 100.0 * (rank + 1), "cpu")
        seeds = bench.workload_seeds(r)

        class Args:
            steps, warmup, gpus = 1, 0, world
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.run_reference(Args, r) if r != 0 else 0  # rank 0's oracle run is too long here
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, r, w, local, ms, units, seeds, rc, buf.getvalue()))
    except Exception as e:  # reported to the parent
        q.put((rank, "error", repr(e)))


def test_two_replicas_on_gloo():
    pytest.importorskip("torch")
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        item = q.get(timeout=120)
        assert item[1] != "error", item
        out[item[0]] = item
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        _, r, w, local, ms, units, seeds, rc, printed = out[rank]
        assert (r, w, local) == (rank, 2, rank)
        assert ms == 11.0 and units == 300.0  # max of 10, 11; sum of 100, 200
        assert rc == 0
    assert out[0][6] != out[1][6]                 # each replica has its own workload
    assert out[1][8] == ""                        # rank 1 prints nothing in the reference arm


def test_single_process_combine_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(3.5, 7.0, "cpu") == (3.5, 7.0)
