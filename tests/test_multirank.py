"""The N-GPU benchmark runs one replica per rank (realisations are independent; the path
has no data exchange) and combines only the timing: max step time over ranks, summed cell
updates.  Checked with world_size 2 on the gloo backend (CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [1.5, 2.0][rank]  # rank 1 is the slower replica
    got = bench.combine_ranks(ms, 65536, "cpu")
    out.put((rank, got))
    dist.destroy_process_group()


def test_combine_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = res[r]
        assert ms == pytest.approx(2.0)
        assert value == pytest.approx(2 * 65536 / 2.0e-3)
