"""The multi-GPU form of this path is replicas only (independent right-hand sides, no data
exchange). What bench.py does across ranks is checked here on CPU with two gloo ranks: the
timing reported is the maximum over ranks and every replica draws a different right-hand side."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2210_11797_gb300 import inputs as I
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
        rub, _rpi = I.draw_rhs(64, bench.replica_rhs_seed(rank), "normal")
        digest = torch.tensor([float(rub.sum())], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, digest)
        out[rank] = (ms, [float(g.item()) for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_differ_in_rhs(repo_root):
    import sys
    if repo_root not in sys.path:
        sys.path.insert(0, repo_root)
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        ms, digests = out[rank]
        assert ms == 15.0                     # the maximum over the two ranks, on both
        assert digests[0] != digests[1]       # independent right-hand sides
