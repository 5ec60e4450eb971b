"""The N > 1 bench path on CPU: two gloo ranks, as torchrun would launch them.

Replicas run independent solves, so the only cross-rank steps are the
barrier, the job time (maximum over ranks) and the work done (sum over
ranks); the reference arm runs on rank 0 alone.
"""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        ms, iters = bench.combine_over_ranks(10.0 + 5.0 * rank, 100 * (rank + 1), torch.device("cpu"), world)
        dist.barrier()

        class A:
            gpus, steps, warmup = world, 1, 0

        ref_rc = bench.run_reference(A()) if rank != 0 else 0
        out[rank] = (ms, iters, ref_rc)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_max_time_and_summed_work():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, iters, ref_rc = res[rank]
        assert ms == 15.0                    # the slowest rank's time
        assert iters == 300.0                # 100 + 200 evaluations
        assert ref_rc == 0                   # the reference arm exits 0 without work on rank != 0
