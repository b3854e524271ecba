"""The bench's multi-GPU host logic on CPU: two gloo ranks, each plotting its
own keys (weak scaling), the job time being the slowest rank's and the value
the nonces of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [100.0, 250.0][rank]          # rank 1 is the slow one
    value, ms_step = bench.aggregate(1 << 20, 5, ms_local, world, "cpu")
    q.put((rank, value, ms_step))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, ms_step in got:
        assert ms_step == pytest.approx(250.0 / 5)
        assert value == pytest.approx((1 << 20) * 5 * 2 / 0.25)


def test_single_rank_aggregate_has_no_collective():
    import bench
    value, ms_step = bench.aggregate(1 << 10, 4, 8.0, 1, "cpu")
    assert ms_step == 2.0 and value == pytest.approx((1 << 10) * 4 / 0.008)
