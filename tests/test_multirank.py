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


def test_launcher_starts_two_gloo_ranks(capfd):
    # bench.spawn_ranks is the path `bench.py --gpus N` takes without an
    # outer launcher: N ranks under torch.distributed.run on 127.0.0.1.
    import json

    import bench
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rank_child.py")
    rc = bench.spawn_ranks(2, [child])
    out = capfd.readouterr().out
    assert rc == 0, out
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["world"] == 2
    assert d["ms_step"] == pytest.approx(250.0 / 5)
    assert d["value"] == pytest.approx((1 << 20) * 5 * 2 / 0.25)


def test_gpus_beyond_visible_devices_fails_loudly():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    n = max(2, torch.cuda.device_count() + 1)
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", str(n),
                        "--steps", "1", "--warmup", "3"], cwd=root, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "CUDA device" in r.stderr
