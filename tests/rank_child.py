"""One rank of the bench launcher test: started by bench.spawn_ranks under
torch.distributed.run (gloo, CPU), it reads its rank from the launcher's
environment, plays a rank whose local time is 100 + 150 * rank ms, and rank
0 prints the aggregated value as JSON."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402

world, rank, local = bench.rank_env()
dist.init_process_group("gloo")
value, ms_step = bench.aggregate(1 << 20, 5, 100.0 + 150.0 * rank, world, "cpu")
if rank == 0:
    print(json.dumps({"world": world, "value": value, "ms_step": ms_step}), flush=True)
dist.barrier()
dist.destroy_process_group()
