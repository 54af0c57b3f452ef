"""Run under torch.distributed.run (gloo, on the host): every rank passes its
own time to bench.max_over_ranks and prints what it got back as JSON."""
import json
import os
import sys

import torch.distributed as dist

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
got = bench.max_over_ranks(1.5 + 2.0 * rank, world)
print(json.dumps({"rank": rank, "world": world, "max": got}), flush=True)
dist.destroy_process_group()
