"""Run under torch.distributed.run (gloo, on the host): every rank passes its
own time to bench.max_over_ranks and writes what it got back as JSON to
<out_dir>/rank<r>.json (one file per rank: the ranks' standard outputs
interleave)."""
import json
import os
import sys

import torch.distributed as dist

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

out_dir = sys.argv[1]
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
got = bench.max_over_ranks(1.5 + 2.0 * rank, world)
with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
    json.dump({"rank": rank, "world": world, "max": got}, f)
dist.destroy_process_group()
