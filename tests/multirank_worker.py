"""One rank of the world-size-2 check in tests/test_multirank.py: gloo on the CPU, launched by
torch.distributed.run exactly as bench.py is for N > 1 (rank, world size and rendezvous from
the environment).  Rank 0 prints one JSON line."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402

rank, world, local = bench.dist_env()
dist.init_process_group("gloo")
bench.barrier()
# every rank contributes its own value; all must see the largest
top = bench.max_over_ranks(1.5 + 2.0 * rank)
seen = [None] * world
dist.all_gather_object(seen, top)
bench.barrier()
if rank == 0:
    print(json.dumps({"world": world, "local": local, "max": top, "seen": seen}))
dist.destroy_process_group()
