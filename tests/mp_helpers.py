"""Worker functions for the multi-process (gloo, CPU) tests; spawned
processes import this module by name."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _init(rank, world, port):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def sharded_oracle_sum(rank, world, port, circuit_text, n, mask, z, form, out_path):
    import numpy as np

    import oracle
    from paper_1912_03243_gb300 import sharding

    dist = _init(rank, world, port)
    zz = np.asarray(z, dtype=np.uint64)

    def share(p, parts):  # CPU stand-in for sv_cut_amplitudes_parts, same signature
        return sum(oracle.cut_amplitudes_part(circuit_text, mask, zz, part, p, form=form, n=n)[0] for part in parts)

    total = sharding.sharded_sum(share, zz.size)
    if rank == 0:
        np.save(out_path, total)
    dist.barrier()
    dist.destroy_process_group()


def bench_max(rank, world, port, out_path):
    import json

    import bench

    dist = _init(rank, world, port)
    v = bench.max_over_ranks(world, float(10 + rank))
    bench.barrier(world)
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"max": v}, f)
    dist.destroy_process_group()


def sharded_oracle_multi_sum(rank, world, port, circuit_text, n, part_of, z, out_path):
    import numpy as np

    import oracle
    from paper_1912_03243_gb300 import sharding

    dist = _init(rank, world, port)

    def share(p, parts):  # CPU stand-in for sv_cut_amplitudes_multi_parts, same signature
        return sum(oracle.cut_amplitudes_multi(circuit_text, part_of, z, part=part, nparts_log2=p, n=n)[0]
                   for part in parts)

    total = sharding.sharded_sum(share, len(z))
    if rank == 0:
        np.save(out_path, total)
    dist.barrier()
    dist.destroy_process_group()


def sharded_library_sum(rank, world, port, circuit_text, n, mask, z, form, out_path):
    """Each rank sums its branch parts with the library on cuda:0 (ranks share
    the one GPU; their kernels are independent) and the shares meet in one
    gloo all-reduce on the host."""
    import numpy as np
    import torch

    from paper_1912_03243_gb300 import sharding

    torch.cuda.set_device(0)
    dist = _init(rank, world, port)
    total = sharding.cut_amplitudes_sharded(circuit_text, n, mask, np.asarray(z, dtype=np.uint64), form=form)
    torch.cuda.synchronize()
    if rank == 0:
        np.save(out_path, total)
    dist.barrier()
    dist.destroy_process_group()
