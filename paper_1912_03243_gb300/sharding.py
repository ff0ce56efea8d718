"""Branch sharding of the decomposition path across processes (Sec. 4: every
term of the Eq. 3 sum is independent; the paper distributes them over MPI
ranks).

The 2^S branches are split into 2^p parts by their low p bits
(p = ceil(log2(world))); rank r takes the parts r, r + world, ...  The
library sums a rank's parts on its GPU in FP64 (sv_cut_amplitudes_parts);
this module only assigns the parts and runs the one collective of the path,
an FP64 all-reduce of the m complex amplitudes.
"""

from __future__ import annotations

import math

import numpy as np


def parts_for_rank(rank: int, world: int) -> tuple[int, list[int]]:
    """(nparts_log2, the parts this rank sums)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    p = max(0, math.ceil(math.log2(world)))
    return p, [part for part in range(1 << p) if part % world == rank]


def sharded_sum(rank_sum_fn, m: int, group=None) -> np.ndarray:
    """rank_sum_fn(nparts_log2, parts) -> complex128[m] is this rank's share
    of the sum (the library's sv_cut_amplitudes_parts, or a CPU stand-in in
    tests); the shares are all-reduced (FP64) across the process group and
    every rank returns the full sum."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    p, parts = parts_for_rank(rank, world)
    share = np.ascontiguousarray(rank_sum_fn(p, parts), dtype=np.complex128)
    if share.shape != (m,):
        raise ValueError(f"rank {rank}: share of shape {share.shape}, expected ({m},)")
    buf = torch.from_numpy(share.view(np.float64).copy())
    if dist.get_backend(group) == "nccl":
        buf = buf.cuda()
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf.cpu().numpy().view(np.complex128).copy()


def cut_amplitudes_sharded(circuit, n: int, mask_a: int, z, form: int = 0, group=None) -> np.ndarray:
    """<z|C|0> for the bit strings z, the branches shared among the ranks of
    the process group (one GPU per rank)."""
    from paper_1912_03243_gb300 import sv

    zz = np.ascontiguousarray(z, dtype=np.uint64)
    return sharded_sum(lambda p, parts: sv.sv_cut_amplitudes_parts(circuit, n, mask_a, zz, p, parts, form)[0],
                       zz.size, group)


def cut_amplitudes_multi_sharded(circuit, n: int, part_of, z_words, form: int = 0, group=None) -> np.ndarray:
    """The same over P partitions (z_words: (m, ceil(n/64)) uint64 bit
    strings)."""
    from paper_1912_03243_gb300 import sv

    zz = np.ascontiguousarray(z_words, dtype=np.uint64).reshape(-1, (n + 63) // 64)
    return sharded_sum(
        lambda p, parts: sv.sv_cut_amplitudes_multi_parts(circuit, n, part_of, zz, p, parts, form)[0],
        zz.shape[0], group)
