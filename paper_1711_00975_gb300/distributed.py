"""Several GPUs on one stream: shard by particle index, sum the sketches.

Count Sketches built with the same parameters on disjoint parts of a stream sum
to the sketch of the whole stream (arXiv:1711.00975 Sec. 5: "all the sketches
can be summed").  Each rank seeks its sketch to the global index of its first
particle (so sampling decisions do not change), updates it with its shard, then
one all-reduce (sum) of the t x W int32 counters gives every rank the counters
of the whole stream; the top-k search follows on any rank.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """(first global index, count) of rank's contiguous shard of n particles."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    lo = n * rank // world
    hi = n * (rank + 1) // world
    return lo, hi - lo


def allreduce_counters(counters, group=None) -> None:
    """Sum int32 counters (a torch tensor, any device) over the process group in
    place.  int32 addition wraps the same way as the sketch's own counters."""
    import torch.distributed as dist
    dist.all_reduce(counters, op=dist.ReduceOp.SUM, group=group)


def merge_sketch_across_ranks(sketch, group=None) -> None:
    """Replace a library sketch's counters with their sum over the group
    (sketch_counters -> all-reduce -> sketch_load_counters, device-resident)."""
    import torch
    out = torch.empty((sketch.rows, sketch.width), dtype=torch.int32, device="cuda")
    from .halosketch import sketch_counters, sketch_load_counters
    sketch_counters(sketch.h, out)
    allreduce_counters(out, group)
    sketch_load_counters(sketch.h, out)
