"""Several GPUs on one stream: shard by particle index, sum the sketches.

Count Sketches built with the same parameters on disjoint parts of a stream sum
to the sketch of the whole stream (arXiv:1711.00975 Sec. 5: all the sketches
can be summed).  Each rank seeks its sketch to the global index of its first
particle (so sampling decisions and the probe of the stream's first particles
do not change), updates it with its shard, then one all-reduce (sum) of the
t x W int32 counters gives every rank the counters of the whole stream; the
top-k search follows on the root rank, whose shard holds the stream's first
particles.
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


class ShardedSketch:
    """One rank's part of a sketch of a stream split by particle index.

    update(shard) adds this rank's contiguous shard [lo, lo + count); merge()
    sums the counters over the group (device-resident buffer, reused);
    topk(k) merges then searches on the root rank and returns (keys, est)
    there, None elsewhere."""

    def __init__(self, sketch, n_total: int, rank: int, world: int, group=None, root: int = 0):
        import torch
        self.sketch = sketch
        self.rank, self.world, self.group, self.root = rank, world, group, root
        self.lo, self.count = shard_range(n_total, rank, world)
        self.buf = torch.empty((sketch.rows, sketch.width), dtype=torch.int32,
                               device=torch.device("cuda", torch.cuda.current_device()))

    def reset(self) -> None:
        self.sketch.reset()
        self.sketch.seek(self.lo)

    def update(self, shard, rate: float = 1.0) -> None:
        """Add this rank's shard (host or device; `count` particles)."""
        self.sketch.update(shard, self.count, rate)

    def merge(self) -> None:
        """Counters of the whole stream on every rank (no-op for one rank)."""
        if self.world > 1:
            from .halosketch import sketch_counters, sketch_load_counters
            sketch_counters(self.sketch.h, self.buf)
            allreduce_counters(self.buf, self.group)
            sketch_load_counters(self.sketch.h, self.buf)

    def topk(self, k: int):
        self.merge()
        if self.rank != self.root:
            return None
        return self.sketch.topk(k)


def merge_sketch_across_ranks(sketch, group=None) -> None:
    """Replace a library sketch's counters with their sum over the group
    (sketch_counters -> all-reduce -> sketch_load_counters, device-resident)."""
    import torch
    out = torch.empty((sketch.rows, sketch.width), dtype=torch.int32,
                      device=torch.device("cuda", torch.cuda.current_device()))
    from .halosketch import sketch_counters, sketch_load_counters
    sketch_counters(sketch.h, out)
    allreduce_counters(out, group)
    sketch_load_counters(sketch.h, out)
