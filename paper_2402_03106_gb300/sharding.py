"""Multi-GPU sharding of a render: one process per GPU.

Paths are independent and every random number is keyed by the global path
id, so rank r of W traces the ids [r * N, (r + 1) * N) (weak scaling, N paths
per rank) and the per-rank histogram estimates are averaged with one FP64
sum all-reduce -- the only exchange the method has.  The result equals a
single render of W * N paths up to FP64 summation order.
"""
from __future__ import annotations


def path_offset(rank: int, paths_per_rank: int) -> int:
    """First global path id of `rank`."""
    return int(rank) * int(paths_per_rank)


def combine(hist, world_size: int, group=None):
    """Average per-rank histogram estimates in place (sum all-reduce / W)."""
    if world_size > 1:
        import torch.distributed as dist
        dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
        hist.div_(world_size)
    return hist


class PipelinedCombine:
    """The combine of step k - 1 overlapped with the render of step k.

    Two histogram buffers alternate.  `begin_step()` starts the all-reduce
    of the previous step's histogram (asynchronous, ordered after the work
    already queued on the stream) and returns the other buffer for this
    step's render; `end_step()` waits for that all-reduce (a wait on the
    stream under NCCL, on the host under gloo), so every exchange completes
    within the step that overlaps it.  `finish()` exchanges the last step's
    histogram, waits, and returns the ranks' average of that step.  With one
    rank there is nothing to exchange: one buffer, no collective.
    """

    def __init__(self, make_buffer, world_size: int, group=None):
        self.world_size = int(world_size)
        self.group = group
        n = 2 if self.world_size > 1 else 1
        self.buffers = [make_buffer() for _ in range(n)]
        self.step = 0
        self.prev = None      # histogram of the previous step, not yet exchanged
        self.work = None      # the all-reduce in flight

    def _reduce(self, hist):
        import torch.distributed as dist
        return dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=self.group, async_op=True)

    def begin_step(self):
        if self.world_size > 1 and self.prev is not None:
            self.work = self._reduce(self.prev)
        buf = self.buffers[self.step % len(self.buffers)]
        self.step += 1
        return buf

    def end_step(self, hist):
        if self.work is not None:
            self.work.wait()
            self.work = None
        self.prev = hist

    def finish(self):
        last = self.prev
        if last is not None and self.world_size > 1:
            self._reduce(last).wait()
            last.div_(self.world_size)
        self.prev = None
        return last


def sharded_gradient(render_fn, adjoint_fn, loss_grad_fn, world_size: int, group=None):
    """One gradient evaluation of a histogram loss across ranks.

    Each rank renders its path-id shard (`render_fn() -> h_r`) and the
    estimates are averaged (the first exchange: the histogram, since dL/dh
    needs the whole image).  Every rank then forms the same loss weights
    `w = loss_grad_fn(h)`, replays its own shard with an independent seed
    (`adjoint_fn(w) -> g_r`, three values) and the gradients are averaged
    (the second exchange: three numbers).  Returns (h, g).
    """
    h = combine(render_fn(), world_size, group)
    g = adjoint_fn(loss_grad_fn(h))
    return h, combine(g, world_size, group)
