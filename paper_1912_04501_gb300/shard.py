"""A solve sharded by target across processes, one GPU each.

The near sum (the dominant cost of an operator application, Sec. 6.2 step 1)
splits by target: every process holds the whole cell (geometry, proxy fit
and density replicated), evaluates the rows of its own bodies, and after
each application the owned slices are all-gathered so that every process
holds the same full vector; GMRES, the wall discrepancy, the proxy fit and
the extraction then run replicated and bit-identical everywhere.  This module
holds the host side: the partition of the bodies and the exchange the
library calls (bie_set_partition); every arithmetic step stays in the
library's kernels.
"""
import ctypes

import numpy as np

EXCHANGE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)


def partition(body_nodes, world):
    """Contiguous ranges of whole bodies, one per rank, balanced by their
    node counts (the targets of the near sum): rank r gets bodies
    [b[r], b[r + 1]); returns the body bounds and the node ranges."""
    counts = np.asarray(body_nodes, dtype=np.int64)
    if world < 1 or world > len(counts):
        raise ValueError("need 1 <= world <= number of bodies")
    cum = np.concatenate([[0], np.cumsum(counts)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        b = int(np.searchsorted(cum, target))
        if b > 0 and abs(cum[b - 1] - target) <= abs(cum[b] - target):
            b -= 1
        b = min(max(b, bounds[-1] + 1), len(counts) - (world - r))
        bounds.append(b)
    bounds.append(len(counts))
    nodes = [(int(cum[bounds[r]]), int(cum[bounds[r + 1]])) for r in range(world)]
    return bounds, nodes


def gather_slices(y, node_ranges, rank, group=None):
    """All-gather of the owned slices of a torch vector y of 2N entries
    (node-major): rank r's rows 2 n0 .. 2 n1 of node range (n0, n1) are
    copied into every other rank's y.  Slices are padded to the longest."""
    import torch
    import torch.distributed as dist
    longest = max(2 * (b - a) for a, b in node_ranges)
    a, b = node_ranges[rank]
    mine = torch.zeros(longest, dtype=y.dtype, device=y.device)
    mine[: 2 * (b - a)] = y[2 * a: 2 * b]
    bufs = [torch.empty_like(mine) for _ in node_ranges]
    dist.all_gather(bufs, mine, group=group)
    for r, (a, b) in enumerate(node_ranges):
        if r != rank:
            y[2 * a: 2 * b] = bufs[r][: 2 * (b - a)]
    return y


class _DeviceVector:
    """A CUDA array of float64 at a raw device pointer (zero-copy view)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3}


class ShardedSolve:
    """Attach a target partition to a Context (one process per GPU, an
    initialised torch.distributed process group over all ranks)."""

    def __init__(self, ctx, body_nodes, rank, world, group=None):
        import torch
        self.ctx, self.rank, self.world, self.group = ctx, rank, world, group
        self.bounds, self.nodes = partition(body_nodes, world)
        self.errors = []

        import torch.distributed as dist
        on_host = dist.get_backend(group) == "gloo"  # a CPU process group gathers host copies

        def exchange(ptr, n2, user):
            try:
                y = torch.as_tensor(_DeviceVector(ptr, n2), device="cuda")
                if on_host:
                    h = y.cpu()
                    gather_slices(h, self.nodes, self.rank, self.group)
                    y.copy_(h)
                else:
                    gather_slices(y, self.nodes, self.rank, self.group)
                torch.cuda.synchronize()
                return 0
            except Exception as e:  # reported through the library's error code
                self.errors.append(repr(e))
                return 1

        self._cb = EXCHANGE(exchange)  # kept alive as long as the partition is set
        ctx.set_partition(self.bounds[rank], self.bounds[rank + 1], self._cb)

    def close(self):
        self.ctx.set_partition(0, self.ctx.n_bodies, None)
        self._cb = None
