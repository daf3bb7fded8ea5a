"""One part of a partitioned function per rank (torch.distributed).

Sec. 4.3 notes that splitting the key set into partitions, each with its own
function, applies to this method too.  With one part per GPU that is the
multi-GPU form: every rank routes its share of the keys by part
(``mphf_route``), one all-to-all hands each rank the keys of its own part, the
rank builds that part's function with no further exchange, and one all-gather
of the part sizes gives every rank the global offsets (the prefix of the part
sizes).  A lookup routes the queries the same way, sends each to the rank
that owns its part, which answers with its function plus its offset
(``mphf_lookup`` + ``mphf_add_offset``); one all-to-all returns the answers
and ``mphf_unroute`` puts them back in query order.  The global indices are
those of ``mphf_build_partitioned`` over the union of the ranks' keys with
K = world size.

The device steps go through ``ops`` (by default the CUDA library); the
exchange and offset logic here is plain torch.distributed (NCCL on GPUs).
"""
from __future__ import annotations

import numpy as np


class CudaOps:
    """The device steps, run by the CUDA library."""

    def __init__(self, device="cuda"):
        import torch
        self.device = torch.device(device)

    def empty(self, n):
        import torch
        return torch.empty(int(n), dtype=torch.int64, device=self.device)

    def route(self, keys, K, part_seed, with_src):
        from . import mphf
        return mphf.route(keys, K, part_seed, with_src=with_src)

    def build(self, keys, gamma, levels, seed):
        from . import mphf
        return mphf.MPHF.build(keys, gamma=gamma, levels=levels, seed=seed)

    def lookup(self, f, keys):
        return f.lookup(keys)

    def add_offset(self, vals, offset):
        from . import mphf
        return mphf.add_offset(vals, offset)

    def unroute(self, vals, src):
        from . import mphf
        return mphf.unroute(vals, src)


def _counts(off: np.ndarray):
    return [int(x) for x in (off[1:] - off[:-1])]


class DistributedMPHF:
    """This rank's part of a function partitioned over the ranks of `group`."""

    def __init__(self, local_keys, part_seed: int = 0, gamma: float = 2.0, levels: int = 25,
                 seed: int = 0, group=None, ops=None):
        import torch
        import torch.distributed as dist
        self.ops = ops or CudaOps()
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.part_seed = int(part_seed)
        routed, _, off = self.ops.route(local_keys, self.world, self.part_seed, False)
        send = _counts(off)
        recv = self._exchange_counts(send)
        mine = self.ops.empty(sum(recv))
        dist.all_to_all_single(mine, routed, recv, send, group=group)
        self.function = self.ops.build(mine, gamma, levels, seed)
        sizes = [torch.zeros(1, dtype=torch.int64, device=self.ops.device)
                 for _ in range(self.world)]
        dist.all_gather(sizes, torch.tensor([mine.numel()], dtype=torch.int64,
                                            device=self.ops.device), group=group)
        self.offsets = np.zeros(self.world + 1, dtype=np.uint64)
        np.cumsum([int(t.item()) for t in sizes], out=self.offsets[1:])
        self.N = int(self.offsets[-1])

    def _exchange_counts(self, send):
        import torch
        import torch.distributed as dist
        s = torch.tensor(send, dtype=torch.int64, device=self.ops.device)
        r = torch.empty_like(s)
        dist.all_to_all_single(r, s, group=self.group)
        return [int(x) for x in r.tolist()]

    def lookup(self, queries):
        """Global indices of this rank's queries (collective: every rank of
        the group calls it, each with its own queries)."""
        import torch.distributed as dist
        routed, src, off = self.ops.route(queries, self.world, self.part_seed, True)
        send = _counts(off)
        recv = self._exchange_counts(send)
        mine = self.ops.empty(sum(recv))
        dist.all_to_all_single(mine, routed, recv, send, group=self.group)
        vals = self.ops.lookup(self.function, mine)
        self.ops.add_offset(vals, int(self.offsets[self.rank]))
        back = self.ops.empty(queries.numel())
        dist.all_to_all_single(back, vals, send, recv, group=self.group)
        return self.ops.unroute(back, src)
