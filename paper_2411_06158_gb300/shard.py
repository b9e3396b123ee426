"""List-sharded search over torch.distributed ranks (Section 5, distributed deployment).

Every rank holds one shard of the IVF lists (``mrq_index_shard``: the global
statistics and all centroids, the members of its own lists), searches the same
queries with the same k, nprobe and options, and the ranks exchange their
answers once (``all_gather`` of the per-rank ids and distances) before the
library merges them (``mrq_merge_topk``).  Argument marshalling and the exchange
only: the search and the merge run in libmrq.

With device tensors the exchange runs on the process group's backend (NCCL);
with host arrays it needs a CPU backend (gloo).
"""
from __future__ import annotations

import numpy as np

from . import mrq_merge_topk, mrq_search


def exchange_and_merge(ids, dists, k: int, group=None):
    """All ranks' (nq, k) answers gathered and merged into the k smallest (dist, id)
    per query; every rank returns the same merged answer, in the kind of memory the
    inputs were in."""
    import torch
    import torch.distributed as dist

    host = not (isinstance(ids, torch.Tensor) and ids.is_cuda)
    ti = torch.as_tensor(np.ascontiguousarray(ids, dtype=np.int64)) if host and not \
        isinstance(ids, torch.Tensor) else ids.contiguous()
    td = torch.as_tensor(np.ascontiguousarray(dists, dtype=np.float32)) if host and not \
        isinstance(dists, torch.Tensor) else dists.contiguous()
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ti) for _ in range(world)]
    gd = [torch.empty_like(td) for _ in range(world)]
    dist.all_gather(gi, ti, group=group)
    dist.all_gather(gd, td, group=group)
    si, sd = torch.stack(gi), torch.stack(gd)
    if host:
        mi, md = mrq_merge_topk(si.numpy(), sd.numpy(), k)
        return mi, md
    return mrq_merge_topk(si, sd, k, stream=torch.cuda.current_stream(si.device))


def search(shard_index, queries, k: int, nprobe: int, opts=None, group=None):
    """One sharded search: this rank's shard searched with ``mrq_search``, then
    ``exchange_and_merge``.  ``queries`` must be the same on every rank."""
    ids, dists = mrq_search(shard_index, queries, k, nprobe, opts)
    return exchange_and_merge(ids, dists, k, group)
