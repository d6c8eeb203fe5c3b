"""Multi-rank host logic of the data-parallel path: an ensemble of independent domains is
split across ranks with no exchange between them (each rank advances its own domains in its
own context); a step's time is the slowest rank's. The ranks meet only in these host-side
reductions (torch.distributed, any backend)."""
import heapq


def shard_domains(cells, world):
    """Assign domains (cell counts `cells`) to `world` ranks, largest first to the rank with
    the fewest cells so far (ties to the lower rank): a deterministic partition that every
    rank computes identically. Returns one list of domain indices per rank, each ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for d in sorted(range(len(cells)), key=lambda i: (-cells[i], i)):
        load, r = heapq.heappop(heap)
        out[r].append(d)
        heapq.heappush(heap, (load + cells[d], r))
    return [sorted(s) for s in out]


def max_over_ranks(x, dist=None, device=None):
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
