"""One flow integrated on several GPUs: the vertex right-hand side split by stored (s, u) pairs.

The paper distributes the flow over compute nodes in superblocks (Sec. 4.4): all transfer
frequencies t, spin components and sites of one (s, u) pair are computed together, and the
self-energy flow is broadcast.  Here every rank (one GPU each) holds the whole state (the
lookups touch arbitrary entries), computes the self-energy flow itself (N values, cheap,
instead of a broadcast) and the vertex flow of one contiguous range of stored pairs
(sr_flow_rhs_pairs: a contiguous slice of the state layout), then one all-gather assembles
the slices and every rank applies the same Euler update (sr_flow_advance).  Every entry is
computed by exactly one rank with the same kernels as on one GPU, so the sharded flow is bit
for bit the single-GPU flow.

The collective goes through torch.distributed (NCCL between GPUs; gloo for the CPU tests).
"""
from __future__ import annotations


def pair_ranges(npair: int, world_size: int):
    """Contiguous ranges of stored pairs, one per rank, sizes differing by at most one."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    base, extra = divmod(npair, world_size)
    out, p = [], 0
    for r in range(world_size):
        n = base + (1 if r < extra else 0)
        out.append((p, p + n))
        p += n
    return out


class ShardedFlow:
    """Euler stepping of `flow` with its vertex right-hand side split over the ranks of a
    torch.distributed process group.  `flow` provides npair, N, ts, n_gamma, entries_per_pair,
    lam, rhs_pairs(lam, p0, p1, dsigma, dgamma) and advance(lam_next, dsigma, dgamma) (the
    library's Flow does); tensors live on `device`."""

    def __init__(self, flow, group=None, device=None):
        import torch
        import torch.distributed as dist
        self.flow = flow
        self.group = group
        self.ws = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.ranges = pair_ranges(flow.npair, self.ws)
        # equal-size slices for the collective: the largest range, padded
        self.chunk = max(p1 - p0 for p0, p1 in self.ranges) * flow.entries_per_pair
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = device
        self.dsigma = torch.empty(flow.N * flow.ts, dtype=torch.float64, device=device)
        # assembled right-hand side in the state layout (rank r's slice starts at its first
        # pair's entry p0(r) * entries_per_pair); the all-gather exchanges ws equal chunks
        self.dgamma = torch.zeros(flow.n_gamma * flow.ts, dtype=torch.float64, device=device)
        self.recv = torch.empty(self.ws * self.chunk, dtype=torch.float64, device=device)
        self.send = torch.zeros(self.chunk, dtype=torch.float64, device=device)

    @property
    def my_pairs(self):
        return self.ranges[self.rank]

    def rhs(self, lam: float):
        """The whole right-hand side at lam (dsigma, dgamma views), assembled from the ranks."""
        import torch.distributed as dist
        fl = self.flow
        p0, p1 = self.my_pairs
        fl.rhs_pairs(lam, p0, p1, self.dsigma, self.dgamma)
        n = fl.n_gamma * fl.ts
        if self.ws > 1:
            e = fl.entries_per_pair
            self.send[:(p1 - p0) * e] = self.dgamma[p0 * e:p1 * e]
            parts = list(self.recv.split(self.chunk))
            dist.all_gather(parts, self.send, group=self.group)
            for (q0, q1), part in zip(self.ranges, parts):
                self.dgamma[q0 * e:q1 * e] = part[:(q1 - q0) * e]
        return self.dsigma, self.dgamma[:n]

    def step(self, lam_next: float):
        """One Euler step of the whole flow (Sec. 4.3) to lam_next."""
        dsig, dG = self.rhs(self.flow.lam)
        self.flow.advance(lam_next, dsig, dG)
