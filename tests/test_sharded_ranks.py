"""The sharded flow's host logic (Sec. 4.4 superblocks: stored (s, u) pairs split over ranks,
one all-gather of the vertex right-hand side per step) with gloo ranks on the CPU.

The library's kernels need a GPU, so the ranks drive a stand-in flow with the same sharding
interface on CPU tensors: a state of npair superblocks and a deterministic right-hand side in
which every entry depends on the whole state (as the lattice sum and the frequency lookups
do), evaluated only for the requested pairs.  The sharded steps must reproduce the unsharded
steps bit for bit.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2109_13317_gb300.sharded import ShardedFlow, pair_ranges  # noqa: E402


class StandInFlow:
    def __init__(self, npair=37, per_pair=24, N=6, seed=3):
        g = torch.Generator().manual_seed(seed)
        self.npair, self.N, self.ts, self.entries_per_pair = npair, N, 1, per_pair
        self.n_gamma = npair * per_pair
        self.G = torch.randn(self.n_gamma, generator=g, dtype=torch.float64)
        self.gam = torch.randn(N, generator=g, dtype=torch.float64)
        self.mix = torch.randn(self.n_gamma, generator=g, dtype=torch.float64)
        self.lam = 2.0

    def rhs_pairs(self, lam, p0, p1, dsigma, dgamma):
        e = self.entries_per_pair
        idx = torch.arange(p0 * e, p1 * e)
        tot = self.G.sum()
        dsigma[:self.N] = torch.tanh(self.gam) * lam + tot * 1e-3
        dgamma[idx] = torch.sin(self.G[idx] * self.mix[idx]) * tot / self.n_gamma + \
            self.G[(idx * 7 + 3) % self.n_gamma] * 0.1 * lam

    def advance(self, lam_next, dsigma, dgamma):
        dl = self.lam - lam_next
        self.gam = self.gam - dl * dsigma[:self.N]
        self.G = self.G - dl * dgamma[:self.n_gamma]
        self.lam = lam_next


LAMS = [2.0, 1.7, 1.3, 1.1]


def _unsharded():
    f = StandInFlow()
    ds = torch.empty(f.N, dtype=torch.float64)
    dG = torch.empty(f.n_gamma, dtype=torch.float64)
    for lam in LAMS[1:]:
        f.rhs_pairs(f.lam, 0, f.npair, ds, dG)
        f.advance(lam, ds, dG)
    return f


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    f = StandInFlow()
    sf = ShardedFlow(f, device=torch.device("cpu"))
    assert (sf.ws, sf.rank) == (ws, rank)
    for lam in LAMS[1:]:
        sf.step(lam)
    out[rank] = (f.G.numpy().tobytes(), f.gam.numpy().tobytes(), sf.my_pairs)
    dist.destroy_process_group()


def test_pair_ranges_cover_every_pair_once():
    for npair in (1, 5, 36, 1176):
        for ws in (1, 2, 3, 7, 8):
            rg = pair_ranges(npair, ws)
            assert len(rg) == ws and rg[0][0] == 0 and rg[-1][1] == npair
            assert all(a[1] == b[0] for a, b in zip(rg[:-1], rg[1:]))
            sizes = [b - a for a, b in rg]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        pair_ranges(4, 0)


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_steps_equal_unsharded_bit_for_bit(ws):
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = _unsharded()
    for r in range(ws):
        G, gam, pairs = out[r]
        assert G == ref.G.numpy().tobytes()
        assert gam == ref.gam.numpy().tobytes()
        assert pairs == pair_ranges(ref.npair, ws)[r]


def test_single_process_without_a_group():
    f = StandInFlow()
    sf = ShardedFlow(f, device=torch.device("cpu"))
    assert (sf.ws, sf.rank, sf.my_pairs) == (1, 0, (0, f.npair))
    for lam in LAMS[1:]:
        sf.step(lam)
    assert torch.equal(f.G, _unsharded().G)
