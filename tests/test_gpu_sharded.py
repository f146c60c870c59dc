"""The sharded right-hand side on the GPU (Sec. 4.4 superblocks): sr_flow_rhs_pairs over a
split of the stored (s, u) pairs assembles to exactly sr_flow_rhs (bit for bit, every core
and precision), sr_flow_advance with that right-hand side is exactly sr_flow_step, and the
torch.distributed driver (NCCL, one rank: only one GPU is available here) steps the flow
exactly as the library does.  Several ranks are covered by the gloo tests of the driver
(tests/test_sharded_ranks.py); the multi-GPU run itself is unmeasured on hardware."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402
from paper_2109_13317_gb300.sharded import ShardedFlow, pair_ranges  # noqa: E402

CASES = [
    ("su2_fp64", lambda: W.square_j1j2(1.0, 0.5), 3, sr.SR_FP64),
    ("su2_fp32", lambda: W.square_j1j2(1.0, 0.5), 3, sr.SR_FP32_MIXED),
    ("xyz_fp32", lambda: W.honeycomb_kitaev(0.2, -1.0), 2, sr.SR_FP32_MIXED),
    ("tri_fp64", lambda: W.kagome_dm(1.0, 0.5), 2, sr.SR_FP64),
]


def _flow(mk, L, prec):
    lat = sr.Lattice.from_model(mk(), L)
    fl = sr.Flow(lat, O.mesh_exponential(7, 0.02, 20.0), 10.0, prec)
    for lam in (6.0, 3.0):
        fl.step(lam, sr.SR_EULER)
    return fl


@pytest.mark.parametrize("name,mk,L,prec", CASES, ids=[c[0] for c in CASES])
def test_pair_ranges_assemble_the_full_rhs(name, mk, L, prec):
    fl = _flow(mk, L, prec)
    ds_ref, dG_ref = fl.rhs(2.1)
    for ws in (2, 3):
        ds = torch.full_like(ds_ref, float("nan"))
        dG = torch.full_like(dG_ref, float("nan"))
        for p0, p1 in pair_ranges(fl.npair, ws):
            fl.rhs_pairs(2.1, p0, p1, ds, dG)
        torch.cuda.synchronize()
        assert torch.equal(ds, ds_ref)
        assert torch.equal(dG, dG_ref)
    # a range writes only its own slice
    dG = torch.full_like(dG_ref, 7.0)
    p0, p1 = pair_ranges(fl.npair, 3)[1]
    fl.rhs_pairs(2.1, p0, p1, ds, dG)
    e = fl.entries_per_pair
    assert torch.equal(dG[p0 * e:p1 * e], dG_ref[p0 * e:p1 * e])
    assert bool((dG[:p0 * e] == 7.0).all()) and bool((dG[p1 * e:] == 7.0).all())
    with pytest.raises(sr.SrError):
        fl.rhs_pairs(2.1, 0, fl.npair + 1, ds, dG)
    # advance with the assembled right-hand side == the library's own Euler step
    g0, G0 = (x.clone() for x in fl.get_state())
    fl.set_state(2.1, g0, G0)   # the right-hand side above is the one at Lambda = 2.1
    fl.advance(1.7, ds_ref, dG_ref)
    g1, G1 = fl.get_state()
    fl.set_state(2.1, g0, G0)
    fl.step(1.7, sr.SR_EULER)
    g2, G2 = fl.get_state()
    assert torch.equal(g1, g2) and torch.equal(G1, G2)
    fl.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_driver_on_one_nccl_rank():
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        a = _flow(lambda: W.square_j1j2(1.0, 0.5), 3, sr.SR_FP32_MIXED)
        b = _flow(lambda: W.square_j1j2(1.0, 0.5), 3, sr.SR_FP32_MIXED)
        sf = ShardedFlow(a)
        for lam in (2.5, 2.0, 1.6):
            sf.step(lam)
            b.step(lam, sr.SR_EULER)
        ga, Ga = a.get_state()
        gb, Gb = b.get_state()
        assert torch.equal(ga, gb) and torch.equal(Ga, Gb)
        assert np.isclose(a.lam, 1.6)
    finally:
        dist.destroy_process_group()
