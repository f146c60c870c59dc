"""Parity of the workload configurations against the oracle.

square_j1_L3 (square J1, L = 3, N = 16, FP64 Euler): the first 20 of the 100 Euler steps and
chi(k) on a momentum grid.  pyrochlore: the reduced variant L = 2, N = 12 (the oracle's
unreduced storage at L = 6, N = 64 would need ~4 GB and one oracle right-hand side at L = 3,
N = 24 already takes ~90 s on 8 cores), FP64 and FP32-mixed right-hand side on an
oracle-evolved state.  honeycomb_hk_L5 (XYZ): one right-hand side on an oracle-evolved state
at the configuration's range, with N reduced to 12.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests.helpers import gpu_comp_map, oracle_to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _load(fl, lat, of, lam):
    gam, G = of.get_state()
    Gg = oracle_to_gpu(of, lat, G, fl.n_comp)
    fl.set_state(lam, torch.tensor(gam, device="cuda"), torch.tensor(Gg.reshape(-1), device="cuda"))


def test_square_j1_L3_euler_flow():
    cfg = W.config("square_j1_L3")
    mesh = O.mesh_exponential(cfg.n_freq, cfg.w_min, cfg.w_max)
    lams = W.lambda_list(cfg.lam_max, cfg.lam_min, cfg.n_steps)[:21]
    of = O.OracleFlow(cfg.model, cfg.L, mesh)
    lat = sr.Lattice.from_model(cfg.model, cfg.L)
    fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP64)
    for a, b in zip(lams[:-1], lams[1:]):
        of.euler(a, b)
        fl.step(b, sr.SR_EULER)
    g_o, G_o = of.get_state()
    g, G = fl.get_state()
    assert _rel(g.cpu().numpy(), g_o) < 1e-10
    exp = oracle_to_gpu(of, lat, G_o, fl.n_comp)
    got = G.cpu().numpy().reshape(exp.shape)
    for c in range(fl.n_comp):
        assert _rel(got[:, :, c], exp[:, :, c]) < 1e-10
    ks = np.linspace(-2 * math.pi, 2 * math.pi, 9)
    kpts = np.array([[a, b, 0.0] for a in ks for b in ks])
    chik, _ = fl.measure(kpts)
    assert _rel(chik, of.chi_k(lams[-1], kpts)) < 1e-10


def test_pyrochlore_reduced_fp32_mixed():
    model = W.nn_heisenberg(W.pyrochlore(), 1.0)
    L, mesh = 2, O.mesh_exponential(12, 0.001, 100.0)
    of = O.OracleFlow(model, L, mesh)
    for a, b in zip([100.0, 30.0, 10.0, 3.0], [30.0, 10.0, 3.0, 1.0]):
        of.euler(a, b)
    lat = sr.Lattice.from_model(model, L)
    for prec, tol in ((sr.SR_FP64, 1e-10), (sr.SR_FP32_MIXED, 1e-3)):
        fl = sr.Flow(lat, mesh, 1.0, prec)
        _load(fl, lat, of, 1.0)
        dg_o, dG_o = of.rhs(0.8)
        dg, dG = fl.rhs(0.8)
        torch.cuda.synchronize()
        assert _rel(dg.cpu().numpy(), dg_o) < 1e-10
        exp = oracle_to_gpu(of, lat, dG_o, fl.n_comp)
        got = dG.cpu().numpy().reshape(exp.shape)
        for c in range(fl.n_comp):
            assert _rel(got[:, :, c], exp[:, :, c]) < tol
        fl.close()


def test_honeycomb_hk_L5_xyz_rhs():
    cfg = W.config("honeycomb_hk_L5")
    mesh = O.mesh_exponential(12, cfg.w_min, cfg.w_max)
    of = O.OracleFlow(cfg.model, cfg.L, mesh)
    for a, b in zip([50.0, 10.0, 3.0], [10.0, 3.0, 1.0]):
        of.euler(a, b)
    lat = sr.Lattice.from_model(cfg.model, cfg.L)
    for prec, tol in ((sr.SR_FP64, 1e-10), (sr.SR_FP32_MIXED, 1e-3)):
        fl = sr.Flow(lat, mesh, 1.0, prec)
        _load(fl, lat, of, 1.0)
        dg_o, dG_o = of.rhs(0.6)
        dg, dG = fl.rhs(0.6)
        torch.cuda.synchronize()
        assert _rel(dg.cpu().numpy(), dg_o) < 1e-10
        exp = oracle_to_gpu(of, lat, dG_o, fl.n_comp)
        got = dG.cpu().numpy().reshape(exp.shape)
        for c in range(fl.n_comp):
            assert _rel(got[:, :, c], exp[:, :, c]) < tol
        fl.close()


def _sampled_parity(of, lat, fl, lam, tol, n_random=40, seed=0):
    """The GPU right-hand side at cutoff lam against the oracle's values of sampled stored
    entries (the mesh corners, the s = u diagonal and random triples, random sites)."""
    dg, dG = fl.rhs(lam)
    torch.cuda.synchronize()
    dG = dG.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s)
    reps = lat.representatives()
    rng = np.random.default_rng(seed)
    N = fl.N
    picks = [(0, 0, 0), (N - 1, N - 1, N - 1), (N - 1, 0, 0), (N - 1, N - 1, 0), (N // 2, N // 2, 1)]
    picks += [tuple(sorted(rng.integers(0, N, 2))[::-1]) + (int(rng.integers(0, N)),) for _ in range(n_random)]
    ent, rs = [], []
    for (si, ui, ti) in picks:
        r = int(rng.integers(0, lat.N_s))
        k = of.find(0, reps[r][:3], int(reps[r][3]))
        assert k >= 0
        ent.append((0, k, si, ti, ui))
        rs.append(r)
    ent = np.array(ent)
    out = of.rhs_entries(lam, ent)
    dg_o = of.prepare(lam)
    # (the self-energy flow vanishes exactly at the bare vertex: compare against max(|.|, 1))
    assert np.abs(dg.cpu().numpy() - dg_o).max() <= max(tol, 1e-10) * max(np.abs(dg_o).max(), 1.0)
    cm = gpu_comp_map(fl.n_comp)
    scale = np.abs(out).max()
    assert scale > 0
    for (b, k, si, ti, ui), r, o in zip(ent, rs, out):
        p = si * (si + 1) // 2 + ui
        for c, oc in enumerate(cm):
            assert abs(dG[p, ti, c, r] - o[oc]) <= tol * scale, (si, ti, ui, r, c, dG[p, ti, c, r], o[oc])


@pytest.mark.parametrize("prec,tol", [(sr.SR_FP64, 1e-10), (sr.SR_FP32_MIXED, 1e-3)])
def test_pyrochlore_full_range_sampled(prec, tol):
    """Pyrochlore J1 at the configuration's full range L = 6 (N_s = 48, N_tot = 459) with the
    frequency mesh reduced to 8 points (0.001..100) so that the oracle's unreduced storage fits:
    sampled entries of the right-hand side on a synthetic symmetric state."""
    from tests.helpers import synthetic_state
    cfg = W.config("pyrochlore_L6")
    mesh = O.mesh_exponential(8, cfg.w_min, cfg.w_max)
    of = O.OracleFlow(cfg.model, cfg.L, mesh)
    gam, G = synthetic_state(of, cfg.model, seed=4)
    of.set_state(gam, G)
    lat = sr.Lattice.from_model(cfg.model, cfg.L)
    assert lat.N_s == 48 and lat.N_tot == 459
    fl = sr.Flow(lat, mesh, 1.0, prec)
    _load(fl, lat, of, 1.0)
    _sampled_parity(of, lat, fl, 0.9, tol)
    fl.close()


@pytest.mark.parametrize("prec,tol", [(sr.SR_FP64, 1e-10), (sr.SR_FP32_MIXED, 1e-3)])
def test_heisenberg_kitaev_full_size_sampled(prec, tol):
    """Honeycomb Heisenberg-Kitaev (XYZ) at the configuration's full size (L = 5, N = 32,
    0.005..50): the first right-hand side of the flow (bare vertex at Lambda = 50, computed
    independently by both sides) on sampled entries."""
    cfg = W.config("honeycomb_hk_L5")
    mesh = O.mesh_exponential(cfg.n_freq, cfg.w_min, cfg.w_max)
    of = O.OracleFlow(cfg.model, cfg.L, mesh)
    lat = sr.Lattice.from_model(cfg.model, cfg.L)
    fl = sr.Flow(lat, mesh, cfg.lam_max, prec)
    _sampled_parity(of, lat, fl, cfg.lam_max, tol, seed=1)
    # and after a quarter of the cutoff range, on the same bare vertex
    _sampled_parity(of, lat, fl, 0.25 * cfg.lam_max, tol, seed=2)
    fl.close()
