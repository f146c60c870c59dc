"""Batched flows (persistent vertex kernel over instances, CUDA-graph Euler loop, autotuner)
against individually stepped flows and the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests.helpers import oracle_to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402

MODELS = [(W.square_j1j2(1.0, 0.3), 2, O.mesh_exponential(7, 0.02, 20.0)),
          (W.nn_heisenberg(W.kagome()), 2, O.mesh_exponential(5, 0.05, 10.0)),
          (W.nn_heisenberg(W.honeycomb()), 3, O.mesh_exponential(6, 0.05, 10.0)),
          (W.honeycomb_kitaev(0.2, -1.0), 1, O.mesh_exponential(5, 0.05, 10.0))]


@pytest.mark.parametrize("use_graph,autotune,mode", [(True, True, 0), (False, False, 0), (True, True, 1), (True, False, 2)])
def test_batch_matches_individual_flows(use_graph, autotune, mode):
    """Every launch form (autotuned, persistent kernels, the instances' own kernels) against the
    same flows stepped one by one."""
    lams = W.lambda_list(8.0, 0.5, 10)
    single, batched = [], []
    for model, L, mesh in MODELS:
        lat = sr.Lattice.from_model(model, L)
        single.append((lat, sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED)))
        batched.append((lat, sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED)))
    for lat, fl in single:
        for lam in lams[1:]:
            fl.step(lam, sr.SR_EULER)
    b = sr.Batch([fl for _, fl in batched])
    b.force_launch(mode)
    b.run(lams, use_graph=use_graph, autotune=autotune)
    if mode == 1:
        assert not any(b.class_launches())
    if mode == 2:
        assert all(b.class_launches())
    info = b.info()
    assert info["units"] == sum(fl.npair * fl.N for _, fl in batched)
    for (lat, f1), (_, f2) in zip(single, batched):
        assert f2.lam == lams[-1]
        g1, G1 = f1.get_state()
        g2, G2 = f2.get_state()
        # same kernels; the node-block size chosen by the autotuner changes only the FP32
        # summation order
        assert (G1 - G2).abs().max().item() <= 1e-5 * G1.abs().max().item()
        assert (g1 - g2).abs().max().item() <= 1e-5 * g1.abs().max().item()
    b.close()


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["autotuned", "persistent", "per_instance"])
def test_batch_instances_against_oracle(mode):
    """Every instance of a batch, in every launch form (mode 1 forces the persistent kernels,
    2 the instances' own kernels, 0 lets the autotuner choose), against the oracle's Euler flow
    of the same model within the FP32-mixed tolerance."""
    lams = W.lambda_list(8.0, 1.0, 6)
    flows, oracles = [], []
    for m, l, ms in MODELS:
        lat = sr.Lattice.from_model(m, l)
        flows.append((lat, sr.Flow(lat, ms, lams[0], sr.SR_FP32_MIXED)))
        of = O.OracleFlow(m, l, ms)
        for a, c in zip(lams[:-1], lams[1:]):
            of.euler(a, c)
        oracles.append(of)
    b = sr.Batch([fl for _, fl in flows])
    b.force_launch(mode)
    b.run(lams, use_graph=True, autotune=(mode == 0))
    if mode == 1:
        assert not any(b.class_launches())
    if mode == 2:
        assert all(b.class_launches())
    for (lat, fl), of in zip(flows, oracles):
        g, G = fl.get_state()
        g_o, G_o = of.get_state()
        assert np.abs(g.cpu().numpy() - g_o).max() <= 1e-3 * np.abs(g_o).max()
        exp = oracle_to_gpu(of, lat, G_o, fl.n_comp)
        got = G.cpu().numpy().reshape(exp.shape)
        for c in range(fl.n_comp):
            assert np.abs(got[:, :, c] - exp[:, :, c]).max() <= 1e-3 * np.abs(exp[:, :, c]).max(), c
    b.close()


def test_batch_wide_rows_persistent_cached_kernel():
    """A size class of wide rows (kagome range 7: 34 irreducible sites, more than 32) runs the
    persistent kernel with the corner-row cache (k_gamma_persistent_su2f<true>); forced
    persistent, it matches the same flows stepped one by one and the oracle."""
    lams = W.lambda_list(8.0, 1.0, 5)
    models = [(W.nn_heisenberg(W.kagome()), 7, O.mesh_exponential(4, 0.05, 10.0)),
              (W.square_j1j2(1.0, 0.3), 2, O.mesh_exponential(5, 0.02, 20.0))]
    single, batched, oracles = [], [], []
    for m, L, ms in models:
        lat = sr.Lattice.from_model(m, L)
        single.append(sr.Flow(lat, ms, lams[0], sr.SR_FP32_MIXED))
        batched.append((lat, sr.Flow(lat, ms, lams[0], sr.SR_FP32_MIXED)))
        of = O.OracleFlow(m, L, ms)
        for a, c in zip(lams[:-1], lams[1:]):
            of.euler(a, c)
        oracles.append(of)
    assert batched[0][0].N_s > 32
    for fl in single:
        for lam in lams[1:]:
            fl.step(lam, sr.SR_EULER)
    b = sr.Batch([fl for _, fl in batched])
    b.force_launch(1)
    b.run(lams, use_graph=True, autotune=True)
    assert not any(b.class_launches())
    for f1, (lat, f2), of in zip(single, batched, oracles):
        g1, G1 = f1.get_state()
        g2, G2 = f2.get_state()
        assert (G1 - G2).abs().max().item() <= 1e-5 * G1.abs().max().item()
        assert (g1 - g2).abs().max().item() <= 1e-5 * g1.abs().max().item()
        g_o, G_o = of.get_state()
        assert np.abs(g2.cpu().numpy() - g_o).max() <= 1e-3 * np.abs(g_o).max()
        exp = oracle_to_gpu(of, lat, G_o, f2.n_comp)
        got = G2.cpu().numpy().reshape(exp.shape)
        for c in range(f2.n_comp):
            assert np.abs(got[:, :, c] - exp[:, :, c]).max() <= 1e-3 * np.abs(exp[:, :, c]).max(), c
    b.close()
    for f in single:
        f.close()
