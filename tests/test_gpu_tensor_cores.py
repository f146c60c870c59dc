"""Tensor-core lattice sum of the FP32-mixed SU2 vertex kernel (tcgen05 MMAs in 3xTF32).

Against the oracle: the tensor-core right-hand side on oracle-evolved states within the
FP32-mixed tolerance (1e-3 normwise per component; the self-energy flow, FP64, within 1e-10).

The same right-hand side with the lattice-sum contraction on the tensor cores and on FP32 CUDA
cores must agree to FP32 rounding (3xTF32 keeps ~22 of the 24 mantissa bits of every product),
and both must stay within the FP32-mixed tolerance of the FP64 kernel.  Lattices cover both
operand packings (<= 32 padded sites: both spin components in one MMA; 33..64: one MMA per
component) and a flow whose t channel has node counts that are not multiples of the MMA K.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests.helpers import evolved_oracle, oracle_to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402


def _state(model, L, n_freq, w_min, w_max, lam_max, lam_stop, n_steps=60):
    """FP64 GPU flow evolved by Euler steps from lam_max until the cutoff drops below lam_stop."""
    lat = sr.Lattice.from_model(model, L)
    mesh = sr.sr_frequency_mesh_exponential(n_freq, w_min, w_max)
    lams = W.lambda_list(lam_max, lam_stop / 10, n_steps)
    fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP64)
    i = 0
    while lams[i] > lam_stop:
        fl.step(lams[i + 1], sr.SR_EULER)
        i += 1
    s, G = fl.get_state()
    lam = fl.lam
    fl.close()
    return lat, mesh, lam, s, G


def _rhs(lat, mesh, lam, s, G, prec, tc=None):
    fl = sr.Flow(lat, mesh, lam, prec)
    if tc is not None:
        fl.tensor_cores = tc
    fl.set_state(lam, s, G)
    ds, dG = fl.rhs(lam)
    torch.cuda.synchronize()
    out = (ds.clone(), dG.clone())
    fl.close()
    return out


def _nerr(a, b):
    return float((a - b).abs().max() / b.abs().max())


CASES = [
    ("square_j1j2_L3", lambda: W.square_j1j2(1.0, 0.5), 3, 12),     # packed, few sites
    ("kagome_L4", lambda: W.nn_heisenberg(W.kagome()), 4, 10),        # packed, N_s = 13
    ("kagome_L6", lambda: W.nn_heisenberg(W.kagome()), 6, 9),         # packed, N_s = 26
    ("kagome_L7", lambda: W.nn_heisenberg(W.kagome()), 7, 8),         # unpacked, N_s = 34
    ("pyrochlore_L3", lambda: W.nn_heisenberg(W.pyrochlore()), 3, 8),
]


ORACLE_CASES = [
    ("square_j1j2", lambda: W.square_j1j2(1.0, 0.5), 2, 7, 0.02, 20.0),
    ("honeycomb", lambda: W.nn_heisenberg(W.honeycomb()), 2, 6, 0.05, 10.0),
    ("kagome", lambda: W.nn_heisenberg(W.kagome()), 2, 5, 0.05, 10.0),
    ("kagome_L7", lambda: W.nn_heisenberg(W.kagome()), 7, 5, 0.05, 10.0),   # N_s = 34: one MMA per component
]


@pytest.mark.parametrize("name,mk,L,N,wmin,wmax", ORACLE_CASES, ids=[c[0] for c in ORACLE_CASES])
def test_tensor_cores_match_oracle(name, mk, L, N, wmin, wmax):
    model = mk()
    mesh = O.mesh_exponential(N, wmin, wmax)
    of = evolved_oracle(model, L, mesh, [8.0, 4.0, 2.0, 1.0])
    lam = 0.7
    dg_o, dG_o = of.rhs(lam)
    lat = sr.Lattice.from_model(model, L)
    fl = sr.Flow(lat, mesh, 1.0, sr.SR_FP32_MIXED)
    fl.tensor_cores = True
    gam, G = of.get_state()
    Gg = oracle_to_gpu(of, lat, G, fl.n_comp)
    fl.set_state(1.0, torch.tensor(gam, device="cuda"), torch.tensor(Gg.reshape(-1), device="cuda"))
    dg, dG = fl.rhs(lam)
    torch.cuda.synchronize()
    assert fl.tensor_cores
    dg = dg.cpu().numpy()
    assert np.abs(dg - dg_o).max() <= 1e-10 * np.abs(dg_o).max()
    got = dG.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s)
    exp = oracle_to_gpu(of, lat, dG_o, fl.n_comp)
    for c in range(fl.n_comp):
        e = exp[:, :, c]
        assert np.abs(got[:, :, c] - e).max() <= 1e-3 * np.abs(e).max(), c
    fl.close()


@pytest.mark.parametrize("name,mk,L,nf", CASES)
def test_tensor_cores_match_cuda_cores(name, mk, L, nf):
    lat, mesh, lam, s, G = _state(mk(), L, nf, 0.01, 20.0, 20.0, 0.7)
    ds_tc, dG_tc = _rhs(lat, mesh, lam, s, G, sr.SR_FP32_MIXED, tc=True)
    ds_fm, dG_fm = _rhs(lat, mesh, lam, s, G, sr.SR_FP32_MIXED, tc=False)
    ds_64, dG_64 = _rhs(lat, mesh, lam, s, G, sr.SR_FP64)
    assert torch.isfinite(dG_tc).all()
    assert torch.equal(ds_tc, ds_fm)                     # the self-energy flow is FP64 in both
    assert _nerr(dG_tc, dG_fm) < 1e-5, _nerr(dG_tc, dG_fm)
    assert _nerr(dG_tc, dG_64) < 1e-3, _nerr(dG_tc, dG_64)
    # per component (density and spin) as well
    sh = (-1, 2, lat.N_s)
    for c in range(2):
        a = dG_tc.view(*sh)[:, c]
        b = dG_64.view(*sh)[:, c]
        assert _nerr(a, b) < 1e-3


def test_tensor_core_operand_packings_are_exercised():
    """The case list spans both packings (<= 32 and 33..64 padded sites)."""
    nsp = []
    for _, mk, L, _ in CASES:
        ns = sr.Lattice.from_model(mk(), L).N_s
        nsp.append((ns + 3) // 4 * 4)
    assert min(nsp) <= 32 < max(nsp) <= 64, nsp


@pytest.mark.parametrize("cfg_name", ["square_j1j2_L7", "pyrochlore_L6"])
def test_tensor_cores_full_size(cfg_name):
    """Full-size workloads (square J1-J2 range 7, 48 frequencies; pyrochlore range 6, 64
    frequencies): tensor-core and CUDA-core kernels on the same mid-flow state."""
    cfg = W.config(cfg_name)
    lat, mesh, lam, s, G = _state(cfg.model, cfg.L, cfg.n_freq, cfg.w_min, cfg.w_max, cfg.lam_max, 1.0, 200)
    _, dG_tc = _rhs(lat, mesh, lam, s, G, sr.SR_FP32_MIXED, tc=True)
    _, dG_fm = _rhs(lat, mesh, lam, s, G, sr.SR_FP32_MIXED, tc=False)
    assert torch.isfinite(dG_tc).all()
    assert _nerr(dG_tc, dG_fm) < 1e-5, _nerr(dG_tc, dG_fm)


def test_tensor_core_switch():
    m = W.square_j1j2(1.0, 0.5)
    lat = sr.Lattice.from_model(m, 2)
    mesh = sr.sr_frequency_mesh_exponential(6, 0.05, 10.0)
    f32 = sr.Flow(lat, mesh, 5.0, sr.SR_FP32_MIXED)
    assert not f32.tensor_cores                   # off by default (the CUDA-core path is faster)
    f32.tensor_cores = True
    assert f32.tensor_cores
    f32.tensor_cores = False
    assert not f32.tensor_cores
    f64 = sr.Flow(lat, mesh, 5.0, sr.SR_FP64)
    assert not f64.tensor_cores
    with pytest.raises(sr.SrError) as e:
        f64.tensor_cores = True
    assert e.value.status == sr.SR_EUNSUPPORTED
    cell, sites, B = W.honeycomb_kitaev_linear()
    latx = sr.Lattice.from_model(W.linear_model(cell, sites, B, [0.2, -1.0]), 2)
    fx = sr.Flow(latx, mesh, 5.0, sr.SR_FP32_MIXED)
    assert not fx.tensor_cores
    with pytest.raises(sr.SrError):
        fx.tensor_cores = True
    for f in (f32, f64, fx):
        f.close()
