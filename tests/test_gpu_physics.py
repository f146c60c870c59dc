"""Loose physics anchors: the paper's worked examples run through the library.

Settings as in the paper's cubic example: 64 positive frequencies (48 for kagome) log-spaced in
0.005..50, range 7, cutoff steps of ratio 0.98 from 50 to 0.01, Euler; FP32-mixed flows.  The
paper reads its critical cutoffs off plotted flows (cubic J1-J2: 0.72 at J2 = 0, 0.3 at
J2 = 0.5; kagome ferromagnet about 0.35; kagome antiferromagnet smooth), so these checks are
loose: the breakdown criterion of `analysis.flow_breakdown` (a significant peak of the
structure-factor maximum), the ordering momenta, and for J2 = 0.5 (a breakdown the paper calls
less pronounced, a kink) the end of the steep growth.  The kagome DM example (TRI core) runs
with 32 frequencies: D = 0.5 breaks down near 0.39, D = 0 flows smoothly, and the on-site
correlation converges in the range for D = 0.1 but not for D = 0.5.
"""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402
from paper_2109_13317_gb300.analysis import flow_breakdown, log_slope, run_susceptibility_flow  # noqa: E402

PI = math.pi


def _kgrid_cubic(n=9):
    ks = np.linspace(0, PI, n)
    return np.array([[a, b, c] for a in ks for b in ks for c in ks])


def _kgrid_plane(n=33):
    ks = np.linspace(-2 * PI, 2 * PI, n)
    return np.array([[a, b, 0.0] for a in ks for b in ks])


def _flow(model, n_freq, kpts):
    lat = sr.Lattice.from_model(model, 7)
    mesh = sr.sr_frequency_mesh_exponential(n_freq, 0.005, 50.0)
    lams = W.lambda_geometric(50.0, 0.01, 0.98)
    fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED)
    rec = run_susceptibility_flow(fl, lams, kpts)
    fl.close()
    return rec


def _at(rec, lam):
    return int(np.argmin(np.abs(rec.lambdas - lam)))


def test_cubic_neel_breakdown():
    rec = _flow(W.cubic_j1j2(1.0, 0.0), 64, _kgrid_cubic())
    lc = flow_breakdown(rec.lambdas, rec.chi_max)
    assert lc is not None and abs(lc / 0.72 - 1) < 0.03, lc
    np.testing.assert_allclose(rec.k_max[_at(rec, lc)], [PI, PI, PI])


def test_cubic_collinear_order_and_end_of_steep_growth():
    rec = _flow(W.cubic_j1j2(1.0, 0.5), 64, _kgrid_cubic())
    assert rec.lambdas[-1] < 0.0102                         # the flow reaches the lowest cutoff
    k = np.sort(rec.k_max[_at(rec, 0.3)])                  # a centre of a zone edge: (0, pi, pi)
    np.testing.assert_allclose(k, [0.0, PI, PI])
    s = log_slope(rec.lambdas, rec.chi_max)
    lam = rec.lambdas[1:]
    steep = s[(lam > 0.45) & (lam < 0.55)].mean()
    flat = s[(lam > 0.2) & (lam < 0.28)].mean()
    assert steep > 2.0 and flat < 0.6, (steep, flat)


def test_kagome_ferromagnet_breakdown():
    rec = _flow(W.nn_heisenberg(W.kagome(), -1.0), 48, _kgrid_plane())
    lc = flow_breakdown(rec.lambdas, rec.chi_max)
    assert lc is not None and 0.25 < lc < 0.45, lc
    np.testing.assert_allclose(rec.k_max[_at(rec, lc)], [0.0, 0.0, 0.0], atol=1e-12)


def test_kagome_antiferromagnet_flows_smoothly():
    rec = _flow(W.nn_heisenberg(W.kagome(), 1.0), 48, _kgrid_plane())
    assert rec.lambdas[-1] < 0.0102
    assert flow_breakdown(rec.lambdas, rec.chi_max) is None


def _onsite_records(model, n_freq=32):
    from paper_2109_13317_gb300.analysis import onsite_flow
    lams = W.lambda_geometric(50.0, 0.01, 0.98)
    recs = []
    for L in (3, 5, 7):
        lat = sr.Lattice.from_model(model, L)
        mesh = sr.sr_frequency_mesh_exponential(n_freq, 0.005, 50.0)
        fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED)
        recs.append(onsite_flow(fl, lams))
        fl.close()
    return recs


def test_onsite_correlation_range_scaling():
    """The paper's range-scaling diagnostic (Sec. 6.2): chi_ii converges in the truncation range
    L = 3, 5, 7 for the kagome antiferromagnet (short-ranged correlations) down to the lowest
    cutoffs, while for the cubic Neel antiferromagnet the curves separate below its breakdown
    (Lambda_c = 0.72)."""
    from paper_2109_13317_gb300.analysis import range_spread
    lam, sp = range_spread(_onsite_records(W.nn_heisenberg(W.kagome(), 1.0)))
    assert sp[lam >= 0.05].max() < 0.01
    lam, sp = range_spread(_onsite_records(W.cubic_j1j2(1.0, 0.0)))
    assert sp[lam >= 1.0].max() < 0.01
    assert sp[(lam > 0.5) & (lam < 0.7)].max() > 0.1


def _dm_flow(D, n_freq=32):
    lat = sr.Lattice.from_model(W.kagome_dm(1.0, D), 7)
    mesh = sr.sr_frequency_mesh_exponential(n_freq, 0.005, 50.0)
    lams = W.lambda_geometric(50.0, 0.01, 0.98)
    fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED)
    rec = run_susceptibility_flow(fl, lams, _kgrid_plane())
    fl.close()
    return rec


def test_kagome_dm_breakdown_and_smooth_heisenberg_limit():
    """The paper's second worked example (TRI core): the kagome antiferromagnet with out-of-plane
    DM couplings D = 0.5 breaks down at Lambda_c = 0.39 (range 7, 64 frequencies) with the
    structure-factor maximum on the boundary of the extended Brillouin zone, while D = 0 flows
    smoothly.  Here 32 frequencies, so the window is loose."""
    rec = _dm_flow(0.5)
    lc = flow_breakdown(rec.lambdas, rec.chi_max)
    assert lc is not None and 0.3 < lc < 0.45, lc
    assert abs(np.linalg.norm(rec.k_max[_at(rec, lc)]) - 2 * PI) < 0.05
    rec0 = _dm_flow(0.0)
    assert rec0.lambdas[-1] < 0.0102
    assert flow_breakdown(rec0.lambdas, rec0.chi_max) is None


def test_kagome_dm_onsite_range_scaling():
    """The paper's range-scaling diagnostic for the DM model (Sec. 6.2): chi_ii at L = 3, 5, 7
    stays converged for D = 0.1, while for D = 0.5 the ranges separate below the breakdown."""
    from paper_2109_13317_gb300.analysis import range_spread
    lam, sp = range_spread(_onsite_records(W.kagome_dm(1.0, 0.1)))
    assert sp[lam >= 0.01].max() < 0.012, sp.max()
    lam, sp = range_spread(_onsite_records(W.kagome_dm(1.0, 0.5)))
    assert sp[lam >= 1.0].max() < 1e-4
    assert sp[(lam > 0.1) & (lam < 0.3)].min() > 0.01
