"""Tangent-linear flow (d chi / d theta by forward-mode dual numbers on the GPU) against the
plain flow, central finite differences of the GPU flow, and central finite differences of
the CPU oracle; the torch.autograd.Function wrapper."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402
from paper_2109_13317_gb300.autograd import susceptibility  # noqa: E402

L = 2
MESH = O.mesh_exponential(6, 0.05, 10.0)
LAMS = W.lambda_list(6.0, 0.8, 8)
KPTS = np.array([[0.0, 0.0, 0.0], [2.0, 0.5, 0.0], [math.pi / 1.5, math.pi / math.sqrt(3), 0.0]])
THETA = np.array([0.2, -1.0])


def _chi_gpu(theta, tangent=False):
    cell, sites, B = W.honeycomb_kitaev_linear()
    model = W.linear_model(cell, sites, B, theta)
    lat = sr.Lattice.from_model(model, L)
    fl = sr.Flow(lat, MESH, LAMS[0], sr.SR_FP64, tangents=B if tangent else None)
    for lam in LAMS[1:]:
        fl.step(lam, sr.SR_EULER)
    if tangent:
        out = fl.measure_tangent(KPTS)
    else:
        out, _ = fl.measure(KPTS, want_ij=False)
    fl.close()
    return out


def _chi_oracle(theta):
    cell, sites, B = W.honeycomb_kitaev_linear()
    model = W.linear_model(cell, sites, B, theta)
    of = O.OracleFlow(model, L, MESH)
    for a, b in zip(LAMS[:-1], LAMS[1:]):
        of.euler(a, b)
    return of.chi_k(LAMS[-1], KPTS)


def test_tangent_value_matches_plain_flow():
    chi, _ = _chi_gpu(THETA, tangent=True)
    ref = _chi_gpu(THETA)
    np.testing.assert_allclose(chi, ref, rtol=1e-12)


def test_tangent_matches_finite_differences():
    chi, dchi = _chi_gpu(THETA, tangent=True)
    h = 1e-5
    for p in range(2):
        e = np.zeros(2)
        e[p] = h
        fd_gpu = (_chi_gpu(THETA + e) - _chi_gpu(THETA - e)) / (2 * h)
        fd_orc = (_chi_oracle(THETA + e) - _chi_oracle(THETA - e)) / (2 * h)
        scale = np.abs(dchi[:, p]).max()
        assert scale > 0
        assert np.abs(dchi[:, p] - fd_gpu).max() <= 1e-5 * scale
        assert np.abs(dchi[:, p] - fd_orc).max() <= 1e-5 * scale


def test_autograd_function():
    cell, sites, B = W.honeycomb_kitaev_linear()
    theta = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
    chi = susceptibility(theta, cell, sites, B, L, MESH, LAMS, KPTS)
    w = torch.tensor([1.0, -0.5, 2.0], dtype=torch.float64)
    (chi * w).sum().backward()
    _, dchi = _chi_gpu(THETA, tangent=True)
    np.testing.assert_allclose(theta.grad.numpy(), w.numpy() @ dchi, rtol=1e-12)


def test_symmetry_breaking_direction_is_rejected():
    cell, sites, B = W.honeycomb_kitaev_linear()
    model = W.linear_model(cell, sites, B, THETA)
    lat = sr.Lattice.from_model(model, L)
    bad = B.copy()
    bad[1, 0] = 0.0          # a Kitaev direction on one bond only breaks the lattice symmetry
    with pytest.raises(sr.SrError) as e:
        sr.Flow(lat, MESH, LAMS[0], sr.SR_FP64, tangents=bad)
    assert e.value.status == 4


# ---- TRI core: the kagome DM model as a function of theta = (J, D) ----

TRI_MESH = O.mesh_exponential(5, 0.05, 10.0)
TRI_LAMS = W.lambda_list(6.0, 1.0, 6)
TRI_THETA = np.array([1.0, 0.5])
TRI_KPTS = np.array([[0.0, 0.0, 0.0], [1.3, -0.4, 0.0], [math.pi, math.pi / math.sqrt(3), 0.0]])


def _chi_tri_gpu(theta, tangent=False):
    cell, sites, B = W.kagome_dm_linear()
    model = W.linear_model(cell, sites, B, theta, "TRI")
    lat = sr.Lattice.from_model(model, 2, backend=sr.SR_TRI)
    fl = sr.Flow(lat, TRI_MESH, TRI_LAMS[0], sr.SR_FP64, tangents=B if tangent else None)
    for lam in TRI_LAMS[1:]:
        fl.step(lam, sr.SR_EULER)
    if tangent:
        out = fl.measure_tangent(TRI_KPTS)
    else:
        out, _ = fl.measure(TRI_KPTS, want_ij=False)
    fl.close()
    return out


def _chi_tri_oracle(theta):
    cell, sites, B = W.kagome_dm_linear()
    model = W.linear_model(cell, sites, B, theta, "TRI")
    of = O.OracleFlowTRI(model, 2, TRI_MESH)
    for a, b in zip(TRI_LAMS[:-1], TRI_LAMS[1:]):
        of.euler(a, b)
    return of.chi_k(TRI_LAMS[-1], TRI_KPTS)


def test_tri_tangent_value_matches_plain_flow():
    """The value part of the TRI tangent flow is the plain FP64 TRI flow."""
    chi, _ = _chi_tri_gpu(TRI_THETA, tangent=True)
    np.testing.assert_allclose(chi, _chi_tri_gpu(TRI_THETA), rtol=1e-12)


def test_tri_tangent_matches_finite_differences():
    """d chi(k) / d(J, D) of the kagome DM model on the TRI core (dual numbers through the TRI
    self-energy flow, vertex flow, node weights and chi) against central differences of the
    GPU flow and of the oracle's TRI flow."""
    chi, dchi = _chi_tri_gpu(TRI_THETA, tangent=True)
    h = 1e-5
    for p in range(2):
        e = np.zeros(2)
        e[p] = h
        fd_gpu = (_chi_tri_gpu(TRI_THETA + e) - _chi_tri_gpu(TRI_THETA - e)) / (2 * h)
        fd_orc = (_chi_tri_oracle(TRI_THETA + e) - _chi_tri_oracle(TRI_THETA - e)) / (2 * h)
        scale = np.abs(dchi[:, p]).max()
        assert scale > 0
        assert np.abs(dchi[:, p] - fd_gpu).max() <= 1e-5 * scale
        assert np.abs(dchi[:, p] - fd_orc).max() <= 1e-5 * scale


def test_tri_symmetry_breaking_direction_is_rejected():
    cell, sites, B = W.kagome_dm_linear()
    lat = sr.Lattice.from_model(W.linear_model(cell, sites, B, TRI_THETA, "TRI"), 2, backend=sr.SR_TRI)
    bad = B.copy()
    bad[1, 0] = 0.0          # the DM term on one bond only breaks the lattice symmetry
    with pytest.raises(sr.SrError) as e:
        sr.Flow(lat, TRI_MESH, TRI_LAMS[0], sr.SR_FP64, tangents=bad)
    assert e.value.status == 4


def test_tri_autograd_function():
    """The torch.autograd.Function over the tangent flow on the TRI core."""
    cell, sites, B = W.kagome_dm_linear()
    theta = torch.tensor(TRI_THETA, dtype=torch.float64, requires_grad=True)
    chi = susceptibility(theta, cell, sites, B, 2, TRI_MESH, TRI_LAMS, TRI_KPTS, backend=sr.SR_TRI)
    w = torch.tensor([1.0, -0.5, 2.0], dtype=torch.float64)
    (chi * w).sum().backward()
    _, dchi = _chi_tri_gpu(TRI_THETA, tangent=True)
    np.testing.assert_allclose(theta.grad.numpy(), w.numpy() @ dchi, rtol=1e-12)
