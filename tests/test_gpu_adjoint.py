"""Reverse-mode adjoint of the FP64 flow.

Pins, none of which uses the adjoint's own arithmetic:
  * dot-product identities <fbar, J ydot> = <J^T fbar, ydot> block by block (self-energy /
    vertex inputs and outputs), with J ydot from the tangent-linear flow (forward-mode dual
    numbers through the forward kernels), for an SU2, an XYZ and a TRI lattice (kagome DM);
  * the same identity for chi(k) and for one Euler step;
  * the checkpointed gradient d chi(k) / d(J, K) against the tangent-linear flow, central
    finite differences of the GPU flow and of the CPU oracle, and at the full Heisenberg-
    Kitaev size (range 5, 32 frequencies, 200 steps, a checkpoint every 20 steps).
"""
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
from paper_2109_13317_gb300.autograd import susceptibility, susceptibility_adjoint  # noqa: E402

MESH = O.mesh_exponential(6, 0.05, 10.0)
LAMS = W.lambda_list(6.0, 0.8, 8)
KPTS = np.array([[0.0, 0.0, 0.0], [2.0, 0.5, 0.0], [math.pi / 1.5, math.pi / math.sqrt(3), 0.0]])
THETA = np.array([0.2, -1.0])
TRI_THETA = np.array([1.0, 0.5])     # kagome DM: (J, D)


def _case(name):
    """(model, tangent directions B (n_par, n_couplings, 3, 3)) of a small test lattice."""
    if name == "square_j1j2":
        m = W.square_j1j2(1.0, 0.5)
        B = np.stack([c.M for c in m.couplings])[None]
        return m, B
    if name == "tri":
        cell, sites, B = W.kagome_dm_linear()
        return W.linear_model(cell, sites, B, TRI_THETA, "TRI"), B
    cell, sites, B = W.honeycomb_kitaev_linear()
    return W.linear_model(cell, sites, B, THETA), B


def _lattice(name, model, L=2):
    return sr.Lattice.from_model(model, L, backend=sr.SR_TRI) if name == "tri" else sr.Lattice.from_model(model, L)


def _interleave(v, d1, d2=None):
    d2 = torch.zeros_like(v) if d2 is None else d2
    return torch.stack([v, d1, d2], dim=1).reshape(-1).contiguous()


def _evolved(name, steps=4):
    model, B = _case(name)
    lat = _lattice(name, model)
    fl = sr.Flow(lat, MESH, LAMS[0], sr.SR_FP64)
    for lam in LAMS[1:steps + 1]:
        fl.step(lam, sr.SR_EULER)
    return lat, B, fl, LAMS[steps]


def _rand(n, seed):
    g = torch.Generator().manual_seed(seed)
    return (torch.rand(n, generator=g, dtype=torch.float64) * 2 - 1).cuda()


@pytest.mark.parametrize("name", ["square_j1j2", "hk", "tri"])
@pytest.mark.parametrize("block", ["ss", "sG", "Gs", "GG"])
def test_rhs_adjoint_dot_product(name, block):
    """<fbar, J ydot> = <J^T fbar, ydot> for each (output, input) block of the Jacobian."""
    lat, B, fl, lam = _evolved(name)
    ys, yG = fl.get_state()
    out_blk, in_blk = block[0], block[1]
    yds = _rand(fl.N, 1) if in_blk == "s" else torch.zeros(fl.N, dtype=torch.float64, device="cuda")
    ydG = _rand(fl.n_gamma, 2) if in_blk == "G" else torch.zeros(fl.n_gamma, dtype=torch.float64, device="cuda")
    fbs = _rand(fl.N, 3) if out_blk == "s" else torch.zeros(fl.N, dtype=torch.float64, device="cuda")
    fbG = _rand(fl.n_gamma, 4) if out_blk == "G" else torch.zeros(fl.n_gamma, dtype=torch.float64, device="cuda")

    ft = sr.Flow(lat, MESH, LAMS[0], sr.SR_FP64, tangents=B)
    ft.set_state(lam, _interleave(ys, yds), _interleave(yG, ydG))
    ts, tG = ft.rhs(lam)
    ts, tG = ts.view(-1, 3), tG.view(-1, 3)
    ps, pG = fl.rhs(lam)
    torch.testing.assert_close(ts[:, 0], ps, rtol=1e-12, atol=1e-14)
    torch.testing.assert_close(tG[:, 0], pG, rtol=1e-12, atol=1e-14)

    bs, bG = fl.rhs_adjoint(lam, fbs, fbG)
    lhs = float((fbs * ts[:, 1]).sum() + (fbG * tG[:, 1]).sum())
    rhs = float((bs * yds).sum() + (bG * ydG).sum())
    scale = float((fbs.abs() * ts[:, 1].abs()).sum() + (fbG.abs() * tG[:, 1].abs()).sum())
    assert scale > 0.0
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    ft.close()
    fl.close()


@pytest.mark.parametrize("name", ["square_j1j2", "hk", "tri"])
@pytest.mark.parametrize("in_blk", ["s", "G"])
def test_chi_adjoint_dot_product(name, in_blk):
    lat, B, fl, lam = _evolved(name)
    ys, yG = fl.get_state()
    yds = _rand(fl.N, 5) if in_blk == "s" else torch.zeros(fl.N, dtype=torch.float64, device="cuda")
    ydG = _rand(fl.n_gamma, 6) if in_blk == "G" else torch.zeros(fl.n_gamma, dtype=torch.float64, device="cuda")
    ft = sr.Flow(lat, MESH, LAMS[0], sr.SR_FP64, tangents=B)
    ft.set_state(lam, _interleave(ys, yds), _interleave(yG, ydG))
    chi, dchi = ft.measure_tangent(KPTS)
    cbar = np.array([0.7, -1.3, 0.4])
    bs, bG = fl.measure_adjoint(KPTS, cbar)
    lhs = float(cbar @ dchi[:, 0])
    rhs = float((bs * yds).sum() + (bG * ydG).sum())
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + np.abs(cbar) @ np.abs(dchi[:, 0])) + 1e-300, (lhs, rhs)
    ft.close()
    fl.close()


def test_step_adjoint_identities():
    lat, B, fl, lam = _evolved("hk")
    lam2 = LAMS[5]
    bs0, bG0 = _rand(fl.N, 7), _rand(fl.n_gamma, 8)
    rs, rG = fl.rhs_adjoint(lam, bs0, bG0)
    os_, oG = fl.step_adjoint(lam, lam2, bs0, bG0, bs0.clone(), bG0.clone())
    dl = lam - lam2
    torch.testing.assert_close(os_, bs0 - dl * rs, rtol=1e-10, atol=1e-13)
    torch.testing.assert_close(oG, bG0 - dl * rG, rtol=1e-10, atol=1e-13)
    # in place (outputs aliasing the inputs)
    a, b = bs0.clone(), bG0.clone()
    fl.step_adjoint(lam, lam2, a, b)
    torch.testing.assert_close(a, os_, rtol=1e-10, atol=1e-13)
    torch.testing.assert_close(b, oG, rtol=1e-10, atol=1e-13)
    # the state must be the forward state at lambda_from
    with pytest.raises(sr.SrError):
        fl.step_adjoint(lam2, LAMS[6], a, b)
    # the state is unchanged by the adjoint
    s1, G1 = fl.get_state()
    fl.rhs_adjoint(lam, bs0, bG0)
    s2, G2 = fl.get_state()
    assert torch.equal(s1, s2) and torch.equal(G1, G2)
    fl.close()


def test_step_adjoint_dot_product_with_tangent_step():
    """<ybar_1, ydot_1> = <step^T ybar_1, ydot_0> with ydot_1 from a tangent Euler step."""
    lat, B, fl, lam = _evolved("square_j1j2")
    lam2 = LAMS[5]
    ys, yG = fl.get_state()
    yds, ydG = _rand(fl.N, 9), _rand(fl.n_gamma, 10)
    ft = sr.Flow(lat, MESH, LAMS[0], sr.SR_FP64, tangents=B)
    ft.set_state(lam, _interleave(ys, yds), _interleave(yG, ydG))
    ft.step(lam2, sr.SR_EULER)
    ts, tG = ft.get_state()
    ts, tG = ts.view(-1, 3)[:, 1], tG.view(-1, 3)[:, 1]
    bs, bG = _rand(fl.N, 11), _rand(fl.n_gamma, 12)
    lhs = float((bs * ts).sum() + (bG * tG).sum())
    os_, oG = fl.step_adjoint(lam, lam2, bs.clone(), bG.clone())
    rhs = float((os_ * yds).sum() + (oG * ydG).sum())
    scale = float((bs.abs() * ts.abs()).sum() + (bG.abs() * tG.abs()).sum())
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs)
    ft.close()
    fl.close()


def test_adjoint_rejects_other_flows():
    model, B = _case("hk")
    lat = sr.Lattice.from_model(model, 2)
    z = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
    f32 = sr.Flow(lat, MESH, LAMS[0], sr.SR_FP32_MIXED)
    with pytest.raises(sr.SrError) as e:
        f32.rhs_adjoint(LAMS[0], z[:f32.N], z[:f32.n_gamma])
    assert e.value.status == sr.SR_EUNSUPPORTED
    ft = sr.Flow(lat, MESH, LAMS[0], sr.SR_FP64, tangents=B)
    with pytest.raises(sr.SrError) as e:
        ft.measure_adjoint(KPTS, np.ones(3))
    assert e.value.status == sr.SR_EUNSUPPORTED
    f32.close()
    ft.close()


def _grad_adjoint(theta, L, mesh, lams, kpts, every):
    cell, sites, B = W.honeycomb_kitaev_linear()
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    chi = susceptibility_adjoint(th, cell, sites, B, L, mesh, lams, kpts, sr.SR_XYZ, every=every)
    grads = []
    for i in range(len(kpts)):
        (gi,) = torch.autograd.grad(chi[i], th, retain_graph=i + 1 < len(kpts))
        grads.append(gi.numpy())
    return chi.detach().numpy(), np.array(grads)


def _grad_tangent(theta, L, mesh, lams, kpts):
    cell, sites, B = W.honeycomb_kitaev_linear()
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    chi = susceptibility(th, cell, sites, B, L, mesh, lams, kpts, sr.SR_XYZ)
    grads = []
    for i in range(len(kpts)):
        (gi,) = torch.autograd.grad(chi[i], th, retain_graph=i + 1 < len(kpts))
        grads.append(gi.numpy())
    return chi.detach().numpy(), np.array(grads)


def _chi_plain(theta, L, mesh, lams, kpts):
    cell, sites, B = W.honeycomb_kitaev_linear()
    lat = sr.Lattice.from_model(W.linear_model(cell, sites, B, theta), L)
    fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP64)
    for lam in lams[1:]:
        fl.step(lam, sr.SR_EULER)
    chi, _ = fl.measure(kpts, want_ij=False)
    fl.close()
    return chi


@pytest.mark.parametrize("every", [1, 3, 20])
def test_adjoint_gradient_small(every):
    chi, g = _grad_adjoint(THETA, 2, MESH, LAMS, KPTS, every)
    chi_t, g_t = _grad_tangent(THETA, 2, MESH, LAMS, KPTS)
    np.testing.assert_allclose(chi, chi_t, rtol=1e-12)
    np.testing.assert_allclose(g, g_t, rtol=1e-9, atol=1e-12 * np.abs(g_t).max())
    h = 1e-5
    for p in range(2):
        e = np.zeros(2)
        e[p] = h
        fd = (_chi_plain(THETA + e, 2, MESH, LAMS, KPTS) - _chi_plain(THETA - e, 2, MESH, LAMS, KPTS)) / (2 * h)
        np.testing.assert_allclose(g[:, p], fd, rtol=1e-5, atol=1e-5 * np.abs(fd).max())


def test_adjoint_gradient_matches_oracle_finite_differences():
    _, g = _grad_adjoint(THETA, 2, MESH, LAMS, KPTS, 3)
    cell, sites, B = W.honeycomb_kitaev_linear()
    h = 1e-5

    def chi_o(theta):
        of = O.OracleFlow(W.linear_model(cell, sites, B, theta), 2, MESH)
        for a, b in zip(LAMS[:-1], LAMS[1:]):
            of.euler(a, b)
        return of.chi_k(LAMS[-1], KPTS)

    for p in range(2):
        e = np.zeros(2)
        e[p] = h
        fd = (chi_o(THETA + e) - chi_o(THETA - e)) / (2 * h)
        np.testing.assert_allclose(g[:, p], fd, rtol=1e-5, atol=1e-5 * np.abs(fd).max())


def test_adjoint_gradient_heisenberg_kitaev_full_size():
    """Range 5, 32 frequencies 0.005..50, 200 Euler steps 50 -> 0.05, checkpoints every 20
    steps; k_max = the maximum of chi(k) over a k grid of the nominal run."""
    cfg = W.config("honeycomb_hk_L5")
    mesh = sr.sr_frequency_mesh_exponential(cfg.n_freq, cfg.w_min, cfg.w_max)
    lams = W.lambda_list(cfg.lam_max, cfg.lam_min, cfg.n_steps)
    theta = np.array([0.2, -1.0])
    ks = np.linspace(-2 * math.pi, 2 * math.pi, 25)
    grid = np.array([[kx, ky, 0.0] for kx in ks for ky in ks])
    chi_grid = _chi_plain(theta, cfg.L, mesh, lams, grid)
    kmax = grid[int(np.argmax(chi_grid))][None]
    chi, g = _grad_adjoint(theta, cfg.L, mesh, lams, kmax, 20)
    chi_t, g_t = _grad_tangent(theta, cfg.L, mesh, lams, kmax)
    np.testing.assert_allclose(chi, chi_t, rtol=1e-12)
    np.testing.assert_allclose(g, g_t, rtol=1e-8)
    h = 1e-5
    for p in range(2):
        e = np.zeros(2)
        e[p] = h
        fd = (_chi_plain(theta + e, cfg.L, mesh, lams, kmax) - _chi_plain(theta - e, cfg.L, mesh, lams, kmax)) / (2 * h)
        np.testing.assert_allclose(g[:, p], fd, rtol=1e-5)


def test_tri_adjoint_gradient():
    """d chi(k) / d(J, D) of the kagome DM model (TRI core) by the checkpointed adjoint against
    the tangent-linear flow and central differences of the oracle's TRI flow."""
    cell, sites, B = W.kagome_dm_linear()
    th = torch.tensor(TRI_THETA, dtype=torch.float64, requires_grad=True)
    chi = susceptibility_adjoint(th, cell, sites, B, 2, MESH, LAMS, KPTS, sr.SR_TRI, every=3)
    g = np.array([torch.autograd.grad(chi[i], th, retain_graph=i + 1 < len(KPTS))[0].numpy() for i in range(len(KPTS))])
    th_t = torch.tensor(TRI_THETA, dtype=torch.float64, requires_grad=True)
    chi_t = susceptibility(th_t, cell, sites, B, 2, MESH, LAMS, KPTS, sr.SR_TRI)
    g_t = np.array([torch.autograd.grad(chi_t[i], th_t, retain_graph=i + 1 < len(KPTS))[0].numpy() for i in range(len(KPTS))])
    np.testing.assert_allclose(chi.detach().numpy(), chi_t.detach().numpy(), rtol=1e-12)
    np.testing.assert_allclose(g, g_t, rtol=1e-9, atol=1e-12 * np.abs(g_t).max())
    h = 1e-5

    def chi_o(theta):
        of = O.OracleFlowTRI(W.linear_model(cell, sites, B, theta, "TRI"), 2, MESH)
        for a, b in zip(LAMS[:-1], LAMS[1:]):
            of.euler(a, b)
        return of.chi_k(LAMS[-1], KPTS)

    for p in range(2):
        e = np.zeros(2)
        e[p] = h
        fd = (chi_o(TRI_THETA + e) - chi_o(TRI_THETA - e)) / (2 * h)
        np.testing.assert_allclose(g[:, p], fd, rtol=1e-5, atol=1e-5 * np.abs(fd).max())
