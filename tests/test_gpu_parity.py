"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 path within 1e-10 relative (normwise per object: max|x - x_ref| / max|x_ref|
for gamma, for each Gamma component and for chi); FP32-mixed path within 1e-3 on Gamma and
1e-4 on chi.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests.helpers import evolved_oracle, gpu_comp_map, oracle_to_gpu, synthetic_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402

FP64_TOL = 1e-10


def _rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def _compare_gamma(got, exp, tol):
    # normwise per component
    for c in range(got.shape[2]):
        e = exp[:, :, c]
        if np.abs(e).max() == 0:
            assert np.abs(got[:, :, c]).max() < 1e-14
            continue
        assert _rel(got[:, :, c], e) < tol, (c, _rel(got[:, :, c], e))


def _gpu_flow(model, L, mesh, lam, prec=sr.SR_FP64):
    lat = sr.Lattice.from_model(model, L)
    fl = sr.Flow(lat, mesh, lam, prec)
    return lat, fl


def _load_oracle_state(fl, lat, of, lam):
    gam, G = of.get_state()
    Gg = oracle_to_gpu(of, lat, G, fl.n_comp)
    fl.set_state(lam, torch.tensor(gam, device="cuda"), torch.tensor(Gg.reshape(-1), device="cuda"))


CASES = [
    ("square_j1j2", lambda: W.square_j1j2(1.0, 0.5), 2, 7, 0.02, 20.0),
    ("honeycomb", lambda: W.nn_heisenberg(W.honeycomb()), 2, 6, 0.05, 10.0),
    ("kagome", lambda: W.nn_heisenberg(W.kagome()), 2, 5, 0.05, 10.0),
    ("honeycomb_kitaev_xyz", lambda: W.honeycomb_kitaev(0.2, -1.0), 2, 5, 0.05, 10.0),
]


@pytest.mark.parametrize("name,mk,L,N,wmin,wmax", CASES)
def test_rhs_parity_evolved_state(name, mk, L, N, wmin, wmax):
    model = mk()
    mesh = O.mesh_exponential(N, wmin, wmax)
    of = evolved_oracle(model, L, mesh, [8.0, 4.0, 2.0, 1.0])
    lam = 0.7
    dg_o, dG_o = of.rhs(lam)
    lat, fl = _gpu_flow(model, L, mesh, 1.0)
    _load_oracle_state(fl, lat, of, 1.0)
    dg, dG = fl.rhs(lam)
    torch.cuda.synchronize()
    dg = dg.cpu().numpy()
    dG = dG.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s)
    assert _rel(dg, dg_o) < FP64_TOL
    exp = oracle_to_gpu(of, lat, dG_o, fl.n_comp)
    _compare_gamma(dG, exp, FP64_TOL)
    # every oracle pair equals the stored value of its image
    cm = gpu_comp_map(fl.n_comp)
    for b in range(of.nb):
        blk = of.block(dG_o, b)
        for k, s in enumerate(of.sites(b)):
            r, perm = lat.map_pair([0, 0, 0, b], s)
            for c in range(fl.n_comp):
                oc = cm[c]
                gc = perm[oc] if fl.n_comp == 4 else c
                e = blk[k, oc]
                g = dG[:, :, gc, r]
                den = max(np.abs(exp).max(), 1e-300)
                assert np.abs(g - e).max() / den < FP64_TOL


def test_rhs_parity_synthetic_state_edge_lambdas():
    """Synthetic symmetric state; cutoffs above w_max, between mesh points, below w_min."""
    model = W.square_j1j2(1.0, 0.5)
    mesh = O.mesh_exponential(6, 0.05, 5.0)
    of = O.OracleFlow(model, 2, mesh)
    gam, G = synthetic_state(of, model, seed=1)
    of.set_state(gam, G)
    lat, fl = _gpu_flow(model, 2, mesh, 1.0)
    _load_oracle_state(fl, lat, of, 1.0)
    for lam in (7.5, 1.234, 0.05, 0.011):
        dg_o, dG_o = of.rhs(lam)
        dg, dG = fl.rhs(lam)
        torch.cuda.synchronize()
        assert _rel(dg.cpu().numpy(), dg_o) < FP64_TOL
        _compare_gamma(dG.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s),
                       oracle_to_gpu(of, lat, dG_o, fl.n_comp), FP64_TOL)


def test_rhs_parity_minimal_mesh_and_onsite_only():
    """Degenerate cases: N = 2 frequencies; truncation range L = 0 (on-site vertex only)."""
    for L, N in ((0, 4), (1, 2)):
        model = W.square_j1j2(1.0, 0.5)
        mesh = O.mesh_exponential(N, 0.1, 3.0)
        of = evolved_oracle(model, L, mesh, [4.0, 2.0, 1.0])
        lat, fl = _gpu_flow(model, L, mesh, 1.0)
        _load_oracle_state(fl, lat, of, 1.0)
        dg_o, dG_o = of.rhs(0.8)
        dg, dG = fl.rhs(0.8)
        torch.cuda.synchronize()
        assert _rel(dg.cpu().numpy(), dg_o) < FP64_TOL
        _compare_gamma(dG.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s),
                       oracle_to_gpu(of, lat, dG_o, fl.n_comp), FP64_TOL)


def test_euler_flow_and_chi_parity():
    model = W.square_j1j2(1.0, 0.4)
    L, mesh = 2, O.mesh_exponential(8, 0.02, 20.0)
    lams = W.lambda_list(20.0, 0.3, 12)
    of = O.OracleFlow(model, L, mesh)
    lat, fl = _gpu_flow(model, L, mesh, lams[0])
    kpts = np.array([[0.0, 0.0, 0.0], [math.pi, math.pi, 0.0], [math.pi, 0.0, 0.0], [0.7, 1.9, 0.0]])
    for a, b in zip(lams[:-1], lams[1:]):
        of.euler(a, b)
        fl.step(b, sr.SR_EULER)
    g_o, G_o = of.get_state()
    g, G = fl.get_state()
    assert _rel(g.cpu().numpy(), g_o) < 1e-9
    _compare_gamma(G.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s),
                   oracle_to_gpu(of, lat, G_o, fl.n_comp), 1e-9)
    # correlations
    chi_o = of.chi(lams[-1])
    chik_o = of.chi_k(lams[-1], kpts, chi_o)
    chik, chi_ij = fl.measure(kpts)
    chi_ij = chi_ij.cpu().numpy()
    sites = fl.chi_sites()
    cm = gpu_comp_map(fl.n_comp)
    for b in range(lat.N_basis):
        for j, s in enumerate(sites[b]):
            k = of.find(b, s[:3] - np.array([0, 0, 0]), int(s[3]))
            assert k >= 0
            for c, oc in enumerate(cm):
                assert abs(chi_ij[b, j, c] - chi_o[b][k, oc]) <= FP64_TOL * np.abs(chi_o[b]).max()
    assert _rel(chik, chik_o) < FP64_TOL


def test_rk_fixed_step_parity():
    model = W.nn_heisenberg(W.kagome())
    L, mesh = 1, O.mesh_exponential(5, 0.05, 10.0)
    of = evolved_oracle(model, L, mesh, [6.0, 3.0])
    lat, fl = _gpu_flow(model, L, mesh, 3.0)
    _load_oracle_state(fl, lat, of, 3.0)
    err_o = of.dp54(3.0, 2.2, 1e-6, 1e-10)
    fl.step(2.2, sr.SR_RK_FIXED, 1e-6, 1e-10)
    err = fl.stats()["last_err"]
    g_o, G_o = of.get_state()
    g, G = fl.get_state()
    assert _rel(g.cpu().numpy(), g_o) < FP64_TOL
    _compare_gamma(G.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s),
                   oracle_to_gpu(of, lat, G_o, fl.n_comp), FP64_TOL)
    assert abs(err - err_o) <= 1e-6 * err_o


@pytest.mark.parametrize("name,mk,L,N,wmin,wmax", CASES)
def test_fp32_mixed_within_tolerance(name, mk, L, N, wmin, wmax):
    """FP32-mixed right-hand side (FP32 rows, products and accumulation; FP64 self-energy,
    propagators and node positions) against the FP64 oracle: 1e-3 on Gamma."""
    model = mk()
    mesh = O.mesh_exponential(N, wmin, wmax)
    of = evolved_oracle(model, L, mesh, [8.0, 4.0, 2.0, 1.0])
    lat, fl = _gpu_flow(model, L, mesh, 1.0, sr.SR_FP32_MIXED)
    _load_oracle_state(fl, lat, of, 1.0)
    dg_o, dG_o = of.rhs(0.7)
    dg, dG = fl.rhs(0.7)
    torch.cuda.synchronize()
    assert _rel(dg.cpu().numpy(), dg_o) < 1e-10   # self-energy flow stays FP64
    _compare_gamma(dG.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s),
                   oracle_to_gpu(of, lat, dG_o, fl.n_comp), 1e-3)


def test_full_size_sampled_parity():
    """Square J1-J2, L = 7, N = 48 (the flagship workload) on a synthetic symmetric state:
    the full GPU right-hand side against oracle values of sampled entries, including the
    s = u diagonal and the mesh ends."""
    cfg = W.config("square_j1j2_L7")
    mesh = O.mesh_exponential(cfg.n_freq, cfg.w_min, cfg.w_max)
    of = O.OracleFlow(cfg.model, cfg.L, mesh)
    gam, G = synthetic_state(of, cfg.model, seed=2)
    of.set_state(gam, G)
    lat, fl = _gpu_flow(cfg.model, cfg.L, mesh, 1.0)
    _load_oracle_state(fl, lat, of, 1.0)
    lam = 0.9
    dg, dG = fl.rhs(lam)
    torch.cuda.synchronize()
    dG = dG.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s)
    reps = lat.representatives()
    rng = np.random.default_rng(0)
    N = cfg.n_freq
    picks = [(0, 0, 0), (N - 1, N - 1, N - 1), (N - 1, 0, 0), (N - 1, N - 1, 0), (10, 3, 10)]
    picks += [tuple(sorted(rng.integers(0, N, 2))[::-1]) + (int(rng.integers(0, N)),) for _ in range(40)]
    ent = []
    for (si, ui, ti) in picks:
        r = int(rng.integers(0, lat.N_s))
        k = of.find(0, reps[r][:3], int(reps[r][3]))
        ent.append((0, k, si, ti, ui, r))
    ent = np.array(ent)
    out = of.rhs_entries(lam, ent[:, :5])
    dg_o = of.prepare(lam)
    assert _rel(dg.cpu().numpy(), dg_o) < FP64_TOL
    scale = np.abs(out).max()
    for (b, k, si, ti, ui, r), o in zip(ent, out):
        p = si * (si + 1) // 2 + ui
        got = dG[p, ti, :, r]
        assert abs(got[0] - o[0]) <= FP64_TOL * scale
        assert abs(got[1] - o[3]) <= FP64_TOL * scale


def test_nonfinite_state_is_reported():
    model = W.square_j1j2(1.0, 0.5)
    mesh = O.mesh_exponential(4, 0.1, 5.0)
    lat, fl = _gpu_flow(model, 1, mesh, 2.0)
    g, G = fl.get_state()
    G[5] = float("nan")
    fl.set_state(2.0, g, G)
    with pytest.raises(sr.SrError) as e:
        fl.step(1.5, sr.SR_EULER)
    assert e.value.status == 5


def _oracle_adaptive(of, lam0, lam1, rtol, atol, h0):
    """Dormand-Prince 5(4) with the stabilised PI controller of Hairer, Norsett & Wanner
    (accepted: h <- h clamp(0.9 err^-0.17 err_prev^0.04, 0.2, 5), no growth right after a
    rejection; rejected: h <- h max(0.2, 0.9 err^-0.2)), driven on the oracle's fixed step;
    returns the accepted cutoffs."""
    lam, h, acc = lam0, h0, [lam0]
    err_prev, rejected = 1e-4, False
    while lam > lam1:
        h_prop = h
        cut = lam + h < lam1
        if cut:
            h = lam1 - lam
        g0, G0 = of.get_state()
        err = of.dp54(lam, lam + h, rtol, atol)
        if err <= 1.0:
            lam = lam + h
            acc.append(lam)
            fac = 5.0 if err == 0 else 0.9 * err ** -0.17 * err_prev ** 0.04
            fac = min(1.0 if rejected else 5.0, max(0.2, fac))
            err_prev = max(err, 1e-4)
            h = h_prop if cut else h * fac
            rejected = False
        else:
            of.set_state(g0, G0)
            h *= max(0.2, min(1.0, 0.9 * err ** -0.2))
            rejected = True
    return acc


def test_adaptive_rk_parity():
    """Adaptive Dormand-Prince: (1) the GPU replays the oracle's accepted steps with fixed DP5
    steps and matches to FP64 tolerance; (2) the GPU's own controller reaches the target and
    agrees with the oracle's adaptive solution to the requested tolerance."""
    model = W.square_j1j2(1.0, 0.5)
    L, mesh = 1, O.mesh_exponential(6, 0.05, 10.0)
    rtol, atol = 1e-6, 1e-10
    of = O.OracleFlow(model, L, mesh)
    acc = _oracle_adaptive(of, 8.0, 2.0, rtol, atol, -0.5)
    assert len(acc) > 3
    g_o, G_o = of.get_state()
    lat, fl = _gpu_flow(model, L, mesh, 8.0)
    for lam in acc[1:]:
        fl.step(lam, sr.SR_RK_FIXED, rtol, atol)
    g, G = fl.get_state()
    assert _rel(g.cpu().numpy(), g_o) < 1e-9
    _compare_gamma(G.cpu().numpy().reshape(fl.npair, fl.N, fl.n_comp, lat.N_s),
                   oracle_to_gpu(of, lat, G_o, fl.n_comp), 1e-9)
    lat2, fl2 = _gpu_flow(model, L, mesh, 8.0)
    reached = fl2.step(2.0, sr.SR_RK_ADAPTIVE, rtol, atol)
    assert reached == 2.0
    st = fl2.stats()
    # first-same-as-last: 7 right-hand sides for the first attempt, 6 for every later one
    assert st["n_accept"] >= 2 and st["n_rhs"] == 6 * (st["n_accept"] + st["n_reject"]) + 1
    g2, G2 = fl2.get_state()
    # the two controllers take different step sequences (different first steps).  The RHS has
    # kinks in Lambda (break points and interpolation corners move with it), across which the
    # embedded error estimate understates the local error, so two rtol = 1e-6 integrations
    # differ at ~1e-4 of the state norm (measured 1.1e-4); both are checked normwise
    got = G2.cpu().numpy().reshape(fl2.npair, fl2.N, fl2.n_comp, lat2.N_s)
    exp = oracle_to_gpu(of, lat2, G_o, fl2.n_comp)
    assert np.abs(got - exp).max() / np.abs(exp).max() < 1e-3
    assert _rel(g2.cpu().numpy(), g_o) < 1e-3
