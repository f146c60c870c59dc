"""GPU parity of the TRI core (all 16 basis functions Gamma^{mu nu}, FP64) against the
oracle's TRI core, through the C ABI.

Tolerance: 1e-10 relative, normwise per component (max|x - x_ref| / max|x_ref|), as for the
other FP64 cores.  Models: the kagome antiferromagnet with out-of-plane DM couplings of the
paper's second worked example (imaginary-class functions generated by the flow), the same
model rotated in spin space (a DM vector along a generic axis: no spin symmetry left), and
the Heisenberg-Kitaev model, where the TRI core must reproduce the XYZ core, and the
Heisenberg-Kitaev-Gamma model (symmetric off-diagonal exchange).
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests.helpers import IMAG_CLASS, tri_oracle_to_gpu, tri_real

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402

TOL = 1e-10


def _rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def _cmp(got, exp, tol=TOL):
    """Normwise per component of [pair][t][c][r] arrays.  A component below 1e-6 of the whole
    vertex's scale is formed by cancellation (e.g. the mixed functions of the Kitaev-Gamma
    model early in the flow) and is compared on that floor."""
    floor = 1e-6 * np.abs(exp).max()
    for c in range(16):
        e = exp[:, :, c]
        if np.abs(e).max() == 0:
            assert np.abs(got[:, :, c]).max() < 1e-14, c
            continue
        err = np.abs(got[:, :, c] - e).max() / max(np.abs(e).max(), floor)
        assert err < tol, (c, err)


def _generic_rotation():
    a, b, c = 0.3, -0.7, 0.5
    th = np.sqrt(a * a + b * b + c * c)
    k = np.array([a, b, c]) / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


MODELS = [
    ("kagome_dm", lambda: W.kagome_dm(1.0, 0.5), 2),
    ("kagome_dm_rotated", lambda: W.rotated(W.kagome_dm(1.0, 0.4), _generic_rotation()), 2),
    ("honeycomb_kitaev", lambda: W.Model(W.honeycomb(), W.honeycomb_kitaev(0.2, -1.0).couplings, "TRI"), 2),
    ("honeycomb_kitaev_gamma", lambda: W.honeycomb_kitaev_gamma(0.1, -1.0, 0.5), 2),
]


def _load(fl, lat, of, lam):
    gam, G = of.get_state()
    Gg = tri_oracle_to_gpu(of, lat, G)
    fl.set_state(lam, torch.tensor(gam, device="cuda"), torch.tensor(Gg.reshape(-1), device="cuda"))


@pytest.mark.parametrize("name,mk,L", MODELS)
def test_tri_rhs_parity(name, mk, L):
    model = mk()
    mesh = O.mesh_exponential(6, 0.05, 10.0)
    of = O.OracleFlowTRI(model, L, mesh)
    for a, b in ((8.0, 4.0), (4.0, 2.0), (2.0, 1.0)):
        of.euler(a, b)
    dg_o, dG_o = of.rhs(0.7)
    lat = sr.Lattice.from_model(model, L, backend=sr.SR_TRI)
    fl = sr.Flow(lat, mesh, 1.0, sr.SR_FP64)
    assert fl.n_comp == 16
    _load(fl, lat, of, 1.0)
    dg, dG = fl.rhs(0.7)
    torch.cuda.synchronize()
    dg = dg.cpu().numpy()
    dG = dG.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s)
    assert _rel(dg, dg_o) < TOL
    exp = tri_oracle_to_gpu(of, lat, dG_o)
    _cmp(dG, exp)
    if name.startswith("kagome"):
        assert np.abs(exp[:, :, IMAG_CLASS]).max() > 1e-8   # the imaginary class is exercised
    # every oracle pair equals the signed stored value of its image
    den = np.abs(exp).max()
    for b in range(of.nb):
        blk = of.block(dG_o, b)
        for k, s in enumerate(of.sites(b)):
            r, comp, sign = lat.map_pair_components([0, 0, 0, b], s)
            e = np.transpose(tri_real(blk[k], 0), (1, 2, 0))       # [pair][t][c]
            g = dG[:, :, comp, r] * sign[None, None, :]
            assert np.abs(g - e).max() / den < TOL
    fl.close()


@pytest.mark.parametrize("name,mk,L", MODELS[:2])
def test_tri_euler_flow_and_chi_parity(name, mk, L):
    """Six Euler steps from the initial condition, then chi_ij (all 16 components) and chi(k)."""
    model = mk()
    mesh = O.mesh_exponential(6, 0.05, 10.0)
    lams = [8.0, 5.0, 3.0, 2.0, 1.4, 1.0, 0.7]
    of = O.OracleFlowTRI(model, L, mesh)
    lat = sr.Lattice.from_model(model, L, backend=sr.SR_TRI)
    fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP64)
    for a, b in zip(lams[:-1], lams[1:]):
        of.euler(a, b)
        fl.step(b, sr.SR_EULER)
    gam, G = fl.get_state()
    torch.cuda.synchronize()
    gam_o, G_o = of.get_state()
    assert _rel(gam.cpu().numpy(), gam_o) < TOL
    _cmp(G.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s), tri_oracle_to_gpu(of, lat, G_o))
    kp = np.array([[0.0, 0.0, 0.0], [1.3, -0.4, 0.0], [np.pi, np.pi / np.sqrt(3), 0.0], [2.1, 0.7, 0.0]])
    ck, cij = fl.measure(kp, want_ij=True)
    chi_o = of.chi(lams[-1])
    ck_o = of.chi_k(lams[-1], kp, chi_o)
    assert _rel(np.asarray(ck), ck_o) < TOL
    cij = cij.cpu().numpy()                      # [b][j][c], j in the library's site order
    sites = fl.chi_sites()
    for b in range(of.nb):
        e = tri_real(chi_o[b], 1)
        got = np.zeros_like(e)
        for jj in range(lat.N_tot):
            k = of.find(b, np.asarray(sites[b, jj, :3]) - 0, int(sites[b, jj, 3]))
            assert k >= 0
            got[k] = cij[b, jj]
        assert _rel(got, e) < TOL, _rel(got, e)
    fl.close()


def test_tri_core_reproduces_xyz_core():
    """Heisenberg-Kitaev model: TRI and XYZ cores agree on every diagonal function after
    Euler steps, the 12 others stay zero, and adaptive steps take the same cutoffs."""
    m = W.honeycomb_kitaev(0.2, -1.0)
    mesh = O.mesh_exponential(8, 0.02, 20.0)
    lx = sr.Lattice.from_model(m, 3)
    lt = sr.Lattice.from_model(m, 3, backend=sr.SR_TRI)
    assert lt.N_s == lx.N_s
    fx = sr.Flow(lx, mesh, 10.0, sr.SR_FP64)
    ft = sr.Flow(lt, mesh, 10.0, sr.SR_FP64)
    def compare(tol):
        gx, Gx = fx.get_state()
        gt, Gt = ft.get_state()
        torch.cuda.synchronize()
        Gx = Gx.cpu().numpy().reshape(fx.npair, fx.N, 4, lx.N_s)
        Gt = Gt.cpu().numpy().reshape(ft.npair, ft.N, 16, lt.N_s)
        assert _rel(gt.cpu().numpy(), gx.cpu().numpy()) < tol
        # component maps of the two cores may differ by the spin permutation of the symmetry
        # used; compare through the pair maps on every representative of the XYZ core, on the
        # scale of the whole vertex (Gamma^00 of this model is ~1e-6 of the spin parts and
        # formed by cancellation, so the cores' different summation orders show there first)
        scale = np.abs(Gx).max()
        for r, rep in enumerate(lx.representatives()):
            rt_, comp, sign = lt.map_pair_components([0, 0, 0, 0], rep)
            for c, cd in enumerate((0, 5, 10, 15)):
                assert np.abs(sign[cd] * Gt[:, :, comp[cd], rt_] - Gx[:, :, c, r]).max() / scale < tol
        off = [c for c in range(16) if c not in (0, 5, 10, 15)]
        assert np.abs(Gt[:, :, off]).max() == 0.0

    for lam in (7.0, 5.0, 3.0):
        fx.step(lam, sr.SR_EULER)
        ft.step(lam, sr.SR_EULER)
    compare(1e-12)
    # adaptive steps toward the strongly renormalised regime amplify the rounding differences
    # of the two summation orders; the controller must still take the same steps
    fx.step(1.0, sr.SR_RK_ADAPTIVE, rtol=1e-5, atol=1e-9)
    ft.step(1.0, sr.SR_RK_ADAPTIVE, rtol=1e-5, atol=1e-9)
    sx, st = fx.stats(), ft.stats()
    assert (sx["n_accept"], sx["n_reject"]) == (st["n_accept"], st["n_reject"])
    compare(1e-8)
    for f in (fx, ft):
        f.close()


def test_tri_sampled_parity_larger_lattice():
    """Kagome DM model at range 4 with 12 frequencies (several node blocks and a ragged last
    block per channel): sampled entries of the right-hand side against the oracle evaluated
    entry by entry."""
    model = W.kagome_dm(1.0, 0.5)
    L, N = 4, 12
    mesh = O.mesh_exponential(N, 0.01, 30.0)
    of = O.OracleFlowTRI(model, L, mesh)
    lat = sr.Lattice.from_model(model, L, backend=sr.SR_TRI)
    fl = sr.Flow(lat, mesh, 12.0, sr.SR_FP64)
    of.euler(12.0, 6.0)
    _load(fl, lat, of, 6.0)
    dg_o = of.prepare(2.0)
    dg, dG = fl.rhs(2.0)
    torch.cuda.synchronize()
    assert _rel(dg.cpu().numpy(), dg_o) < TOL
    dG = dG.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s)
    reps = lat.representatives()
    rng = np.random.default_rng(4)
    pairs = [(s, u) for s in range(N) for u in range(s + 1)]
    scale = np.abs(dG).max()
    for _ in range(24):
        r = int(rng.integers(0, lat.N_s))
        p = int(rng.integers(0, len(pairs)))
        ti = int(rng.integers(0, N))
        si, ui = pairs[p]
        rep = reps[r]
        e = tri_real(of.rhs_point(0, rep[:3], int(rep[3]), mesh[si], mesh[ti], mesh[ui]), 0)
        assert np.abs(dG[p, ti, :, r] - e).max() / scale < TOL
    fl.close()


@pytest.mark.parametrize("name,mk,L", MODELS[:2])
def test_tri_fp32_mixed_parity(name, mk, L):
    """FP32-mixed TRI flow (FP64 state, lookups and self-energy; rows, products and node sums in
    FP32): right-hand side within 1e-3 of the oracle (normwise per component), and after six
    Euler steps the state within 1e-3 and chi(k) within 1e-4."""
    model = mk()
    mesh = O.mesh_exponential(8, 0.03, 20.0)
    lams = [8.0, 5.0, 3.0, 2.0, 1.4, 1.0, 0.7]
    of = O.OracleFlowTRI(model, L, mesh)
    lat = sr.Lattice.from_model(model, L, backend=sr.SR_TRI)
    fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED)
    for a, b in zip(lams[:-1], lams[1:]):
        of.euler(a, b)
        fl.step(b, sr.SR_EULER)
    gam, G = fl.get_state()
    torch.cuda.synchronize()
    gam_o, G_o = of.get_state()
    assert _rel(gam.cpu().numpy(), gam_o) < 1e-3
    _cmp(G.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s), tri_oracle_to_gpu(of, lat, G_o), 1e-3)
    kp = np.array([[0.0, 0.0, 0.0], [1.3, -0.4, 0.0], [np.pi, np.pi / np.sqrt(3), 0.0]])
    ck, _ = fl.measure(kp, want_ij=False)
    assert _rel(np.asarray(ck), of.chi_k(lams[-1], kp)) < 1e-4
    # right-hand side at the oracle's state
    _load(fl, lat, of, lams[-1])
    dg_o, dG_o = of.rhs(0.5)
    dg, dG = fl.rhs(0.5)
    torch.cuda.synchronize()
    assert _rel(dg.cpu().numpy(), dg_o) < 1e-10          # the self-energy flow stays FP64
    _cmp(dG.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s), tri_oracle_to_gpu(of, lat, dG_o), 1e-3)
    fl.close()


def test_tri_unsupported_requests():
    lat = sr.Lattice.from_model(W.kagome_dm(1.0, 0.5), 1, backend=sr.SR_TRI)
    mesh = O.mesh_exponential(5, 0.05, 10.0)
    fl = sr.Flow(lat, mesh, 5.0, sr.SR_FP32_MIXED)
    with pytest.raises(sr.SrError) as e:
        fl.tensor_cores = True
    assert e.value.status == sr.SR_EUNSUPPORTED
    # the adjoint is defined for FP64 flows
    with pytest.raises(sr.SrError) as e:
        fl.rhs_adjoint(4.0, torch.zeros(fl.N, dtype=torch.float64, device="cuda"),
                       torch.zeros(fl.n_gamma, dtype=torch.float64, device="cuda"))
    assert e.value.status == sr.SR_EUNSUPPORTED
    fl.close()


@pytest.mark.parametrize("mode", [0, 1], ids=["autotuned", "persistent_others"])
def test_tri_flows_in_a_batch(mode):
    """TRI instances inside a batch (beside an SU2 and an XYZ instance): their own vertex kernel
    in the batch's captured step, the self-energy flow, nodes, update and FP32 copy in the
    batch's launches.  Bit for bit the same TRI flow stepped alone, and within the FP32-mixed
    tolerance of the oracle's TRI flow; forcing the persistent kernels (mode 1) leaves the TRI
    class on its own kernels."""
    lams = [8.0, 5.0, 3.0, 2.0, 1.4, 1.0]
    tri_models = [W.kagome_dm(1.0, 0.5), W.rotated(W.kagome_dm(1.0, 0.4), _generic_rotation())]
    mesh = O.mesh_exponential(5, 0.05, 10.0)
    lats = [sr.Lattice.from_model(m, 2, backend=sr.SR_TRI) for m in tri_models]
    alone = [sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED) for lat in lats]
    inb = [sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED) for lat in lats]
    others = [sr.Flow(sr.Lattice.from_model(W.square_j1j2(1.0, 0.3), 2), mesh, lams[0], sr.SR_FP32_MIXED),
              sr.Flow(sr.Lattice.from_model(W.honeycomb_kitaev(0.2, -1.0), 1), mesh, lams[0], sr.SR_FP32_MIXED)]
    for fl in alone:
        for lam in lams[1:]:
            fl.step(lam, sr.SR_EULER)
    b = sr.Batch(inb + others)
    b.force_launch(mode)
    b.run(lams, use_graph=True, autotune=True)
    launches = b.class_launches()
    classes = b.classes()
    assert len(launches) == len(classes)
    assert launches[-1]            # the TRI class (sorted last) runs the instances' own kernels
    for model, lat, f1, f2 in zip(tri_models, lats, alone, inb):
        g1, G1 = f1.get_state()
        g2, G2 = f2.get_state()
        assert f2.lam == lams[-1]
        assert torch.equal(G1, G2) and torch.equal(g1, g2)
        of = O.OracleFlowTRI(model, 2, mesh)
        for a, c in zip(lams[:-1], lams[1:]):
            of.euler(a, c)
        gam_o, G_o = of.get_state()
        assert _rel(g2.cpu().numpy(), gam_o) < 1e-3
        _cmp(G2.cpu().numpy().reshape(f2.npair, f2.N, 16, lat.N_s), tri_oracle_to_gpu(of, lat, G_o), 1e-3)
    b.close()
    for f in alone + inb + others:
        f.close()


@pytest.mark.parametrize("L,N", [(0, 2), (1, 2), (1, 3)])
def test_tri_edge_cases_against_oracle(L, N):
    """Degenerate sizes of the TRI core: range 0 (the on-site vertex only, one table entry), the
    smallest mesh (2 frequencies: one interval per axis), and a 3-point mesh; three Euler steps
    and the right-hand side against the oracle in FP64 and FP32-mixed."""
    model = W.kagome_dm(1.0, 0.5)
    mesh = O.mesh_exponential(N, 0.1, 5.0)
    lams = [4.0, 3.0, 2.0, 1.5]
    of = O.OracleFlowTRI(model, L, mesh)
    for a, b in zip(lams[:-1], lams[1:]):
        of.euler(a, b)
    dg_o, dG_o = of.rhs(1.2)
    lat = sr.Lattice.from_model(model, L, backend=sr.SR_TRI)
    for prec, tol in ((sr.SR_FP64, TOL), (sr.SR_FP32_MIXED, 1e-3)):
        fl = sr.Flow(lat, mesh, lams[0], prec)
        for b in lams[1:]:
            fl.step(b, sr.SR_EULER)
        _, G = fl.get_state()
        _, G_o = of.get_state()
        torch.cuda.synchronize()
        _cmp(G.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s), tri_oracle_to_gpu(of, lat, G_o), tol)
        _load(fl, lat, of, lams[-1])
        dg, dG = fl.rhs(1.2)
        torch.cuda.synchronize()
        assert _rel(dg.cpu().numpy(), dg_o) < 1e-10
        _cmp(dG.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s), tri_oracle_to_gpu(of, lat, dG_o), tol)
        fl.close()


def test_tri_adaptive_steps_finite():
    """Adaptive Dormand-Prince steps of the TRI core reach the target cutoff in FP64 and in
    FP32-mixed with finite states that agree to 1e-3 of the vertex scale (the two controllers
    take slightly different step sequences: FP32 rounding enters the embedded error estimate)."""
    lat = sr.Lattice.from_model(W.kagome_dm(1.0, 0.5), 2, backend=sr.SR_TRI)
    mesh = O.mesh_exponential(8, 0.02, 20.0)
    states, counts = [], []
    for prec in (sr.SR_FP64, sr.SR_FP32_MIXED):
        fl = sr.Flow(lat, mesh, 10.0, prec)
        reached = fl.step(0.5, sr.SR_RK_ADAPTIVE, rtol=1e-5, atol=1e-9)
        assert reached == 0.5
        _, G = fl.get_state()
        assert torch.isfinite(G).all()
        states.append(G.cpu().numpy())
        counts.append(fl.stats()["n_accept"])
        fl.close()
    assert np.abs(states[1] - states[0]).max() / np.abs(states[0]).max() < 1e-3
    assert abs(counts[0] - counts[1]) <= 0.2 * counts[0]


@pytest.mark.parametrize("prec,tol", [(sr.SR_FP64, TOL), (sr.SR_FP32_MIXED, 1e-3)])
def test_tri_full_size_sampled_parity(prec, tol):
    """The bench's TRI workload at full size (kagome DM, range 7, 32 frequencies: N_s = 34,
    2543 lattice-sum entries of 64 products each) in the launch configuration the bench times:
    the initial vertex J/4 with a synthetic self-energy gamma(w) (both sides set it; the
    self-energy flow of the bare vertex vanishes, the propagators do not), right-hand side at
    Lambda = 0.9 against the oracle on 48 sampled (site, triple) points, all 16 functions."""
    cfg = W.config("kagome_dm_L7")
    mesh = O.mesh_exponential(cfg.n_freq, cfg.w_min, cfg.w_max)
    gam = 0.2 * np.tanh(mesh) + 0.05 * mesh / (1 + mesh)
    of = O.OracleFlowTRI(cfg.model, cfg.L, mesh)
    _, G0 = of.get_state()
    of.set_state(gam, G0)
    lat = sr.Lattice.from_model(cfg.model, cfg.L)
    fl = sr.Flow(lat, mesh, cfg.lam_max, prec)
    _, Gd = fl.get_state()
    fl.set_state(cfg.lam_max, torch.tensor(gam, device="cuda"), Gd)
    dg, dG = fl.rhs(0.9)
    torch.cuda.synchronize()
    dG = dG.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s)
    reps = lat.representatives()
    rng = np.random.default_rng(9)
    N = cfg.n_freq
    pairs = [(s, u) for s in range(N) for u in range(s + 1)]
    ent, where = [], []
    for _ in range(48):
        r = int(rng.integers(0, lat.N_s))
        p = int(rng.integers(0, len(pairs)))
        ti = int(rng.integers(0, N))
        k = of.find(0, reps[r][:3], int(reps[r][3]))
        si, ui = pairs[p]
        ent.append((0, k, si, ti, ui))
        where.append((p, ti, r))
    got_o = of.rhs_entries(0.9, np.array(ent, dtype=np.int32))
    scale = np.abs(dG).max()
    assert scale > 0
    for (p, ti, r), e in zip(where, got_o):
        assert np.abs(dG[p, ti, :, r] - tri_real(e, 0)).max() / scale < tol
    fl.close()


def test_tri_structure_factor_components():
    """analysis.structure_factor_components on a TRI flow: the xx + yy + zz components equal the
    library's chi(k), and chi^{xy}(k) = conj(chi^{yx}(k))."""
    from paper_2109_13317_gb300.analysis import structure_factor_components
    lat = sr.Lattice.from_model(W.kagome_dm(1.0, 0.5), 2, backend=sr.SR_TRI)
    fl = sr.Flow(lat, O.mesh_exponential(6, 0.05, 10.0), 5.0, sr.SR_FP64)
    fl.step(3.0, sr.SR_EULER)
    kp = np.array([[0.0, 0.0, 0.0], [1.1, -0.3, 0.0], [np.pi, 0.7, 0.0]])
    F = structure_factor_components(fl, kp)
    ck, _ = fl.measure(kp, want_ij=False)
    np.testing.assert_allclose((F[:, 5] + F[:, 10] + F[:, 15]).real, ck, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(F[:, 6], np.conj(F[:, 9]), rtol=1e-12, atol=1e-15)
    fl.close()


def test_tri_rk_fixed_step_parity():
    """One Dormand-Prince 5(4) step of the TRI core (SR_RK_FIXED) against the oracle's TRI step:
    state within 1e-10 and the same normwise error estimate."""
    model = W.kagome_dm(1.0, 0.5)
    L, mesh = 1, O.mesh_exponential(5, 0.05, 10.0)
    of = O.OracleFlowTRI(model, L, mesh)
    for a, b in ((6.0, 4.0), (4.0, 3.0)):
        of.euler(a, b)
    lat = sr.Lattice.from_model(model, L, backend=sr.SR_TRI)
    fl = sr.Flow(lat, mesh, 3.0, sr.SR_FP64)
    _load(fl, lat, of, 3.0)
    err_o = of.dp54(3.0, 2.2, 1e-6, 1e-10)
    fl.step(2.2, sr.SR_RK_FIXED, 1e-6, 1e-10)
    err = fl.stats()["last_err"]
    g, G = fl.get_state()
    torch.cuda.synchronize()
    g_o, G_o = of.get_state()
    assert _rel(g.cpu().numpy(), g_o) < TOL
    _cmp(G.cpu().numpy().reshape(fl.npair, fl.N, 16, lat.N_s), tri_oracle_to_gpu(of, lat, G_o))
    assert abs(err - err_o) <= 1e-6 * err_o
    fl.close()
