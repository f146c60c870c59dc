"""Pins of the oracle's general time-reversal-invariant (TRI) core (no GPU).

The TRI core keeps all 16 basis functions Gamma^{mu nu} of Eq. (frg:parametrization) of
arXiv:2109.13317 as complex numbers.  It is pinned by: hand-derived trace forms of the five
spin contractions of Eq. (frg:flowexplicit:2particle); reduction to the spin-diagonal oracle
on a Kitaev-like model (the paper: a core with fewer symmetry requirements may run a model of
higher symmetry); the real / imaginary classes of Eq. (frg:parametrizationBasis2p); covariance
under a global spin rotation; the closed-form first right-hand side at the bare vertex of a
Dzyaloshinskii-Moriya model (operator squares in the two-spin space); the frequency and site
relations of Eq. (frg:parametrizationBasis2p) with the mu <-> nu transposition.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

SIG = [np.eye(2, dtype=complex), np.array([[0, 1], [1, 0]], dtype=complex),
       np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], dtype=complex)]
REAL = np.array([(c // 4 == 0) == (c % 4 == 0) for c in range(16)])   # xi(mu) xi(nu) = 1


def _tr(*ms):
    out = np.eye(2, dtype=complex)
    for m in ms:
        out = out @ m
    return np.trace(out)


def _op(G, crossed=False):
    """Two-spin operator of a vertex G (4 x 4 components): sum G^{kl} sigma^k (x) sigma^l, or the
    crossed operator sum G^{kl} sigma^k (x) sigma^{l T}."""
    return sum(G[k, l] * np.kron(SIG[k], SIG[l].T if crossed else SIG[l]) for k in range(4) for l in range(4))


def _coeffs(T, crossed=False):
    """Components C^{rho lambda} of an operator in the basis of _op (Hilbert-Schmidt norm 4)."""
    return np.array([[np.trace(np.kron(SIG[r], SIG[l].T if crossed else SIG[l]) @ T) / 4 for l in range(4)]
                     for r in range(4)])


def test_tri_tables_match_trace_forms():
    """The oracle's tables come from literal index loops over Pauli matrices; here each term is
    derived by hand into operator products and traces:
      s (term 0):  T = O_A O_B, O = sum G^{kl} s^k (x) s^l               (ladder in the pair space)
      u (term 4):  T = K_B K_A, K = sum G^{kl} s^k (x) s^{lT}            (crossed pairing)
      t lattice sum (term 1): out^{kn} = sum_{lm} A^{kl} B^{mn} tr(s^l s^m)
      t on-site (term 2): out^{mu nu} = sum A^{mu l} C^{mn} tr(s^nu s^m s^l s^n) / 2
      t on-site (term 3): out^{mu nu} = sum C^{kl} B^{m nu} tr(s^mu s^l s^m s^k) / 2
    and Sigma / chi tables: hartree^{kl} = tr s^k tr s^l / 2, fock^{kl} = tr(s^l s^k) / 2,
    chi_dir = tr(s^mu s^k) tr(s^nu s^l), chi_exc = tr(s^mu s^l s^nu s^k)."""
    coef, hart, fock, cdir, cexc = O.tri_spin_tables()
    E = np.eye(16).reshape(16, 4, 4)
    for x in range(16):
        for y in range(16):
            A, B = E[x], E[y]
            s = _coeffs(_op(A) @ _op(B)).reshape(16)
            u = _coeffs(_op(B, True) @ _op(A, True), True).reshape(16)
            t1 = np.einsum("kl,mn,lm->kn", A, B, np.array([[_tr(SIG[l], SIG[m]) for m in range(4)] for l in range(4)]))
            t2 = np.zeros((4, 4), complex)
            t3 = np.zeros((4, 4), complex)
            for mu in range(4):
                for nu in range(4):
                    t2[mu, nu] = sum(A[mu, l] * B[m, n] * _tr(SIG[nu], SIG[m], SIG[l], SIG[n]) / 2
                                     for l in range(4) for m in range(4) for n in range(4))
                    t3[mu, nu] = sum(A[k, l] * B[m, nu] * _tr(SIG[mu], SIG[l], SIG[m], SIG[k]) / 2
                                     for k in range(4) for l in range(4) for m in range(4))
            for term, ref in ((0, s), (1, t1.reshape(16)), (2, t2.reshape(16)), (3, t3.reshape(16)), (4, u)):
                np.testing.assert_allclose(coef[term, :, x, y], ref, atol=1e-13, err_msg=f"term {term} x {x} y {y}")
    for x in range(16):
        k, l = divmod(x, 4)
        np.testing.assert_allclose(hart[x], np.trace(SIG[k]) * np.trace(SIG[l]) / 2, atol=1e-14)
        np.testing.assert_allclose(fock[x], _tr(SIG[l], SIG[k]) / 2, atol=1e-14)
        for o in range(16):
            mu, nu = divmod(o, 4)
            np.testing.assert_allclose(cdir[o, x], _tr(SIG[mu], SIG[k]) * _tr(SIG[nu], SIG[l]), atol=1e-14)
            np.testing.assert_allclose(cexc[o, x], _tr(SIG[mu], SIG[l], SIG[nu], SIG[k]), atol=1e-14)


def test_tri_tables_reduce_to_diagonal_tables():
    coef, *_ = O.tri_spin_tables()
    dcoef, *_ = O.spin_tables()
    d = [0, 5, 10, 15]
    for term in range(5):
        sub = coef[term][np.ix_(d, d, d)]
        np.testing.assert_allclose(sub.real, dcoef[term], atol=1e-14)
        np.testing.assert_allclose(sub.imag, 0.0, atol=1e-14)


@pytest.fixture(scope="module")
def hk_pair():
    mesh = O.mesh_exponential(6, 0.05, 10.0)
    m = W.honeycomb_kitaev(0.2, -1.0)
    d, t = O.OracleFlow(m, 1, mesh), O.OracleFlowTRI(m, 1, mesh)
    for f in (d, t):
        f.euler(5.0, 4.0)
        f.euler(4.0, 3.0)
    return d, t


def test_tri_reduces_to_diagonal_oracle(hk_pair):
    """Kitaev-like model (XYZ): the TRI core's diagonal components equal the spin-diagonal
    oracle's and the 12 others stay exactly zero, for the state after two Euler steps, the
    right-hand side and the correlations."""
    d, t = hk_pair
    gd, Gd = d.get_state()
    gt, Gt = t.get_state()
    np.testing.assert_allclose(gt, gd, rtol=1e-13, atol=1e-18)
    dgd, dGd = d.rhs(2.2)
    dgt, dGt = t.rhs(2.2)
    np.testing.assert_allclose(dgt, dgd, rtol=1e-12, atol=1e-18)
    cd, ct = d.chi(2.2), t.chi(2.2)
    diag = [0, 5, 10, 15]
    for b in range(d.nb):
        for X, Y in ((d.block(Gd, b), t.block(Gt, b)), (d.block(dGd, b), t.block(dGt, b))):
            np.testing.assert_allclose(Y[:, diag].real, X, rtol=1e-12, atol=1e-16)
            assert np.abs(Y[:, diag].imag).max() == 0.0
            assert np.abs(np.delete(Y, diag, axis=1)).max() == 0.0
        np.testing.assert_allclose(ct[b][:, diag].real, cd[b], rtol=1e-12, atol=1e-16)
        assert np.abs(np.delete(ct[b], diag, axis=1)).max() == 0.0


@pytest.fixture(scope="module")
def dm_flow():
    mesh = O.mesh_exponential(6, 0.05, 10.0)
    f = O.OracleFlowTRI(W.kagome_dm(1.0, 0.5), 1, mesh)
    f.euler(5.0, 4.0)
    f.euler(4.0, 3.0)
    return f


def test_tri_real_imaginary_classes(dm_flow):
    """Eq. (frg:parametrizationBasis2p): Gamma^{mu nu} is real if xi(mu) xi(nu) = 1 and
    imaginary otherwise.  The flow preserves the classes exactly, the mixed (imaginary)
    components are generated by the DM couplings, and the self-energy flow stays real."""
    f = dm_flow
    g, G = f.get_state()
    dg, dG = f.rhs(2.2)
    for X in (G, dG):
        for b in range(f.nb):
            B = f.block(X, b)
            assert np.abs(B[:, REAL].imag).max() == 0.0
            assert np.abs(B[:, ~REAL].real).max() == 0.0
            assert np.abs(B[:, ~REAL].imag).max() > 1e-7
    assert O.OracleFlowTRI.sigma_imag() == 0.0
    chi = f.chi(2.2)
    for c in chi:
        assert np.abs(c[:, REAL].imag).max() == 0.0
        assert np.abs(c[:, ~REAL].real).max() == 0.0


def test_tri_spin_rotation_covariance():
    """A global SO(3) rotation R of every coupling (M -> R M R^T) rotates the flow:
    Gamma^{mu nu} -> R4 Gamma R4^T with R4 = diag(1, R), for the right-hand side and chi."""
    from scipy.spatial.transform import Rotation
    mesh = O.mesh_exponential(6, 0.05, 10.0)
    m = W.kagome_dm(1.0, 0.5)
    R = Rotation.from_rotvec([0.3, -0.7, 0.5]).as_matrix()
    a = O.OracleFlowTRI(m, 1, mesh)
    b = O.OracleFlowTRI(W.rotated(m, R), 1, mesh)
    for f in (a, b):
        f.euler(5.0, 4.0)
    dga, dGa = a.rhs(3.0)
    dgb, dGb = b.rhs(3.0)
    np.testing.assert_allclose(dgb, dga, rtol=1e-12, atol=1e-17)
    R4 = np.eye(4)
    R4[1:, 1:] = R
    for bb in range(a.nb):
        A = a.block(dGa, bb).reshape(a.nsite[bb], 4, 4, a.npair, a.N)
        B = b.block(dGb, bb).reshape(a.nsite[bb], 4, 4, a.npair, a.N)
        np.testing.assert_allclose(np.einsum("ma,nb,kabpt->kmnpt", R4, R4, A), B, rtol=0, atol=1e-14)
    ca, cb = a.chi(3.0), b.chi(3.0)
    for bb in range(a.nb):
        A = ca[bb].reshape(-1, 4, 4)
        np.testing.assert_allclose(np.einsum("ma,nb,kab->kmn", R4, R4, A), cb[bb].reshape(-1, 4, 4), rtol=0, atol=1e-15)


def _bare_channel_integrals(lam, v):
    th = 1.0 if v - 2 * lam >= 0 else 0.0
    base = (2.0 / lam) * (1.0 / (v + lam) - (th / (v - lam) if th else 0.0))
    return base, -base, -base


def _J(model, i, j):
    acc = np.zeros((3, 3))
    for c in model.couplings:
        f, t = np.array(c.frm), np.array(c.to)
        if f[3] == i[3] and t[3] == j[3] and np.all(t[:3] - f[:3] == np.array(j[:3]) - np.array(i[:3])):
            acc += c.M
        if t[3] == i[3] and f[3] == j[3] and np.all(f[:3] - t[:3] == np.array(j[:3]) - np.array(i[:3])):
            acc += c.M.T
    return acc


@pytest.mark.parametrize("lam", [6.1, 1.7])
def test_tri_first_rhs_at_bare_vertex_closed_form(lam):
    """Kagome DM model at the initial condition (gamma = 0, Gamma = J/4 with off-diagonal J):
    dGamma = (1/2pi) [I_s C(O^2) + I_u C_x(K^2) - 2 I_t sum_j G_{1j} G_{j2}] with G = J/4 in
    the spin block, O / K the direct / crossed two-spin operators of G (see the trace-form
    test), I_s, I_t, I_u the closed-form bubbles; the on-site terms vanish (J_ii = 0)."""
    model = W.kagome_dm(1.0, 0.5)
    L = 2
    mesh = O.mesh_exponential(5, 0.05, 30.0)
    f = O.OracleFlowTRI(model, L, mesh)
    dg, dG = f.rhs(lam)
    np.testing.assert_array_equal(dg, 0.0)
    N = f.N
    pairs = [(s, u) for s in range(N) for u in range(s + 1)]
    for b in range(f.nb):
        sites = [tuple(int(x) for x in s) for s in f.sites(b)]
        blk = f.block(dG, b)
        i1 = (0, 0, 0, b)
        in_range = {b2: set(tuple(int(x) for x in s) for s in f.sites(b2)) for b2 in range(f.nb)}
        for k, i2 in enumerate(sites):
            G12 = np.zeros((4, 4), complex)
            G12[1:, 1:] = _J(model, i1, i2) / 4
            S = _coeffs(_op(G12) @ _op(G12))
            U = _coeffs(_op(G12, True) @ _op(G12, True), True)
            rpa = np.zeros((4, 4), complex)
            for j in sites:
                rel = (j[0] - i2[0], j[1] - i2[1], j[2] - i2[2], j[3])
                # j within range of i2: i2 -> j seen from i2's basis site
                if (-rel[0], -rel[1], -rel[2], i2[3]) not in in_range[j[3]]:
                    continue
                A = np.zeros((4, 4))
                B = np.zeros((4, 4))
                A[1:, 1:] = _J(model, i1, j) / 4
                B[1:, 1:] = _J(model, j, i2) / 4
                rpa += 2 * A @ B
            for p, (si, ui) in enumerate(pairs):
                for ti in range(N):
                    Is = _bare_channel_integrals(lam, mesh[si])[0]
                    It = _bare_channel_integrals(lam, mesh[ti])[1]
                    Iu = _bare_channel_integrals(lam, mesh[ui])[2]
                    ref = (Is * S + Iu * U - It * rpa) / (2 * math.pi)
                    np.testing.assert_allclose(blk[k, :, p, ti], ref.reshape(16), rtol=0, atol=1e-14)


def test_tri_flow_symmetry_relations(dm_flow):
    """Eq. (frg:parametrizationBasis2p) for dGamma at generic (s, t, u), all 16 components:
    t -> -t with xi(mu) xi(nu); s -> -s with site exchange and mu <-> nu; u -> -u with
    xi(mu) xi(nu), site exchange and mu <-> nu; s <-> u with -xi(nu).  As for the diagonal
    core, the discretization preserves them to discretization error only."""
    f = dm_flow
    f.prepare(2.2)
    rng = np.random.default_rng(12)
    xi = np.array([1, -1, -1, -1])
    xx = np.outer(xi, xi).reshape(16)
    tr = np.arange(16).reshape(4, 4).T.reshape(16)
    sites = f.sites(0)
    for _ in range(5):
        k = int(rng.integers(1, len(sites)))
        s2 = sites[k]
        d, b2 = s2[:3], int(s2[3])
        s, t, u = rng.uniform(0.05, 6.0, size=3)
        ref = f.rhs_point(0, d, b2, s, t, u)
        scale = np.abs(ref).max()
        assert scale > 0
        tol = dict(rtol=0, atol=3e-2 * scale)
        np.testing.assert_allclose(f.rhs_point(0, d, b2, s, -t, u) * xx, ref, **tol)
        # exchanged pair (i2, i1) seen from basis b2: site -d of basis 0
        np.testing.assert_allclose(f.rhs_point(b2, -d, 0, -s, t, u)[tr], ref, **tol)
        np.testing.assert_allclose(f.rhs_point(b2, -d, 0, s, t, -u)[tr] * xx, ref, **tol)
        np.testing.assert_allclose(f.rhs_point(0, d, b2, u, t, s) * -np.tile(xi, 4), ref, **tol)


def test_tri_rhs_entries_match_full_rhs(dm_flow):
    """The sampled-entry evaluation (used for timing samples) equals the full right-hand side."""
    f = dm_flow
    dg, dG = f.rhs(1.9)
    ent = np.array([[0, 1, 3, 2, 1], [1, 4, 5, 0, 5], [2, 0, 2, 4, 0]], dtype=np.int32)
    got = f.rhs_entries(1.9, ent)
    pairs = [(s, u) for s in range(f.N) for u in range(s + 1)]
    for e, g in zip(ent, got):
        b, k, si, ti, ui = (int(x) for x in e)
        np.testing.assert_allclose(g, f.block(dG, b)[k, :, pairs.index((si, ui)), ti], rtol=0, atol=1e-15)


def test_tri_chi_bare_vertex_closed_form():
    """Constant Gamma = J/4 with off-diagonal (DM) J: chi^{mu nu}_{ij} = -J^{mu nu}_{ij} /
    (4 pi^2 Lambda^2) for i != j and every spin pair mu, nu (the product quadrature integrates
    G^2 exactly, and the direct vertex term is 4 Gamma^{mu nu}); the functions with a density
    index vanish; on site (J_ii = 0) only the bubble 1/(2 pi Lambda) delta_{mu nu} remains."""
    mesh = O.mesh_exponential(10, 0.01, 20.0)
    model = W.kagome_dm(1.0, 0.5)
    f = O.OracleFlowTRI(model, 2, mesh)
    lam = 0.8
    chi = f.chi(lam)
    for b in range(f.nb):
        for k, s in enumerate(f.sites(b)):
            c = chi[b][k].reshape(4, 4)
            if int(s[3]) == b and not np.any(s[:3]):
                np.testing.assert_allclose(c, np.eye(4) / (2 * math.pi * lam), rtol=1e-13, atol=1e-17)
                continue
            J = f.coupling(b, k)
            np.testing.assert_allclose(c[1:, 1:].real, -J / (4 * math.pi ** 2 * lam ** 2), rtol=1e-12, atol=1e-16)
            assert np.abs(c[1:, 1:].imag).max() == 0.0
            assert np.abs(c[0, :]).max() < 1e-16 and np.abs(c[:, 0]).max() < 1e-16
    assert np.abs(model.couplings[0].M - model.couplings[0].M.T).max() > 0.9   # DM part present


def test_tri_dp54_step_matches_diagonal_oracle(hk_pair):
    """The TRI core's Dormand-Prince step on a Kitaev-like model equals the spin-diagonal
    oracle's step (same tableau and normwise error) on the diagonal functions."""
    d, t = hk_pair
    ed = d.dp54(2.5, 2.1, 1e-6, 1e-10)
    et = t.dp54(2.5, 2.1, 1e-6, 1e-10)
    np.testing.assert_allclose(et, ed, rtol=1e-10)
    _, Gd = d.get_state()
    _, Gt = t.get_state()
    for b in range(d.nb):
        np.testing.assert_allclose(t.block(Gt, b)[:, [0, 5, 10, 15]].real, d.block(Gd, b), rtol=1e-12, atol=1e-16)
