"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: values printed in the
paper, closed forms derived by hand from the flow equations, invariants the equations
imply, or quadrature error bounds.  References are to arXiv:2109.13317.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- meshes (Sec. 5.2)

def test_frequency_mesh_matches_printed_values():
    row = [r for r in _read_golden("paper_meshes.txt") if r[0] == "freq"][0]
    n, wmin, wmax = int(row[1]), float(row[2]), float(row[3])
    first = [float(row[5]), float(row[6])]
    last = [float(row[8]), float(row[9])]
    m = O.mesh_exponential(n, wmin, wmax)
    assert len(m) == n
    np.testing.assert_allclose(m[:2], first, rtol=5e-6)
    np.testing.assert_allclose(m[-2:], last, rtol=5e-6)
    assert np.all(np.diff(m) > 0)
    # log spacing: constant ratio
    r = m[1:] / m[:-1]
    np.testing.assert_allclose(r, r[0], rtol=1e-12)


def test_cutoff_mesh_matches_printed_values():
    row = [r for r in _read_golden("paper_meshes.txt") if r[0] == "cutoff"][0]
    lmin, lmax, b = float(row[1]), float(row[2]), float(row[3])
    lam = O.cutoff_exponential(lmin, lmax, b)
    np.testing.assert_allclose(lam[:2], [float(row[5]), float(row[6])], rtol=1e-12)
    np.testing.assert_allclose(lam[-2:], [float(row[8]), float(row[9])], rtol=5e-6)
    assert lam[-1] >= lmin and lam[-1] * b < lmin


# ---------------------------------------------------------------- lattice (Sec. 4.1)

@pytest.mark.parametrize("name,L,ntot", [(r[0], int(r[1]), int(r[2])) for r in
                                         _read_golden("paper_lattice_counts.txt") if int(r[2]) > 0])
def test_sites_within_range_match_printed_counts(name, L, ntot):
    cell = W.CELLS[name]()
    f = O.OracleFlow(W.nn_heisenberg(cell), L, np.array([0.1, 1.0]))
    for b in range(cell.n_basis):
        assert f.nsite[b] == ntot


def test_square_range_counts_closed_form():
    # sites within Manhattan distance L on the square lattice: 2L^2 + 2L + 1
    for L in range(0, 8):
        f = O.OracleFlow(W.nn_heisenberg(W.square()), L, np.array([0.1, 1.0]))
        assert f.nsite[0] == 2 * L * L + 2 * L + 1


def test_couplings_symmetric():
    f = O.OracleFlow(W.honeycomb_kitaev(0.2, -1.0), 2, np.array([0.1, 1.0]))
    for b in range(2):
        sites = f.sites(b)
        for k, s in enumerate(sites):
            J = f.coupling(b, k)
            # reverse pair: from site s (cell n, basis b') back to (0, b)
            kk = f.find(int(s[3]), [-int(s[0]), -int(s[1]), -int(s[2])], b)
            np.testing.assert_array_equal(J.T, f.coupling(int(s[3]), kk))


# ---------------------------------------------------------------- spin algebra (Sec. 3)

def test_spin_tables_match_hand_derived_su2_and_xyz_rules():
    """The oracle contracts Pauli matrices numerically.  Check against the projected
    equations derived by hand with sigma^k sigma^l = delta + i eps sigma^m:
    s channel  (00) sum_k A_k B_k,  (mm) A0 Bm + Am B0 - (Aa Bb + Ab Ba)
    u channel  (00) sum_k A_k B_k,  (mm) A0 Bm + Am B0 + (Aa Bb + Ab Ba)
    t lattice sum 2 A_c B_c; on-site terms A_c sum_k s(k,c) C_k with s = -1 iff k, c
    distinct spatial indices; Sigma: Hartree 2 Gamma^00, Fock sum_k Gamma^kk."""
    coef, h, f, cd, cx, closed = O.spin_tables()
    assert closed
    exp = np.zeros((5, 4, 4, 4))
    for c in range(4):
        for k in range(4):
            exp[0, c, k, k] += 1.0 if c == 0 else 0.0
            exp[4, c, k, k] += 1.0 if c == 0 else 0.0
    for m in (1, 2, 3):
        a, b = [x for x in (1, 2, 3) if x != m]
        for t in (0, 4):
            exp[t, m, 0, m] += 1
            exp[t, m, m, 0] += 1
        exp[0, m, a, b] -= 1
        exp[0, m, b, a] -= 1
        exp[4, m, a, b] += 1
        exp[4, m, b, a] += 1

    def sgn(k, c):
        return -1.0 if (k != 0 and c != 0 and k != c) else 1.0
    for c in range(4):
        exp[1, c, c, c] = 2.0
        for k in range(4):
            exp[2, c, c, k] = sgn(k, c)
            exp[3, c, k, c] = sgn(k, c)
    np.testing.assert_array_equal(coef, exp)
    np.testing.assert_array_equal(h, [2, 0, 0, 0])
    np.testing.assert_array_equal(f, [1, 1, 1, 1])
    # chi: direct tr(s^mu s^k)^2 = 4 delta; exchange tr(s^mu s^k s^mu s^k) = 2 s(k, mu)
    np.testing.assert_array_equal(cd, 4 * np.eye(4))
    np.testing.assert_array_equal(cx, [[2 * sgn(k, m) for k in range(4)] for m in range(4)])


def test_su2_reduction_reuther_woelfle_form():
    """With Gamma^11 = Gamma^22 = Gamma^33 = s and Gamma^00 = d the tables reduce to the SU(2)
    equations: s channel (d, s) -> (dd + 3ss, 2ds - 2ss); u channel -> (dd + 3ss, 2ds + 2ss);
    on-site (A, C) -> (Ad (Cd + 3Cs), As (Cd - Cs))."""
    coef = O.spin_tables()[0]
    rng = np.random.default_rng(1)
    for _ in range(5):
        ad, as_, bd, bs = rng.normal(size=4)
        A = np.array([ad, as_, as_, as_])
        B = np.array([bd, bs, bs, bs])
        out = [np.einsum("ckl,k,l->c", coef[t], A, B) for t in range(5)]
        np.testing.assert_allclose(out[0], [ad * bd + 3 * as_ * bs] + [ad * bs + as_ * bd - 2 * as_ * bs] * 3, atol=1e-14)
        np.testing.assert_allclose(out[4], [ad * bd + 3 * as_ * bs] + [ad * bs + as_ * bd + 2 * as_ * bs] * 3, atol=1e-14)
        np.testing.assert_allclose(out[2], [ad * (bd + 3 * bs)] + [as_ * (bd - bs)] * 3, atol=1e-14)
        np.testing.assert_allclose(out[3], [bd * (ad + 3 * as_)] + [bs * (ad - as_)] * 3, atol=1e-14)


# ---------------------------------------------------------------- interpolation (Sec. 4.2)

def _fill_linear(f, coeffs):
    """Fill the stored octant with Gamma^{cc}(s,t,u) = a_c + b_c (s+u) + c_c t for c >= 1 and
    b_0 (s - u) for c = 0 (symmetric / antisymmetric under s <-> u as the relations demand),
    with site-dependent constants a_c(k)."""
    gam, G = f.get_state()
    N = f.N
    w = f.mesh
    si, ui = [], []
    for s in range(N):
        for u in range(s + 1):
            si.append(s)
            ui.append(u)
    si = np.array(si)
    ui = np.array(ui)
    S = w[si][:, None]
    U = w[ui][:, None]
    T = w[None, :]
    for b in range(f.nb):
        blk = f.block(G, b)
        for k in range(f.nsite[b]):
            a, bb, cc, b0 = coeffs(b, k)
            blk[k, 0] = b0 * (S - U) + 0 * T
            for c in (1, 2, 3):
                blk[k, c] = a[c] + bb[c] * (S + U) + cc[c] * T
    f.set_state(gam, G)


def test_interpolation_exact_for_linear_vertex_with_symmetry_relations():
    cell = W.square()
    mesh = O.mesh_exponential(10, 0.05, 20.0)
    f = O.OracleFlow(W.nn_heisenberg(cell), 2, mesh)
    rng = np.random.default_rng(3)
    sites = f.sites(0)
    # site constants must respect inversion (Gamma_{i1 i2} = Gamma_{i2 i1} on this lattice)
    keyvals = {}

    def coeffs(b, k):
        n = sites[k]
        key = (abs(n[0]), abs(n[1])) if abs(n[0]) >= abs(n[1]) else (abs(n[1]), abs(n[0]))
        if key not in keyvals:
            keyvals[key] = rng.normal(size=4)
        return keyvals[key], np.array([0, 0.3, -0.2, 0.1]), np.array([0, -0.15, 0.25, 0.05]), 0.4
    _fill_linear(f, coeffs)
    cl = lambda x: min(max(abs(x), mesh[0]), mesh[-1])
    for _ in range(300):
        k = int(rng.integers(0, len(sites)))
        s, t, u = rng.uniform(-25, 25, size=3)
        a, bb, cc, b0 = coeffs(0, k)
        v = f.lookup(0, sites[k][:3], 0, s, t, u)
        exp = [b0 * (cl(s) - cl(u))] + [a[c] + bb[c] * (cl(s) + cl(u)) + cc[c] * cl(t) for c in (1, 2, 3)]
        np.testing.assert_allclose(v, exp, rtol=1e-12, atol=1e-12)
    # beyond the truncation range the vertex vanishes
    np.testing.assert_array_equal(f.lookup(0, [3, 0, 0], 0, 1.0, 1.0, 1.0), 0.0)


def test_lookup_site_exchange_on_noncentrosymmetric_pairs():
    """Gamma_{i1 i2}(s,t,u) = Gamma_{i2 i1}(-s,t,u) (Eq. frg:parametrizationBasis2p): fill
    honeycomb sites with distinct constants and check sign flips read the reverse pair."""
    f = O.OracleFlow(W.nn_heisenberg(W.honeycomb()), 2, O.mesh_exponential(6, 0.1, 10.0))
    gam, G = f.get_state()
    rng = np.random.default_rng(5)
    for b in range(2):
        blk = f.block(G, b)
        for k in range(f.nsite[b]):
            blk[k, 1:] = rng.normal()
    f.set_state(gam, G)
    for b in range(2):
        for k, s in enumerate(f.sites(b)):
            d = s[:3]
            rev = f.lookup(int(s[3]), -d, b, 1.0, 2.0, 0.5)
            np.testing.assert_array_equal(f.lookup(b, d, int(s[3]), -1.0, 2.0, 0.5), rev)
            np.testing.assert_array_equal(f.lookup(b, d, int(s[3]), 1.0, 2.0, -0.5), rev)
            np.testing.assert_array_equal(f.lookup(b, d, int(s[3]), -1.0, -2.0, -0.5),
                                          f.lookup(b, d, int(s[3]), 1.0, 2.0, 0.5))


# ---------------------------------------------------------------- first RHS, closed form

def _bare_channel_integrals(lam, v):
    """delta-part propagator integrals at gamma = 0 (derived by hand from the sharp cutoff):
    I_s(s) = (2/L)[1/(s+L) - th(s-2L)/(s-L)], I_t = I_u = -I_s."""
    th = 1.0 if v - 2 * lam >= 0 else 0.0
    base = (2.0 / lam) * (1.0 / (v + lam) - (th / (v - lam) if th else 0.0))
    return base, -base, -base


def _bond_distance_sites(cell, L):
    """Test-side BFS (independent of the oracle): dict site -> bond distance from (0,0,0,0)."""
    from collections import deque
    start = (0, 0, 0, 0)
    dist = {start: 0}
    q = deque([start])
    while q:
        cur = q.popleft()
        if dist[cur] >= L:
            continue
        for (fb, tb, d0, d1, d2) in cell.bonds:
            for sgn, a, b in ((1, fb, tb), (-1, tb, fb)):
                if cur[3] != a:
                    continue
                nx = (cur[0] + sgn * d0, cur[1] + sgn * d1, cur[2] + sgn * d2, b)
                if nx not in dist:
                    dist[nx] = dist[cur] + 1
                    q.append(nx)
    return dist


def _J(model, i, j):
    """Coupling matrix J_{ij} from the model's interaction list (reading: J_ij = M, J_ji = M^T)."""
    acc = np.zeros((3, 3))
    for c in model.couplings:
        f, t = np.array(c.frm), np.array(c.to)
        if f[3] == i[3] and t[3] == j[3] and np.all(t[:3] - f[:3] == np.array(j[:3]) - np.array(i[:3])):
            acc += c.M
        if t[3] == i[3] and f[3] == j[3] and np.all(f[:3] - t[:3] == np.array(j[:3]) - np.array(i[:3])):
            acc += c.M.T
    return acc


@pytest.mark.parametrize("lam", [7.3, 1.9])
def test_first_rhs_at_bare_vertex_closed_form(lam):
    """At the initial condition (gamma = 0, Gamma = J/4) the Katanin part vanishes and the
    delta parts of the three bubbles integrate in closed form; the lattice sum reduces to
    sum_j J_{i1 j} J_{j i2}.  SU(2): dGamma^00 = (1/2pi) 3 (J/4)^2 (I_s + I_u),
    dGamma^zz = (1/2pi)[-2 (J/4)^2 I_s + 2 (J/4)^2 I_u - 2 I_t sum_j J_1j J_j2 / 16]."""
    model = W.square_j1j2(1.0, 0.5)
    L = 3
    mesh = O.mesh_exponential(7, 0.05, 30.0)
    f = O.OracleFlow(model, L, mesh)
    dg, dG = f.rhs(lam)
    np.testing.assert_array_equal(dg, 0.0)
    dist = _bond_distance_sites(model.cell, L)
    sites = f.sites(0)
    blk = f.block(dG, 0)
    i1 = (0, 0, 0, 0)
    assert set(map(tuple, sites)) == set(dist.keys())
    N = f.N
    pairs = [(s, u) for s in range(N) for u in range(s + 1)]
    for k, s2 in enumerate(sites):
        i2 = tuple(int(x) for x in s2)
        J12 = _J(model, i1, i2)[2, 2]
        # lattice sum over j within range of both sites
        rpa = 0.0
        for j in dist:
            if j in dist:
                dj2 = (i2[0] - j[0], i2[1] - j[1], i2[2] - j[2], i2[3])
                rj = (-j[0] + i2[0], -j[1] + i2[1], -j[2] + i2[2])
                # j within range of i2: shift to i2-centred coordinates
                if (j[0] - i2[0], j[1] - i2[1], j[2] - i2[2], j[3]) in dist:
                    rpa += _J(model, i1, j)[2, 2] * _J(model, j, i2)[2, 2]
        for p, (si, ui) in enumerate(pairs):
            for ti in range(N):
                Is = _bare_channel_integrals(lam, mesh[si])[0]
                It = _bare_channel_integrals(lam, mesh[ti])[1]
                Iu = _bare_channel_integrals(lam, mesh[ui])[2]
                e0 = 3 * (J12 / 4) ** 2 * (Is + Iu) / (2 * math.pi)
                ez = (-2 * (J12 / 4) ** 2 * Is + 2 * (J12 / 4) ** 2 * Iu - 2 * It * rpa / 16) / (2 * math.pi)
                got = blk[k, :, p, ti]
                np.testing.assert_allclose(got[0], e0, rtol=1e-12, atol=1e-15)
                np.testing.assert_allclose(got[1:], [ez] * 3, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- Sigma flow, closed form

def test_sigma_flow_closed_form_for_linear_density_vertex():
    """Gamma^00_{ij}(s,t,u) = a_j (s - u) (antisymmetric under s <-> u), spin parts zero and a
    given gamma: the self-energy flow is
    dgamma(w) = -(1/2pi)[H(w, L) - H(w, -L)] / (L + gamma(L)),
    H(w, w2) = 2 sum_j a_j (c|w+w2| - c|w-w2|) - a_0 (c|w+w2| - c(0)), c = clamp to the mesh."""
    cell = W.square()
    mesh = O.mesh_exponential(12, 0.01, 40.0)
    f = O.OracleFlow(W.nn_heisenberg(cell), 2, mesh)
    rng = np.random.default_rng(7)
    sites = f.sites(0)
    a = {}
    for k, s in enumerate(sites):
        key = tuple(sorted((abs(int(s[0])), abs(int(s[1])))))
        a.setdefault(key, rng.normal())
    ak = np.array([a[tuple(sorted((abs(int(s[0])), abs(int(s[1])))))] for s in sites])
    gam0, G = f.get_state()
    G[:] = 0.0
    blk = f.block(G, 0)
    N = f.N
    si = np.array([s for s in range(N) for u in range(s + 1)])
    ui = np.array([u for s in range(N) for u in range(s + 1)])
    for k in range(len(sites)):
        blk[k, 0] = (ak[k] * (mesh[si] - mesh[ui]))[:, None] * np.ones(N)[None, :]
    gam = 0.1 * np.sqrt(mesh)
    f.set_state(gam, G)
    cl = lambda x: min(max(abs(x), mesh[0]), mesh[-1])
    onsite = [k for k, s in enumerate(sites) if not np.any(s)][0]
    gL = np.interp(2.5, mesh, gam)
    for lam in (2.5,):
        for n, w in enumerate(mesh):
            def H(w2):
                hart = 2 * np.sum(ak * (cl(w + w2) - cl(w - w2)))
                fock = ak[onsite] * (cl(w + w2) - cl(0.0))
                return hart - fock
            exp = -(H(lam) - H(-lam)) / (lam + gL) / (2 * math.pi)
            got = f.sigma_rhs_point(w, lam)
            np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- quadrature of the Katanin part

def _odd_interp(mesh, vals, x):
    if x == 0.0:
        return 0.0
    v = np.interp(abs(x), mesh, vals)
    return v if x > 0 else -v


@pytest.mark.parametrize("ch", [0, 1, 2])
def test_regular_part_trapezoid_converges_to_adaptive_quadrature(ch):
    """Regular (Katanin) weights: sum_k W_k must approach (1/2pi) times the integral of
    g(a) r(b) + g(b) r(a) over the support, clipped to [-w_max, w_max], with the error
    shrinking like h^2 under mesh refinement.  The integrand here is built by the test
    from the paper's propagators with gamma and dgamma given as smooth odd functions."""
    lam, v = 0.7, 1.3
    errs = []
    for n in (40, 80, 160):
        mesh = O.mesh_exponential(n, 0.01, 30.0)
        f = O.OracleFlow(W.nn_heisenberg(W.square()), 1, mesh)
        gam = 0.3 * np.tanh(mesh)
        _, G = f.get_state()
        G[:] = 0.0
        f.set_state(gam, G)
        f.prepare(lam)  # dgamma = 0 for a zero vertex; set it by hand next
        dgam = -0.2 * mesh / (1 + mesh ** 2)
        f.lib.or_state_set(f.st, np.ascontiguousarray(gam), G)
        # inject the Katanin input through the scratch (dgam) slot
        import ctypes as C
        class _St(C.Structure):
            _fields_ = [("la", C.c_void_p), ("N", C.c_int), ("w", C.POINTER(C.c_double)), ("npair", C.c_int),
                        ("off", C.c_void_p), ("ntot", C.c_size_t), ("gam", C.POINTER(C.c_double)),
                        ("G", C.POINTER(C.c_double)), ("dgam", C.POINTER(C.c_double)), ("lam", C.c_double)]
        st = C.cast(f.st, C.POINTER(_St)).contents
        for i in range(n):
            st.dgam[i] = dgam[i]
        st.lam = lam
        x, Wt = f.channel_nodes(ch, v)
        reg = Wt[4:].sum() * 2 * math.pi

        def gr(a, b):
            ga = a + _odd_interp(mesh, gam, a)
            gb = b + _odd_interp(mesh, gam, b)
            return -_odd_interp(mesh, dgam, b) / (ga * gb * gb)

        def P(x):
            if ch == 0:
                a, b = x, v - x
            elif ch == 1:
                a, b = x, x - v
            else:
                a, b = x, v + x
            if abs(a) < lam or abs(b) < lam:
                return 0.0
            return gr(a, b) + gr(b, a)
        wmax = mesh[-1]
        brk = sorted(set([-wmax, wmax, lam, -lam] + ([v + lam, v - lam] if ch != 2 else [-v + lam, -v - lam])))
        brk = [b for b in brk if -wmax <= b <= wmax]
        ref = 0.0
        for lo, hi in zip(brk[:-1], brk[1:]):
            ref += integrate.quad(P, lo, hi, limit=400, points=[p for p in mesh if lo < p < hi][:300],
                                  epsabs=1e-13, epsrel=1e-11)[0]
        errs.append(abs(reg - ref) / abs(ref))
    assert errs[-1] < 6e-3
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 2.5


# ---------------------------------------------------------------- invariants of the flow

def _evolved(model, L, mesh, lams):
    f = O.OracleFlow(model, L, mesh)
    for a, b in zip(lams[:-1], lams[1:]):
        f.euler(a, b)
    return f


@pytest.fixture(scope="module")
def evolved_square():
    mesh = O.mesh_exponential(8, 0.02, 20.0)
    f = _evolved(W.square_j1j2(1.0, 0.4), 2, mesh, [8.0, 4.0, 2.0, 1.2])
    return f


def test_self_energy_flow_needs_equivalent_basis_sites():
    """The oracle keeps one self-energy for all sites (Sec. 4.1 reduction to a reference site),
    so it evaluates the self-energy flow at every basis site: on lattices whose sites are all
    equivalent (kagome, honeycomb) they agree to rounding; on the Lieb lattice (corner sites
    with four neighbours, edge sites with two) they differ, and the oracle returns NaN instead
    of basis site 0's flow."""
    mesh = O.mesh_exponential(5, 0.05, 10.0)
    O.OracleFlow.sigma_basis_spread(reset=True)
    for cell in (W.kagome(), W.honeycomb()):
        f = _evolved(W.nn_heisenberg(cell), 2, mesh, [8.0, 4.0, 2.0])
        dg, _ = f.rhs(1.3)
        assert np.all(np.isfinite(dg)) and np.abs(dg).max() > 0
    assert O.OracleFlow.sigma_basis_spread(reset=True) < 1e-12
    lieb = W.UnitCell("lieb", np.eye(3), np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0]], dtype=float),
                      [(0, 1, 0, 0, 0), (1, 0, 1, 0, 0), (0, 2, 0, 0, 0), (2, 0, 0, 1, 0)])
    f = O.OracleFlow(W.nn_heisenberg(lieb), 2, mesh)
    f.euler(8.0, 4.0)   # the bare vertex has no self-energy flow; the first step makes one
    dg = f.prepare(2.0)
    assert np.all(np.isnan(dg))
    assert O.OracleFlow.sigma_basis_spread(reset=True) > 1e-3


def test_self_energy_flow_is_odd(evolved_square):
    f = evolved_square
    for w in (0.03, 0.5, 1.7, 9.0, 30.0):
        a = f.sigma_rhs_point(w, 0.9)
        b = f.sigma_rhs_point(-w, 0.9)
        assert a != 0.0
        np.testing.assert_allclose(b, -a, rtol=1e-13, atol=1e-16)


def test_su2_closure_and_site_equivalence(evolved_square):
    """Heisenberg model: dGamma^xx = dGamma^yy = dGamma^zz; symmetry-equivalent pairs
    (square-lattice point group) flow identically; density vertex antisymmetric at s = u."""
    f = evolved_square
    dg, dG = f.rhs(0.9)
    blk = f.block(dG, 0)
    np.testing.assert_allclose(blk[:, 1], blk[:, 2], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(blk[:, 1], blk[:, 3], rtol=1e-12, atol=1e-15)
    sites = f.sites(0)
    groups = {}
    for k, s in enumerate(sites):
        key = tuple(sorted((abs(int(s[0])), abs(int(s[1])))))
        groups.setdefault(key, []).append(k)
    for ks in groups.values():
        for k in ks[1:]:
            np.testing.assert_allclose(blk[k], blk[ks[0]], rtol=1e-11, atol=1e-14)


def test_flow_symmetry_relations(evolved_square):
    """Eq. (frg:parametrizationBasis2p) for dGamma at generic (s,t,u): t -> -t, s -> -s with
    site exchange, u -> -u with site exchange, s <-> u with factor -xi(nu).  These are
    relations of the continuum flow; the trapezoid / trilinear discretization preserves them
    to discretization error only (measured ~1e-3 at N = 8..32, none to rounding).  A wrong
    argument or sign in any channel breaks them at O(1)."""
    f = evolved_square
    f.prepare(0.9)
    rng = np.random.default_rng(11)
    sites = f.sites(0)
    for _ in range(6):
        k = int(rng.integers(0, len(sites)))
        d = sites[k][:3]
        s, t, u = rng.uniform(0.05, 6.0, size=3)
        ref = f.rhs_point(0, d, 0, s, t, u)
        scale = np.abs(ref).max()
        assert scale > 0
        tol = dict(rtol=0, atol=3e-2 * scale)
        np.testing.assert_allclose(f.rhs_point(0, d, 0, s, -t, u), ref, **tol)
        np.testing.assert_allclose(f.rhs_point(0, -d, 0, -s, t, u), ref, **tol)
        np.testing.assert_allclose(f.rhs_point(0, -d, 0, s, t, -u), ref, **tol)
        np.testing.assert_allclose(f.rhs_point(0, d, 0, u, t, s), ref * np.array([-1, 1, 1, 1]), **tol)


# ---------------------------------------------------------------- susceptibility (Eq. frg:correlation)

def test_chi_bare_bubble_and_first_order():
    """J = 0: the vertex stays zero and chi_ii = 1/(2 pi Lambda) exactly, chi_{i != j} = 0.
    Constant Gamma = J/4: chi^zz_{ij} = -J_ij / (4 pi^2 Lambda^2) for i != j (exact under the
    product quadrature, whose weights integrate G^2 exactly)."""
    mesh = O.mesh_exponential(10, 0.01, 20.0)
    model = W.nn_heisenberg(W.square(), 0.0)
    f = O.OracleFlow(model, 2, mesh)
    for lam in (0.003, 0.37, 5.0, 25.0):
        chi = f.chi(lam)[0]
        sites = f.sites(0)
        on = [k for k, s in enumerate(sites) if not np.any(s)][0]
        np.testing.assert_allclose(chi[on], 1.0 / (2 * math.pi * lam), rtol=1e-13)
        mask = np.ones(len(sites), bool)
        mask[on] = False
        np.testing.assert_array_equal(chi[mask], 0.0)
    model = W.square_j1j2(1.0, 0.3)
    f = O.OracleFlow(model, 2, mesh)
    lam = 0.8
    chi = f.chi(lam)[0]
    for k, s in enumerate(f.sites(0)):
        if not np.any(s):
            np.testing.assert_allclose(chi[k, 1:], 1.0 / (2 * math.pi * lam), rtol=1e-13)
            continue
        J = f.coupling(0, k)[2, 2]
        np.testing.assert_allclose(chi[k, 1:], -J / (4 * math.pi ** 2 * lam ** 2), rtol=1e-12, atol=1e-16)
        assert abs(chi[k, 0]) < 1e-16


def test_chi_k_real_and_symmetric(evolved_square):
    f = evolved_square
    k = np.array([[0.3, 1.1, 0.0], [-0.3, -1.1, 0.0], [math.pi, math.pi, 0.0]])
    v = f.chi_k(1.2, k)
    np.testing.assert_allclose(v[0], v[1], rtol=1e-13)
    assert v[2] > v[0]


# ---------------------------------------------------------------- stepping (Sec. 4.3)

def test_euler_is_state_minus_step_times_rhs():
    mesh = O.mesh_exponential(6, 0.05, 10.0)
    f = _evolved(W.square_j1j2(1.0, 0.5), 1, mesh, [5.0, 2.0])
    g0, G0 = f.get_state()
    dg, dG = f.rhs(2.0)
    f.euler(2.0, 1.5)
    g1, G1 = f.get_state()
    np.testing.assert_allclose(g1, g0 - 0.5 * dg, rtol=1e-15, atol=1e-18)
    np.testing.assert_allclose(G1, G0 - 0.5 * dG, rtol=1e-15, atol=1e-18)


def test_dp54_tableau_order_conditions():
    """Dormand-Prince 5(4): row sums equal c, and the order conditions of a fifth-order
    (b5) and fourth-order (b4) method hold (Butcher trees up to order 5 / 4)."""
    c, a, b5, b4 = O.dp54_tableau()
    A = np.zeros((7, 7))
    A[:, :6] = a
    np.testing.assert_allclose(A.sum(1), c, atol=1e-15)
    from math import factorial
    Ac = A @ c
    conds = [  # (function of b, exact value, order)
        (lambda b: b.sum(), 1.0, 1), (lambda b: b @ c, 1 / 2, 2), (lambda b: b @ c ** 2, 1 / 3, 3),
        (lambda b: b @ Ac, 1 / 6, 3), (lambda b: b @ c ** 3, 1 / 4, 4), (lambda b: b @ (c * Ac), 1 / 8, 4),
        (lambda b: b @ (A @ c ** 2), 1 / 12, 4), (lambda b: b @ (A @ Ac), 1 / 24, 4),
        (lambda b: b @ c ** 4, 1 / 5, 5), (lambda b: b @ (c ** 2 * Ac), 1 / 10, 5),
        (lambda b: b @ (Ac * Ac), 1 / 20, 5), (lambda b: b @ (c * (A @ c ** 2)), 1 / 15, 5),
        (lambda b: b @ (A @ c ** 3), 1 / 20, 5), (lambda b: b @ (c * (A @ Ac)), 1 / 30, 5),
        (lambda b: b @ (A @ (c * Ac)), 1 / 40, 5), (lambda b: b @ (A @ (A @ c ** 2)), 1 / 60, 5),
        (lambda b: b @ (A @ (A @ Ac)), 1 / 120, 5)]
    for fn, v, order in conds:
        np.testing.assert_allclose(fn(b5), v, rtol=1e-13)
        if order <= 4:
            np.testing.assert_allclose(fn(b4), v, rtol=1e-13)
    # the embedded fourth-order solution is genuinely different from the fifth-order one
    assert abs(b4 @ c ** 4 - 1 / 5) > 1e-4


def test_dp54_step_agrees_with_fine_steps():
    """One Dormand-Prince step agrees with 16 substeps to high accuracy (the right-hand side
    is only piecewise smooth in Lambda, so no asymptotic rate is asserted)."""
    mesh = O.mesh_exponential(5, 0.1, 10.0)
    model = W.square_j1j2(1.0, 0.5)
    base = _evolved(model, 1, mesh, [6.0, 4.0])
    g0, G0 = base.get_state()
    a = O.OracleFlow(model, 1, mesh)
    a.set_state(g0, G0)
    err = a.dp54(4.0, 3.6, 1e-6, 1e-10)
    b = O.OracleFlow(model, 1, mesh)
    b.set_state(g0, G0)
    lams = np.linspace(4.0, 3.6, 17)
    for x, y in zip(lams[:-1], lams[1:]):
        b.dp54(x, y, 1e-6, 1e-10)
    ga, Ga = a.get_state()
    gb, Gb = b.get_state()
    # Euler with the same 16 substeps differs at first order, much more than the RK pair
    e = O.OracleFlow(model, 1, mesh)
    e.set_state(g0, G0)
    for x, y in zip(lams[:-1], lams[1:]):
        e.euler(x, y)
    ge, Ge = e.get_state()
    d_rk = np.abs(Ga - Gb).max() / np.abs(Gb).max()
    d_eu = np.abs(Ge - Gb).max() / np.abs(Gb).max()
    assert d_rk < 1e-6 and d_eu > 100 * d_rk
    assert err > 0


def test_rhs_finite_when_cutoff_equals_a_mesh_point():
    """Lambda on a mesh point makes a delta point fall on w = 0 with theta = 0: the term is
    absent (G vanishes below the cutoff) and the RHS stays finite."""
    mesh = O.mesh_exponential(6, 0.05, 5.0)
    f = _evolved(W.square_j1j2(1.0, 0.5), 1, mesh, [4.0, 2.0, 1.0])
    for lam in (mesh[0], mesh[2], mesh[-1]):
        dg, dG = f.rhs(lam)
        assert np.all(np.isfinite(dg)) and np.all(np.isfinite(dG))
