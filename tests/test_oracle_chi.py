"""Pins of the oracle's correlation function (Sec. 3, Eq. frg:correlation) against closed
forms and continuum integrals (no GPU).

The vertex term of Eq. (frg:correlation) contracts Gamma((i,w1,a1'),(j,w2,a2');(i,w1,a1),
(j,w2,a2)) with sigma^mu sigma^nu.  By the parametrization Eq. (frg:parametrization) it has
two parts:
  direct:   Gamma^{kl}_{ij}(w1+w2, 0, w1-w2)      times tr(s^mu s^k) tr(s^nu s^l),
  exchange: Gamma^{kl}_{ii}(w1+w2, w2-w1, 0)      times tr(s^mu s^l s^nu s^k), only for i = j,
entering as direct - exchange (the -(1' <-> 2') of the parametrization).  The traces are
computed here from explicit Pauli matrices; the oracle builds its tables by index loops.

Pins:
  * a self-energy gamma != 0 and a frequency-independent vertex: the product quadrature is
    exact (its node weights integrate G^2 = -1/(w+gamma(w))^2 exactly for piecewise-linear
    gamma), so chi equals a closed form in I = int_{|w|>Lambda} dw / (w+gamma(w))^2, which is
    computed here by adaptive quadrature (1e-12);
  * a frequency-dependent vertex a phi(t) + b psi(min(s, u)) on the on-site and on the
    off-site pairs: the direct part sees psi(||w1|-|w2||) and phi(0), the exchange part
    phi(|w1-w2|) and psi(0).  The oracle must converge (second order in the mesh spacing) to
    the continuum double integrals, computed here by nested adaptive quadrature, and the
    alternative routings (t and u exchanged in either part) must be far outside the
    tolerance.
Both for the spin-diagonal oracle (XYZ storage) and for the general time-reversal-invariant
core (all 16 functions, symmetric spin-spin couplings).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import oracle as O

SIG = [np.eye(2, dtype=complex), np.array([[0, 1], [1, 0]], dtype=complex),
       np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], dtype=complex)]


def _tr(*ms):
    out = np.eye(2, dtype=complex)
    for m in ms:
        out = out @ m
    return np.trace(out)


# tr(s^mu s^k) tr(s^nu s^l) and tr(s^mu s^l s^nu s^k), indexed [mu][nu][k][l]
DIR = np.array([[[[_tr(SIG[m], SIG[k]) * _tr(SIG[n], SIG[l]) for l in range(4)] for k in range(4)]
                 for n in range(4)] for m in range(4)])
EXC = np.array([[[[_tr(SIG[m], SIG[l], SIG[n], SIG[k]) for l in range(4)] for k in range(4)]
                 for n in range(4)] for m in range(4)])

TAU, SIGMA, RHO = 1.5, 3.0, 2.5   # widths of the three frequency shapes


def phi(x):
    return np.exp(-np.asarray(x) ** 2 / (2 * TAU ** 2))


def psi(x):
    return np.exp(-np.asarray(x) ** 2 / (2 * SIGMA ** 2))


def rho(x):
    return np.exp(-np.asarray(x) ** 2 / (2 * RHO ** 2))


def _g2_integral(mesh, gam, lam):
    """int_{Lambda}^{inf} dw / (w + gamma(w))^2 with gamma linear between mesh points and
    constant beyond the last one (the interpolation of Sec. 4.2), by adaptive quadrature."""
    def gamma(w):
        return np.interp(w, mesh, gam)
    pts = [m for m in mesh if m > lam]
    f = lambda w: 1.0 / (w + gamma(w)) ** 2
    val = 0.0
    edges = [lam] + pts
    for a, b in zip(edges[:-1], edges[1:]):
        val += integrate.quad(f, a, b, epsabs=0, epsrel=1e-13)[0]
    top = edges[-1]
    val += integrate.quad(f, top, np.inf, epsabs=0, epsrel=1e-13)[0]
    return val


def _continuum(lam):
    """Double integrals over |w1|, |w2| > Lambda with measure dw1 dw2 / (w1^2 w2^2) (gamma = 0),
    by nested adaptive quadrature over a, b = |w1|, |w2| >= Lambda (|w1 + w2| and |w1 - w2| are
    a + b and |a - b| for equal signs, the other way round for opposite signs):
      I2 = int 1 = (2 / Lambda)^2,
      J_psi = int psi(||w1| - |w2||),  J_phi = int phi(|w1 - w2|),
      K_dir = int rho(|w1| + |w2|),   K_exc = int rho(|w1 + w2|) phi(|w1 - w2|),
      K_mut = int rho(|w1 - w2|) phi(|w1 - w2|)."""
    opt = dict(epsabs=1e-14, epsrel=1e-12, limit=200)

    def diag_split(F):
        # int_lam^inf int_lam^inf F(a + b, |a - b|) / (a^2 b^2) for F symmetric in a <-> b:
        # twice the part b = a + d, d > 0
        inner = lambda a: integrate.quad(lambda d: F(2 * a + d, d) / (a + d) ** 2, 0, np.inf, **opt)[0] / a ** 2
        return 2 * integrate.quad(inner, lam, np.inf, **opt)[0]

    def same(Fp, Fm):
        # sum over the four sign combinations of F(|w1 + w2|, |w1 - w2|): two equal-sign ones
        # (F(a + b, |a - b|)) and two opposite-sign ones (F(|a - b|, a + b))
        return 2 * diag_split(Fp) + 2 * diag_split(Fm)

    J_psi = same(lambda p, m: psi(m), lambda p, m: psi(m))          # ||w1|-|w2|| = |a - b|
    J_phi = same(lambda p, m: phi(m), lambda p, m: phi(p))
    K_dir = same(lambda p, m: rho(p), lambda p, m: rho(p))          # |w1|+|w2| = a + b
    K_exc = same(lambda p, m: rho(p) * phi(m), lambda p, m: rho(m) * phi(p))
    K_mut = same(lambda p, m: rho(m) * phi(m), lambda p, m: rho(p) * phi(p))
    return dict(I2=(2.0 / lam) ** 2, J_psi=float(J_psi), J_phi=float(J_phi), K_dir=float(K_dir),
                K_exc=float(K_exc), K_mut=float(K_mut))


def _vertex_term(A, B, C, onsite, J, route="paper"):
    """-(1/16 pi^2) x (direct - exchange) for the vertex A^{kl} phi(t) + B^{kl} psi(min(s,u)) +
    C^{kl} rho(max(s,u)) phi(t) (4 x 4 coefficient matrices), chi^{mu nu} as a 4 x 4 array.
    route names the arguments each part reads: "paper" = direct (w1+w2, 0, w1-w2), exchange
    (w1+w2, w2-w1, 0); plausible mistakes: "swap_dir" / "swap_exc" exchange the t and u slots
    of one part, "exc_s" reads s = w1 - w2 in the exchange part."""
    # (phi part, psi part, rho phi part) of each argument routing
    at_t0 = (phi(0) * J["I2"], J["J_psi"], phi(0) * J["K_dir"])   # (w1+w2, 0, w1-w2)
    at_u0 = (J["J_phi"], psi(0) * J["I2"], J["K_exc"])             # (w1+w2, w2-w1, 0)
    exc_s = (J["J_phi"], psi(0) * J["I2"], J["K_mut"])             # (w1-w2, w2-w1, 0)
    d_args = at_u0 if route == "swap_dir" else at_t0
    e_args = {"swap_exc": at_t0, "exc_s": exc_s}.get(route, at_u0)
    Vd = A * d_args[0] + B * d_args[1] + C * d_args[2]
    Ve = A * e_args[0] + B * e_args[1] + C * e_args[2]
    out = np.einsum("mnkl,kl->mn", DIR, Vd)
    if onsite:
        out = out - np.einsum("mnkl,kl->mn", EXC, Ve)
    return -out / (16 * math.pi ** 2)


@pytest.fixture(scope="module")
def continuum():
    return _continuum(1.0)


def _sym_spin(rng):
    """Random symmetric spin-spin coefficients (density row / column zero), 4 x 4."""
    m = np.zeros((4, 4))
    x = rng.normal(size=(3, 3))
    m[1:, 1:] = 0.5 * (x + x.T)
    return m


def _fill_diag(f, shapes, const=False):
    """Spin-diagonal oracle: the pair of basis b and site gets Gamma^{cc} = A^{cc} phi(t) +
    B^{cc} psi(u) + C^{cc} rho(s) phi(t) on the stored octant (s >= u; the s <-> u relation then
    makes these psi(min(s, u)) and rho(max(s, u))), (A, B, C) = shapes(b, site), or the constant
    A^{cc} with const; the density component stays zero."""
    gam, G = f.get_state()
    N = f.N
    si, ui = np.array([(s, u) for s in range(N) for u in range(s + 1)]).T
    S = f.mesh[si][:, None]
    U = f.mesh[ui][:, None]
    T = f.mesh[None, :]
    for b in range(f.nb):
        blk = f.block(G, b)
        for k, site in enumerate(f.sites(b)):
            A, B, C = shapes(b, site)
            blk[k, 0] = 0.0
            for c in (1, 2, 3):
                blk[k, c] = (A[c, c] + 0.0 * U * T if const
                             else A[c, c] * phi(T) + B[c, c] * psi(U) + C[c, c] * rho(S) * phi(T))
    return gam, G


def _fill_tri(f, shapes, const=False):
    """As _fill_diag for the TRI core, all 16 functions Gamma^{mu nu}."""
    gam, G = f.get_state()
    N = f.N
    si, ui = np.array([(s, u) for s in range(N) for u in range(s + 1)]).T
    S = f.mesh[si][:, None]
    U = f.mesh[ui][:, None]
    T = f.mesh[None, :]
    for b in range(f.nb):
        blk = f.block(G, b)
        for k, site in enumerate(f.sites(b)):
            A, B, C = shapes(b, site)
            for mu in range(4):
                for nu in range(4):
                    blk[k, 4 * mu + nu] = (A[mu, nu] + 0.0 * U * T if const else
                                           A[mu, nu] * phi(T) + B[mu, nu] * psi(U) + C[mu, nu] * rho(S) * phi(T))
    return gam, G


def _is_onsite(b, site):
    return int(site[3]) == b and not np.any(site[:3])


# ---------------------------------------------------------------- bubble with a self-energy

@pytest.mark.parametrize("lam", [0.013, 0.6, 7.0])
def test_chi_bubble_with_self_energy_exact(lam):
    """Vertex zero, odd gamma != 0: chi^{mu mu}_{ii} = (1/2 pi) int_{Lambda}^{inf} dw /
    (w + gamma(w))^2 (the bubble -(1/8 pi) int G^2 tr(s^mu s^mu) with G = 1/(i(w+gamma)))
    exactly, and chi_{i != j} = 0."""
    mesh = O.mesh_exponential(14, 0.01, 30.0)
    f = O.OracleFlow(W.nn_heisenberg(W.square(), 0.0), 2, mesh)
    gam, G = f.get_state()
    gam = 0.4 * np.sin(mesh) / (1 + 0.1 * mesh) + 0.05 * mesh ** 0.5
    f.set_state(gam, np.zeros_like(G))
    ref = _g2_integral(mesh, gam, lam) / (2 * math.pi)
    chi = f.chi(lam)[0]
    for k, site in enumerate(f.sites(0)):
        if _is_onsite(0, site):
            np.testing.assert_allclose(chi[k], ref, rtol=1e-11)
        else:
            np.testing.assert_array_equal(chi[k], 0.0)


def test_chi_constant_vertex_with_self_energy_exact():
    """Frequency-independent vertex, gamma != 0: the product quadrature is exact, so
    chi^{mu mu} = delta_ij I/(2 pi) - (I'^2 / 16 pi^2) [4 c_mu - delta_ij sum_k
    tr(s^mu s^k s^mu s^k) c_k], with I' = 2 int_{Lambda}^{inf} dw/(w+gamma)^2 over both signs;
    on-site coefficients c_k all different (XYZ storage), off-site d_k."""
    mesh = O.mesh_exponential(12, 0.02, 40.0)
    model = W.nn_heisenberg(W.square(), 0.0)
    model.backend = "XYZ"
    f = O.OracleFlow(model, 2, mesh)
    rng = np.random.default_rng(11)
    c_on = np.diag([0.0, 0.61, -0.37, 0.23])
    d_off = {}

    def shapes(b, site):
        if _is_onsite(b, site):
            return c_on, None, None
        key = tuple(sorted(np.abs(site[:2])))   # constants respect the lattice's point group
        if key not in d_off:
            d_off[key] = np.diag(np.r_[0.0, rng.normal(size=3)])
        return d_off[key], None, None
    gam_v = 0.3 * np.tanh(mesh) + 0.02 * mesh
    _, G = _fill_diag(f, shapes, const=True)
    f.set_state(gam_v, G)
    lam = 0.45
    I = _g2_integral(mesh, gam_v, lam)
    Ip2 = (2 * I) ** 2
    chi = f.chi(lam)[0]
    for k, site in enumerate(f.sites(0)):
        on = _is_onsite(0, site)
        C = shapes(0, site)[0]
        exp = np.einsum("mnkl,kl->mn", DIR, C).real
        if on:
            exp = exp - np.einsum("mnkl,kl->mn", EXC, C).real
        exp = -Ip2 * np.diag(exp) / (16 * math.pi ** 2)
        if on:
            exp = exp + I / (2 * math.pi)
        np.testing.assert_allclose(chi[k], exp, rtol=1e-11, atol=1e-15)
    # the exchange part is a visible share of the on-site value
    k_on = [k for k, s in enumerate(f.sites(0)) if _is_onsite(0, s)][0]
    exc_share = np.einsum("mnkl,kl->mn", EXC, c_on).real.diagonal() * Ip2 / (16 * math.pi ** 2)
    assert np.abs(exc_share).max() > 0.05 * np.abs(chi[k_on]).max()


def test_tri_chi_constant_vertex_with_self_energy_exact():
    """TRI core: symmetric spin-spin on-site coefficients c^{kl} (all 9, off-diagonal ones
    included) and off-site d^{kl}, gamma != 0: chi^{mu nu} = delta_ij delta_{mu nu} I/(2 pi) -
    (I'^2/16 pi^2) [sum_kl tr(s^mu s^k) tr(s^nu s^l) c^{kl} - delta_ij sum_kl
    tr(s^mu s^l s^nu s^k) c^{kl}] for all 16 (mu, nu), imaginary parts included."""
    mesh = O.mesh_exponential(10, 0.02, 40.0)
    model = W.nn_heisenberg(W.square(), 0.0)
    f = O.OracleFlowTRI(model, 1, mesh)
    rng = np.random.default_rng(5)
    c_on = _sym_spin(rng)
    d_off = _sym_spin(rng)
    shapes = lambda b, s: ((c_on if _is_onsite(b, s) else d_off), None, None)
    _, G = _fill_tri(f, shapes, const=True)
    gam_v = 0.25 * np.tanh(2 * mesh)
    f.set_state(gam_v, G)
    lam = 0.7
    I = _g2_integral(mesh, gam_v, lam)
    Ip2 = (2 * I) ** 2
    chi = f.chi(lam)[0]
    for k, site in enumerate(f.sites(0)):
        on = _is_onsite(0, site)
        C = c_on if on else d_off
        V = np.einsum("mnkl,kl->mn", DIR, C)
        if on:
            V = V - np.einsum("mnkl,kl->mn", EXC, C)
        exp = -Ip2 * V / (16 * math.pi ** 2)
        if on:
            exp = exp + np.eye(4) * I / (2 * math.pi)
        np.testing.assert_allclose(chi[k].reshape(4, 4), exp, rtol=1e-11, atol=1e-15)
    # off-diagonal couplings reach mixed components through the exchange traces
    assert np.abs(np.einsum("mnkl,kl->mn", EXC, c_on)[0, 1:]).max() + \
        np.abs(np.einsum("mnkl,kl->mn", EXC, c_on)[1:, 1:] - np.diag(np.diag(
            np.einsum("mnkl,kl->mn", EXC, c_on)[1:, 1:]))).max() > 0.1


# ---------------------------------------------------------------- frequency routing

A_ON, B_ON, C_ON = np.diag([0.0, 0.7, -0.4, 0.25]), np.diag([0.0, -0.3, 0.55, 0.9]), np.diag([0.0, 1.6, 1.9, -1.3])
A_OFF, B_OFF, C_OFF = np.diag([0.0, 0.2, 0.5, -0.6]), np.diag([0.0, 0.45, -0.15, 0.3]), np.diag([0.0, -0.4, 0.1, 0.6])


def _routing_errors(N, continuum, tri=False):
    """Per stored pair of a square lattice (range 1): (on site?, normwise relative error of the
    oracle's vertex term against the continuum value, smallest relative distance to a wrongly
    routed continuum value)."""
    mesh = O.mesh_exponential(N, 1e-2, 1e2)
    model = W.nn_heisenberg(W.square(), 0.0)
    if tri:
        f = O.OracleFlowTRI(model, 1, mesh)
        rng = np.random.default_rng(23)
        mats = {on: (_sym_spin(rng), _sym_spin(rng), 3 * _sym_spin(rng)) for on in (True, False)}
        gam, G = _fill_tri(f, lambda b, s: mats[_is_onsite(b, s)])
    else:
        model.backend = "XYZ"
        f = O.OracleFlow(model, 1, mesh)
        mats = {True: (A_ON, B_ON, C_ON), False: (A_OFF, B_OFF, C_OFF)}
        gam, G = _fill_diag(f, lambda b, s: mats[_is_onsite(b, s)])
    f.set_state(gam, G)
    chi = f.chi(1.0)[0]
    out = []
    for k, site in enumerate(f.sites(0)):
        on = _is_onsite(0, site)
        got = chi[k].reshape(4, 4) if tri else np.diag(chi[k])
        if on:
            got = got - np.eye(4) / (2 * math.pi)   # bubble (gamma = 0), pinned above
        wrong = ("swap_dir", "swap_exc", "exc_s") if on else ("swap_dir",)   # no exchange part off site
        refs = {r: _vertex_term(*mats[on], on, continuum, r) for r in ("paper",) + wrong}
        if not tri:
            refs = {r: np.diag(np.diag(v)) for r, v in refs.items()}
        scale = np.abs(refs["paper"]).max()
        out.append((on, np.abs(got - refs["paper"]).max() / scale,
                    min(np.abs(got - refs[r]).max() for r in wrong) / scale))
    return out


@pytest.mark.parametrize("tri", [False, True], ids=["diagonal", "tri"])
def test_chi_frequency_routing_converges_to_continuum(continuum, tri):
    """Vertex A phi(t) + B psi(min(s, u)) + C rho(max(s, u)) phi(t) on every pair, gamma = 0,
    Lambda = 1, mesh 0.01..100: chi's vertex term converges to the continuum integrals at
    second order in the mesh spacing (normwise relative error below 1.5e-2 at N = 24 and 3e-3
    at N = 48, falling by more than 2.5x per doubling), while reading t and u the other way
    round in either part, or s = w1 - w2 in the exchange part, would miss by more than 10 % --
    so the pin fixes the arguments (w1+w2, 0, w1-w2) and (w1+w2, w2-w1, 0), the exchange sign
    and its on-site restriction."""
    e24 = _routing_errors(24, continuum, tri)
    e48 = _routing_errors(48, continuum, tri)
    for (on, err24, _), (_, err48, miss48) in zip(e24, e48):
        assert err24 < 1.5e-2, (on, err24)
        assert err48 < 3e-3, (on, err48)
        assert err24 / max(err48, 1e-12) > 2.5, (on, err24, err48)
        assert miss48 > 0.1, (on, miss48)
    assert any(on for on, _, _ in e48) and not all(on for on, _, _ in e48)
