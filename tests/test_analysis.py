"""Host-side flow-breakdown criterion on synthetic susceptibility flows (no GPU)."""
import numpy as np
import pytest

from paper_2109_13317_gb300.analysis import flow_breakdown, log_slope

LAMS = 50.0 * 0.98 ** np.arange(1, 422)


def test_smooth_flow_has_no_breakdown():
    # a smooth, monotonically growing flow (Curie-like with a finite low-cutoff limit)
    chi = 1.0 / (LAMS + 0.2)
    assert flow_breakdown(LAMS, chi) is None


def test_peak_is_detected_at_its_cutoff():
    lc = 0.72
    chi = np.where(LAMS > lc, 1.0 / (LAMS - 0.6), 1.0 / (lc - 0.6) - 3.0 * (lc - LAMS))
    got = flow_breakdown(LAMS, chi)
    assert got is not None
    # the flow peaks on the first grid point at or below lc
    assert abs(got - LAMS[LAMS <= lc][0]) < 1e-12


def test_kink_without_decrease_is_not_a_peak():
    lc = 0.3
    # growing flow whose slope changes abruptly at lc but keeps growing: no peak
    chi = np.where(LAMS > lc, 1.0 / (LAMS + 0.1), 1.0 / (lc + 0.1) + 0.2 * (lc - LAMS))
    assert flow_breakdown(LAMS, chi) is None
    s = log_slope(LAMS, chi)
    assert s.shape == (LAMS.size - 1,)
    above, below = s[LAMS[1:] > 1.2 * lc], s[LAMS[1:] < 0.8 * lc]
    assert above.min() > 2 * below.max() > 0


def test_log_slope_of_a_power_law():
    chi = LAMS ** -1.5
    np.testing.assert_allclose(log_slope(LAMS, chi), 1.5, rtol=1e-12)


def test_wiggles_below_the_drop_margin_are_not_a_peak():
    chi = 1.0 / (LAMS + 0.2)
    chi = chi * (1 + 5e-3 * np.cos(np.arange(LAMS.size)))
    assert flow_breakdown(LAMS, chi) is None


def test_bad_input():
    with pytest.raises(ValueError):
        flow_breakdown(LAMS[::-1], 1.0 / LAMS[::-1])
    with pytest.raises(ValueError):
        flow_breakdown(LAMS[:2], LAMS[:2])


def test_range_spread():
    from paper_2109_13317_gb300.analysis import range_spread
    lam = LAMS[:5]
    recs = [(lam, np.array([1.0, 2.0, 3.0, 4.0, 5.0])), (lam, np.array([1.0, 2.0, 3.3, 4.0, 5.0])),
            (lam[:4], np.array([1.0, 2.0, 2.7, 4.4]))]
    l2, sp = range_spread(recs)
    assert l2.shape == (4,)
    np.testing.assert_allclose(sp, [0.0, 0.0, 0.6 / 3.0, 0.4 / (12.4 / 3)])
    with pytest.raises(ValueError):
        range_spread([(lam, lam), (lam * 1.01, lam)])


def test_fourier_components_against_oracle_structure_factor():
    """The host Fourier sum of the oracle's TRI correlations: the xx + yy + zz components give
    the oracle's structure factor (real), and chi^{xy}(k) = conj(chi^{yx}(k)) (chi^{mu nu}_{ij} =
    chi^{nu mu}_{ji})."""
    import workloads as W
    from oracle import oracle as O
    from paper_2109_13317_gb300.analysis import fourier_components
    mesh = O.mesh_exponential(6, 0.05, 10.0)
    of = O.OracleFlowTRI(W.kagome_dm(1.0, 0.5), 2, mesh)
    of.euler(5.0, 3.0)
    chi = of.chi(2.0)
    nb = of.nb
    nt = len(chi[0])
    c = np.zeros((nb, nt, 16), complex)
    dr = np.zeros((nb, nt, 3))
    for b in range(nb):
        c[b] = chi[b]
        for k, s in enumerate(of.sites(b)):
            dr[b, k] = of.basis[b] - of.position(s)
    kp = np.array([[0.0, 0.0, 0.0], [1.1, -0.3, 0.0], [np.pi, 0.7, 0.0]])
    F = fourier_components(c, dr, kp)
    np.testing.assert_allclose((F[:, 5] + F[:, 10] + F[:, 15]).real, of.chi_k(2.0, kp, chi), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose((F[:, 5] + F[:, 10] + F[:, 15]).imag, 0.0, atol=1e-14)
    np.testing.assert_allclose(F[:, 6], np.conj(F[:, 9]), rtol=1e-12, atol=1e-15)
    # the DM couplings leave an antisymmetric xy part in real space (its Fourier sum cancels
    # here: site inversion maps the up onto the down triangles with the same DM vectors)
    assert np.abs(c[..., 6] - c[..., 9]).max() > 1e-6
