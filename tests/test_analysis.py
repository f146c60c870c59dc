"""Host-side flow-breakdown criterion on synthetic susceptibility flows (no GPU)."""
import numpy as np
import pytest

from paper_2109_13317_gb300.analysis import flow_breakdown

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


def test_kink_is_detected():
    lc = 0.3
    # growing flow whose slope changes abruptly at lc but keeps growing (no peak)
    chi = np.where(LAMS > lc, 1.0 / (LAMS + 0.1), 1.0 / (lc + 0.1) + 0.2 * (lc - LAMS))
    got = flow_breakdown(LAMS, chi)
    assert got is not None and abs(np.log(got / lc)) < 0.05


def test_noise_below_the_margin_is_not_a_peak():
    chi = 1.0 / (LAMS + 0.2)
    chi = chi * (1 + 1e-6 * np.cos(np.arange(LAMS.size)))
    assert flow_breakdown(LAMS, chi) is None


def test_bad_input():
    with pytest.raises(ValueError):
        flow_breakdown(LAMS[::-1], 1.0 / LAMS[::-1])
    with pytest.raises(ValueError):
        flow_breakdown(LAMS[:3], LAMS[:3])
