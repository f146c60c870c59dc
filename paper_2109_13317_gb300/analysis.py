"""Analysis of a flow's susceptibility: the structure-factor maximum along the cutoff and the
flow-breakdown criterion (arXiv:2109.13317, Sec. 3 and the worked example of Sec. 6.1).

A smooth flow of the dominant structure-factor component chi_max(Lambda) down to the lowest
cutoff indicates a non-magnetic ground state; a breakdown of the smooth flow at a critical
cutoff Lambda_c indicates the onset of magnetic order.  The paper reads Lambda_c off the
plotted flow; `flow_breakdown` states a criterion that needs no plot: scanning from large to
small cutoff, the first local maximum of chi_max after which chi_max falls by more than
`drop` (relative) within the next `window` cutoffs.  A breakdown that shows only as a kink --
the steep growth of chi_max ending without a decrease -- is not a peak; `log_slope` gives
d ln chi_max / d ln(1/Lambda) along the flow to look at it.

A second diagnostic for subtle breakdowns is the scaling of the on-site correlation chi_ii with
the truncation range L (Sec. 6.2): with short-ranged correlations chi_ii(Lambda) converges
quickly in L; once correlations become long-ranged (Lambda < Lambda_c in an ordered system)
the curves for different L separate.  `onsite_flow` records chi_ii along a flow and
`range_spread` compares such records across ranges.

Everything here is host-side bookkeeping over values the library measured.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from .binding import SR_ENONFINITE, SR_EULER, Flow, SrError


@dataclass
class SusceptibilityFlow:
    lambdas: np.ndarray        # cutoffs at which chi(k) was measured (descending)
    chi_max: np.ndarray        # max over the momenta of chi(k) at each cutoff
    k_max: np.ndarray          # the momentum of the maximum at each cutoff (n, 3)


def run_susceptibility_flow(flow: Flow, lambdas: Sequence[float], kpts, method: int = SR_EULER,
                            stop_on_nonfinite: bool = True) -> SusceptibilityFlow:
    """Step `flow` through `lambdas` (the first is the flow's current cutoff) and record the
    structure-factor maximum over `kpts` after every step.  After a breakdown the vertex can
    grow without bound; with `stop_on_nonfinite` a step that yields non-finite values ends
    the record there instead of raising."""
    kp = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
    lams: List[float] = []
    cm: List[float] = []
    km: List[np.ndarray] = []
    for lam in list(lambdas)[1:]:
        try:
            flow.step(float(lam), method)
        except SrError as e:
            if stop_on_nonfinite and e.status == SR_ENONFINITE:
                break
            raise
        ck, _ = flow.measure(kp, want_ij=False)
        i = int(np.argmax(ck))
        lams.append(float(lam))
        cm.append(float(ck[i]))
        km.append(kp[i].copy())
    return SusceptibilityFlow(np.array(lams), np.array(cm), np.array(km))


def flow_breakdown(lambdas: Sequence[float], chi_max: Sequence[float], drop: float = 0.02,
                   window: int = 10) -> Optional[float]:
    """Critical cutoff of a flow breakdown (a significant peak of chi_max), or None when chi_max
    has no such peak (criterion in the module docstring).  `lambdas` must be strictly
    decreasing."""
    lam = np.asarray(lambdas, dtype=np.float64)
    y = np.asarray(chi_max, dtype=np.float64)
    if lam.ndim != 1 or lam.shape != y.shape or lam.size < 3:
        raise ValueError("need matching 1-d arrays of at least 3 cutoffs")
    if not np.all(np.diff(lam) < 0):
        raise ValueError("cutoffs must be strictly decreasing")
    for i in range(1, lam.size - 1):
        if y[i] >= y[i - 1] and y[i] >= y[i + 1] and y[i + 1:i + 1 + window].min() < (1.0 - drop) * y[i]:
            return float(lam[i])
    return None


def log_slope(lambdas: Sequence[float], chi_max: Sequence[float]) -> np.ndarray:
    """d ln chi_max / d ln(1 / Lambda) between consecutive cutoffs (positive while chi_max grows
    as the cutoff decreases)."""
    lam = np.asarray(lambdas, dtype=np.float64)
    y = np.asarray(chi_max, dtype=np.float64)
    return -np.diff(np.log(y)) / np.diff(np.log(lam))


def onsite_correlation(flow: Flow) -> float:
    """The on-site spin correlation chi^{zz}_{ii} of the current state, averaged over the basis
    sites (the first site of every basis site's list is the site itself)."""
    _, chi_ij = flow.measure(None, want_ij=True)
    c = chi_ij.cpu().numpy()
    if c.shape[2] == 2:
        return float(c[:, 0, 1].mean())            # SU2: component 1 is the spin part
    if c.shape[2] == 16:
        return float(c[:, 0, 15].mean())           # TRI: mu nu = zz
    return float(c[:, 0, 3].mean())                # XYZ: zz


def onsite_flow(flow: Flow, lambdas: Sequence[float], method: int = SR_EULER, stop_on_nonfinite: bool = True):
    """chi_ii after every step through `lambdas` (the first is the current cutoff): (cutoffs,
    values).  A non-finite step ends the record (see run_susceptibility_flow)."""
    lams: List[float] = []
    vals: List[float] = []
    for lam in list(lambdas)[1:]:
        try:
            flow.step(float(lam), method)
        except SrError as e:
            if stop_on_nonfinite and e.status == SR_ENONFINITE:
                break
            raise
        lams.append(float(lam))
        vals.append(onsite_correlation(flow))
    return np.array(lams), np.array(vals)


def range_spread(records) -> tuple:
    """Relative spread (max - min) / mean of chi_ii across truncation ranges at the cutoffs all
    records share; `records` is a sequence of (cutoffs, values) on one cutoff grid.  Returns
    (cutoffs, spread)."""
    n = min(len(r[0]) for r in records)
    lam = np.asarray(records[0][0][:n])
    for r in records:
        if not np.allclose(r[0][:n], lam, rtol=0, atol=0):
            raise ValueError("records must share their cutoff grid")
    v = np.stack([np.asarray(r[1][:n]) for r in records])
    return lam, (v.max(axis=0) - v.min(axis=0)) / np.abs(v.mean(axis=0))


def fourier_components(chi_ij: np.ndarray, dr: np.ndarray, kpts) -> np.ndarray:
    """Momentum-resolved correlations of every stored spin component (Eq. frg:structurefactor
    for one component instead of the trace): out[k, c] = (1/N_b) sum_{b, j} exp(i k (r_b - r_j))
    chi^c_{b j} with chi_ij of shape (N_b, N_tot, n_c) and dr the matching (N_b, N_tot, 3)
    displacements r_b - r_j.  Complex: for a TRI model chi^{mu nu}_{ij} and chi^{mu nu}_{ji}
    differ (e.g. the antisymmetric part from DM couplings), so the mu != nu components carry an
    imaginary part; the sum of the xx, yy, zz components is the real structure factor."""
    c = np.asarray(chi_ij)
    d = np.asarray(dr, dtype=np.float64)
    kp = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
    ph = np.exp(1j * np.einsum("ka,bja->kbj", kp, d))
    return np.einsum("kbj,bjc->kc", ph, c) / c.shape[0]


def chi_displacements(flow: Flow) -> np.ndarray:
    """r_b - r_j (shape (N_b, N_tot, 3)) of the flow's correlation pairs, in the order of the
    chi_ij array that `Flow.measure` returns."""
    lat = flow.lattice
    sites = flow.chi_sites()
    pos = (sites[..., 0:1] * lat.prim[0] + sites[..., 1:2] * lat.prim[1] + sites[..., 2:3] * lat.prim[2] +
           lat.basis[sites[..., 3]])
    return lat.basis[:, None, :] - pos


def structure_factor_components(flow: Flow, kpts) -> np.ndarray:
    """`fourier_components` of the flow's current correlations: complex (n_k, n_c), component
    index as in the state layout (TRI: mu * 4 + nu)."""
    _, chi_ij = flow.measure(None, want_ij=True)
    return fourier_components(chi_ij.cpu().numpy(), chi_displacements(flow), kpts)
