"""Analysis of a flow's susceptibility: the structure-factor maximum along the cutoff and the
flow-breakdown criterion (arXiv:2109.13317, Sec. 3 and the worked example of Sec. 6.1).

A smooth flow of the dominant structure-factor component chi_max(Lambda) down to the lowest
cutoff indicates a non-magnetic ground state; a breakdown of the smooth flow at a critical
cutoff Lambda_c -- a peak, or a kink where the flow stops being smooth -- indicates the onset
of magnetic order.  The paper reads Lambda_c off the plotted flow; `flow_breakdown` states a
criterion that can be applied without plotting:

* scanning from large to small cutoff, the first local maximum of chi_max (a peak);
* otherwise the kink: the largest relative jump of the second derivative of chi_max with
  respect to ln Lambda, if it exceeds `kink_factor` times the median jump of the flow;
* otherwise no breakdown (None).

Everything here is host-side bookkeeping over values the library measured.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from .binding import SR_EULER, Flow


@dataclass
class SusceptibilityFlow:
    lambdas: np.ndarray        # cutoffs at which chi(k) was measured (descending)
    chi_max: np.ndarray        # max over the momenta of chi(k) at each cutoff
    k_max: np.ndarray          # the momentum of the maximum at each cutoff (n, 3)


def run_susceptibility_flow(flow: Flow, lambdas: Sequence[float], kpts, method: int = SR_EULER) -> SusceptibilityFlow:
    """Step `flow` through `lambdas` (the first is the flow's current cutoff) and record the
    structure-factor maximum over `kpts` after every step."""
    kp = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
    lams: List[float] = []
    cm: List[float] = []
    km: List[np.ndarray] = []
    for lam in list(lambdas)[1:]:
        flow.step(float(lam), method)
        ck, _ = flow.measure(kp, want_ij=False)
        i = int(np.argmax(ck))
        lams.append(float(lam))
        cm.append(float(ck[i]))
        km.append(kp[i].copy())
    return SusceptibilityFlow(np.array(lams), np.array(cm), np.array(km))


def flow_breakdown(lambdas: Sequence[float], chi_max: Sequence[float], rel_peak: float = 1e-4,
                   kink_factor: float = 20.0) -> Optional[float]:
    """Critical cutoff of a flow breakdown, or None for a smooth flow (criterion in the module
    docstring).  `lambdas` must be strictly decreasing."""
    lam = np.asarray(lambdas, dtype=np.float64)
    y = np.asarray(chi_max, dtype=np.float64)
    if lam.ndim != 1 or lam.shape != y.shape or lam.size < 5:
        raise ValueError("need matching 1-d arrays of at least 5 cutoffs")
    if not np.all(np.diff(lam) < 0):
        raise ValueError("cutoffs must be strictly decreasing")
    # a peak: chi_max stops growing (relative margin rel_peak against discretisation noise)
    for i in range(1, lam.size - 1):
        if y[i] > y[i - 1] * (1 + rel_peak) and y[i] > y[i + 1] * (1 + rel_peak):
            return float(lam[i])
    # a kink: a jump of the second derivative in x = ln(Lambda)
    x = np.log(lam)
    d1 = np.diff(y) / np.diff(x)                   # between points
    d2 = np.diff(d1) / (0.5 * (x[2:] - x[:-2]))    # at interior points
    jump = np.abs(np.diff(d2)) / np.maximum(np.abs(y[2:-1]), 1e-300)
    if jump.size < 3:
        return None
    med = float(np.median(jump))
    j = int(np.argmax(jump))
    if med > 0 and jump[j] > kink_factor * med:
        return float(lam[j + 2])
    return None
