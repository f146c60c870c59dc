"""Shared test helpers: oracle <-> library layout mapping and synthetic symmetric states.

Inputs for the CUDA path always come from the oracle or from analytic formulas written
here; nothing computed by the CUDA path is fed back to the oracle.
"""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import oracle as O
from workloads import synthetic_state  # noqa: F401  (input generator, re-exported for the tests)


def gpu_comp_map(n_comp: int):
    """Oracle component (0 = density, 1..3 = x, y, z) of each library component."""
    return [0, 3] if n_comp == 2 else [0, 1, 2, 3]


def oracle_to_gpu(of: "O.OracleFlow", lat, arr_oracle: np.ndarray, n_comp: int) -> np.ndarray:
    """Map an oracle Gamma array (layout [b][k][c][pair][t]) onto the library layout
    [pair][t][c][r] through the library's representative sites (pairs (ref, rep_r))."""
    reps = lat.representatives()
    blk = of.block(arr_oracle, 0)
    cm = gpu_comp_map(n_comp)
    out = np.zeros((of.npair, of.N, n_comp, lat.N_s))
    for r, rep in enumerate(reps):
        k = of.find(0, rep[:3], int(rep[3]))
        assert k >= 0, "representative outside the oracle's range"
        for c, oc in enumerate(cm):
            out[:, :, c, r] = blk[k, oc]
    return out


def evolved_oracle(model, L, mesh, lams):
    of = O.OracleFlow(model, L, mesh)
    for a, b in zip(lams[:-1], lams[1:]):
        of.euler(a, b)
    return of


IMAG_CLASS = np.array([(c // 4 == 0) != (c % 4 == 0) for c in range(16)])


def tri_real(arr: np.ndarray, axis: int) -> np.ndarray:
    """Library storage of complex TRI values along the component axis: the real part of the
    real-class functions, the imaginary part of the six imaginary-class ones."""
    sh = [1] * arr.ndim
    sh[axis] = 16
    m = IMAG_CLASS.reshape(sh)
    return np.where(m, arr.imag, arr.real)


def tri_oracle_to_gpu(of: "O.OracleFlowTRI", lat, arr_oracle: np.ndarray) -> np.ndarray:
    """Map an oracle TRI Gamma array (complex, layout [b][k][mu nu][pair][t]) onto the library
    layout [pair][t][mu nu][r] (real storage) through the representative sites."""
    reps = lat.representatives()
    blk = of.block(arr_oracle, 0)
    out = np.zeros((of.npair, of.N, 16, lat.N_s))
    for r, rep in enumerate(reps):
        k = of.find(0, rep[:3], int(rep[3]))
        assert k >= 0, "representative outside the oracle's range"
        out[:, :, :, r] = np.transpose(tri_real(blk[k], 0), (1, 2, 0))
    return out
