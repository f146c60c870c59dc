"""Shared test helpers: oracle <-> library layout mapping and synthetic symmetric states.

Inputs for the CUDA path always come from the oracle or from analytic formulas written
here; nothing computed by the CUDA path is fed back to the oracle.
"""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import oracle as O


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


def synthetic_state(of: "O.OracleFlow", model, seed: int = 0, amp: float = 0.3):
    """A smooth frequency-dependent vertex that respects every symmetry of an SU(2) lattice
    model: a function of the pair's Euclidean distance only, antisymmetric under s <-> u for
    the density part and symmetric for the spin part, plus the bare coupling J/4.  Returns
    (gamma, Gamma) in the oracle layout."""
    rng = np.random.default_rng(seed)
    coef = rng.normal(size=(32, 4))
    gam, G = of.get_state()
    N = of.N
    w = of.mesh
    si = np.array([s for s in range(N) for u in range(s + 1)])
    ui = np.array([u for s in range(N) for u in range(s + 1)])
    S, U = w[si][:, None], w[ui][:, None]
    T = w[None, :]
    for b in range(of.nb):
        blk = of.block(G, b)
        sites = of.sites(b)
        rb = of.basis[b]
        for k, s in enumerate(sites):
            dist = float(np.linalg.norm(of.position(s) - rb))
            key = int(round(dist * 1000)) % 32
            a0, a1, a2, a3 = coef[key]
            J = of.coupling(b, k)
            damp = np.exp(-0.3 * dist)
            blk[k, 0] = amp * damp * a0 * (S - U) / (1.0 + S + U + T)
            for c in (1, 2, 3):
                blk[k, c] = J[c - 1, c - 1] / 4.0 + amp * damp * (a1 / (1.0 + 0.5 * (S + U) + T) + a2 * np.exp(-(S + U) / (1.0 + T)) * 0.2)
    gam = 0.2 * np.tanh(w) + 0.05 * w / (1 + w)
    return gam, G


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
