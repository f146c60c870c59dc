"""Synthetic workload definitions shared by the tests, the benchmark and the oracle.

This module holds inputs only: lattice unit cells (primitive vectors, basis sites, bonds),
spin-model couplings and run configurations (frequency range, truncation range, cutoff
range).  It contains none of the flow-equation arithmetic; the CUDA path and the CPU oracle
each turn these inputs into meshes, vertex tables and flows on their own.

Unit cells and models follow the paper's resource-file format (arXiv:2109.13317, Sec. 5.3
"Definition of lattice graphs" and Sec. 5.4 "Definition of spin interactions"): a site is
(n0, n1, n2, b) = n0 a0 + n1 a1 + n2 a2 + basis[b]; a bond joins basis site `from` of one
cell to basis site `to` of the cell shifted by (da0, da1, da2); an interaction couples
S_from . M . S_to with a 3x3 matrix M.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

S3 = math.sqrt(3.0)


@dataclass
class UnitCell:
    name: str
    prim: np.ndarray            # 3 x 3, row i = a_i
    basis: np.ndarray           # nb x 3
    bonds: List[Tuple[int, int, int, int, int]]  # (from, to, da0, da1, da2)

    @property
    def n_basis(self) -> int:
        return self.basis.shape[0]


@dataclass
class Coupling:
    frm: Tuple[int, int, int, int]   # (n0, n1, n2, b)
    to: Tuple[int, int, int, int]
    M: np.ndarray                    # 3 x 3, already multiplied by the coupling constant


@dataclass
class Model:
    cell: UnitCell
    couplings: List[Coupling]
    backend: str = "SU2"             # "SU2", "XYZ" or "TRI"


def _cell(name, prim, basis, bonds) -> UnitCell:
    return UnitCell(name, np.asarray(prim, dtype=np.float64), np.asarray(basis, dtype=np.float64),
                    [tuple(int(v) for v in b) for b in bonds])


# --- unit cells (paper Sec. 5.3 listings; pyrochlore and diamond from crystal geometry) ---

def square() -> UnitCell:
    return _cell("square", [[1, 0, 0], [0, 1, 0], [0, 0, 1]], [[0, 0, 0]],
                 [(0, 0, 1, 0, 0), (0, 0, 0, 1, 0)])


def honeycomb() -> UnitCell:
    return _cell("honeycomb", [[1.5, S3 / 2, 0], [1.5, -S3 / 2, 0], [0, 0, 1]],
                 [[0, 0, 0], [1, 0, 0]],
                 [(0, 1, 0, 0, 0), (1, 0, 1, 0, 0), (1, 0, 0, 1, 0)])


def kagome() -> UnitCell:
    return _cell("kagome", [[2, 0, 0], [1, S3, 0], [0, 0, 1]],
                 [[0, 0, 0], [1, 0, 0], [0.5, S3 / 2, 0]],
                 [(0, 1, 0, 0, 0), (0, 2, 0, 0, 0), (1, 2, 0, 0, 0),
                  (1, 0, 1, 0, 0), (2, 0, 0, 1, 0), (2, 1, -1, 1, 0)])


def cubic() -> UnitCell:
    return _cell("cubic", [[1, 0, 0], [0, 1, 0], [0, 0, 1]], [[0, 0, 0]],
                 [(0, 0, 1, 0, 0), (0, 0, 0, 1, 0), (0, 0, 0, 0, 1)])


def diamond() -> UnitCell:
    """FCC primitives (conventional cube of edge 1) with a two-site basis."""
    return _cell("diamond", [[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]],
                 [[0, 0, 0], [0.25, 0.25, 0.25]],
                 [(0, 1, 0, 0, 0), (0, 1, -1, 0, 0), (0, 1, 0, -1, 0), (0, 1, 0, 0, -1)])


def pyrochlore() -> UnitCell:
    """FCC primitives with a four-site tetrahedral basis; 6 'up' and 6 'down' bonds per cell."""
    return _cell("pyrochlore", [[0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]],
                 [[0, 0, 0], [0, 0.25, 0.25], [0.25, 0, 0.25], [0.25, 0.25, 0]],
                 [(0, 1, 0, 0, 0), (0, 2, 0, 0, 0), (0, 3, 0, 0, 0),
                  (1, 2, 0, 0, 0), (1, 3, 0, 0, 0), (2, 3, 0, 0, 0),
                  (0, 1, -1, 0, 0), (0, 2, 0, -1, 0), (0, 3, 0, 0, -1),
                  (1, 2, 1, -1, 0), (1, 3, 1, 0, -1), (2, 3, 0, 1, -1)])


CELLS = {f.__name__: f for f in (square, honeycomb, kagome, cubic, diamond, pyrochlore)}

I3 = np.eye(3)


def _diag(i):
    m = np.zeros((3, 3))
    m[i, i] = 1.0
    return m


def nn_heisenberg(cell: UnitCell, J: float = 1.0) -> Model:
    """Heisenberg coupling J on every bond of the unit cell."""
    cps = [Coupling((0, 0, 0, f), (d0, d1, d2, t), J * I3) for (f, t, d0, d1, d2) in cell.bonds]
    return Model(cell, cps, "SU2")


def square_j1j2(J1: float = 1.0, J2: float = 0.5) -> Model:
    m = nn_heisenberg(square(), J1)
    if J2 != 0.0:
        m.couplings += [Coupling((0, 0, 0, 0), (1, 1, 0, 0), J2 * I3),
                        Coupling((0, 0, 0, 0), (1, -1, 0, 0), J2 * I3)]
    return m


def cubic_j1j2(J1: float = 1.0, J2: float = 0.0) -> Model:
    """Simple-cubic J1-J2 Heisenberg model of the paper's first worked example: J1 on the three
    bonds of the unit cell, J2 on the six face diagonals per cell."""
    m = nn_heisenberg(cubic(), J1)
    if J2 != 0.0:
        m.couplings += [Coupling((0, 0, 0, 0), (d0, d1, d2, 0), J2 * I3)
                        for (d0, d1, d2) in ((0, 1, -1), (0, 1, 1), (1, -1, 0), (1, 0, -1), (1, 0, 1), (1, 1, 0))]
    return m


def honeycomb_kitaev(J: float = 0.2, K: float = -1.0) -> Model:
    """Heisenberg-Kitaev model of the paper's model listing: Heisenberg J on the three bonds,
    Kitaev K as xx, yy, zz on the three bond directions."""
    c = honeycomb()
    to = [(0, 0, 0, 1), (0, -1, 0, 1), (-1, 0, 0, 1)]
    cps = [Coupling((0, 0, 0, 0), t, J * I3 + K * _diag(i)) for i, t in enumerate(to)]
    return Model(c, cps, "XYZ")


def dm_matrix(D) -> np.ndarray:
    """Coupling matrix of D . (S_from x S_to): M[a][b] = sum_c eps_{c a b} D_c."""
    D = np.asarray(D, dtype=np.float64)
    return np.array([[0.0, D[2], -D[1]], [-D[2], 0.0, D[0]], [D[1], -D[0], 0.0]])


def kagome_dm(J: float = 1.0, D: float = 0.5) -> Model:
    """Kagome Heisenberg antiferromagnet with out-of-plane Dzyaloshinskii-Moriya vectors of the
    paper's second worked example (Sec. 6.2 model listing): on each of the six directed
    nearest-neighbour bonds per cell, J S_from . S_to + D (S_from x S_to)_z, i.e. the terms xy
    and -yx with weight D.  Needs the TRI core."""
    c = kagome()
    directed = [((0, 0, 0, 1), (0, 0, 0, 0)), ((0, 0, 0, 0), (0, 0, 0, 2)),
                ((-1, 0, 0, 1), (0, 0, 0, 0)), ((0, 0, 0, 0), (0, -1, 0, 2)),
                ((0, 0, 0, 2), (0, 0, 0, 1)), ((0, -1, 0, 2), (-1, 0, 0, 1))]
    M = J * I3 + dm_matrix((0.0, 0.0, D))
    return Model(c, [Coupling(f, t, M.copy()) for f, t in directed], "TRI")


def rotated(model: Model, R: np.ndarray, backend: str = "TRI") -> Model:
    """The same model with every coupling matrix rotated in spin space, M -> R M R^T."""
    R = np.asarray(R, dtype=np.float64)
    return Model(model.cell, [Coupling(c.frm, c.to, R @ c.M @ R.T) for c in model.couplings], backend)


def honeycomb_kitaev_gamma(J: float = 0.1, K: float = -1.0, G: float = 0.5) -> Model:
    """Heisenberg-Kitaev-Gamma model on the honeycomb lattice: on a bond of type gamma (x, y, z
    for the three bond directions), J S.S + K S^g S^g + G (S^a S^b + S^b S^a) with (a, b) the other
    two components.  The symmetric off-diagonal G term needs the TRI core."""
    c = honeycomb()
    to = [(0, 0, 0, 1), (0, -1, 0, 1), (-1, 0, 0, 1)]
    cps = []
    for g, t in enumerate(to):
        a, b = [x for x in range(3) if x != g]
        M = J * I3 + K * _diag(g)
        M[a, b] += G
        M[b, a] += G
        cps.append(Coupling((0, 0, 0, 0), t, M))
    return Model(c, cps, "TRI")


def honeycomb_kitaev_linear():
    """Heisenberg-Kitaev couplings as a linear function of theta = (J, K): the unit cell, the
    coupling sites and the basis matrices B (2, n_couplings, 3, 3) with M_c = J B[0, c] +
    K B[1, c]."""
    c = honeycomb()
    to = [(0, 0, 0, 1), (0, -1, 0, 1), (-1, 0, 0, 1)]
    sites = [((0, 0, 0, 0), t) for t in to]
    B = np.zeros((2, 3, 3, 3))
    for i in range(3):
        B[0, i] = I3
        B[1, i] = _diag(i)
    return c, sites, B


def kagome_dm_linear():
    """The kagome DM model as a linear function of theta = (J, D): the unit cell, the six
    directed bonds of kagome_dm and the basis matrices B (2, 6, 3, 3) with M_c = J B[0, c] +
    D B[1, c] (Heisenberg and out-of-plane DM parts)."""
    c = kagome()
    sites = [((0, 0, 0, 1), (0, 0, 0, 0)), ((0, 0, 0, 0), (0, 0, 0, 2)),
             ((-1, 0, 0, 1), (0, 0, 0, 0)), ((0, 0, 0, 0), (0, -1, 0, 2)),
             ((0, 0, 0, 2), (0, 0, 0, 1)), ((0, -1, 0, 2), (-1, 0, 0, 1))]
    B = np.zeros((2, len(sites), 3, 3))
    for i in range(len(sites)):
        B[0, i] = I3
        B[1, i] = dm_matrix((0.0, 0.0, 1.0))
    return c, sites, B


def linear_model(cell, sites, B, theta, backend="XYZ") -> Model:
    M = np.einsum("p,pcij->cij", np.asarray(theta, dtype=np.float64), B)
    return Model(cell, [Coupling(f, t, M[k]) for k, (f, t) in enumerate(sites)], backend)


@dataclass
class FlowConfig:
    """One run configuration: model, truncation range, frequency mesh and cutoff range."""
    name: str
    model: Model
    L: int
    n_freq: int
    w_min: float
    w_max: float
    lam_max: float
    lam_min: float
    n_steps: int                 # log-spaced steps (Euler); for adaptive runs the output grid
    method: str = "euler"        # "euler" or "rk"
    rtol: float = 1e-6
    atol: float = 1e-10


def config(name: str) -> FlowConfig:
    """The workload configurations, by short name."""
    if name == "square_j1_L3":
        return FlowConfig(name, nn_heisenberg(square(), 1.0), 3, 16, 0.005, 50.0, 50.0, 0.05, 100)
    if name == "square_j1j2_L7":
        return FlowConfig(name, square_j1j2(1.0, 0.5), 7, 48, 0.001, 100.0, 100.0, 0.01, 100,
                          method="rk", rtol=1e-6, atol=1e-10)
    if name == "pyrochlore_L6":
        return FlowConfig(name, nn_heisenberg(pyrochlore(), 1.0), 6, 64, 0.001, 100.0, 100.0, 0.01, 400)
    if name == "cubic_j1j2_L7":
        # the paper's first worked example (J2 = 0); cutoff ratio 0.98 per step from 50 to 0.01
        return FlowConfig(name, cubic_j1j2(1.0, 0.0), 7, 64, 0.005, 50.0, 50.0, 0.01, 422)
    if name == "honeycomb_hk_L5":
        return FlowConfig(name, honeycomb_kitaev(0.2, -1.0), 5, 32, 0.005, 50.0, 50.0, 0.05, 200)
    if name == "kagome_dm_L7":
        # the paper's second worked example (TRI core) at D = 0.5, range 7, with 32 of its 64
        # frequencies; 200 log steps from 50 to 0.01
        return FlowConfig(name, kagome_dm(1.0, 0.5), 7, 32, 0.005, 50.0, 50.0, 0.01, 200)
    raise KeyError(name)


def batched_instances(seed: int = 0, n: int = 64):
    """The batched coupling sweep: square J1-J2 (J2/J1 ~ U[0,1], range 5..9) and kagome J1
    (range 4..8), 32..64 frequencies each.  Seeded; returns a list of FlowConfig."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nw = int(rng.integers(32, 65))
        if i < (3 * n) // 4:
            j2 = float(rng.uniform(0.0, 1.0))
            L = int(rng.integers(5, 10))
            out.append(FlowConfig(f"sq{i}", square_j1j2(1.0, j2), L, nw, 0.005, 50.0, 50.0, 0.05, 100))
        else:
            L = int(rng.integers(4, 9))
            out.append(FlowConfig(f"kg{i}", nn_heisenberg(kagome(), 1.0), L, nw, 0.005, 50.0, 50.0, 0.05, 100))
    return out


def lambda_geometric(lam_max: float, lam_min: float, step: float) -> np.ndarray:
    """The paper's exponential cutoff discretisation with a fixed ratio: lam_max step^n for
    n = 0, 1, ... while the value is >= lam_min."""
    n = int(math.floor(math.log(lam_min / lam_max) / math.log(step) + 1e-9))
    return lam_max * step ** np.arange(n + 1)


def lambda_list(lam_max: float, lam_min: float, n_steps: int) -> np.ndarray:
    """n_steps log steps from lam_max to lam_min: n_steps + 1 points, endpoints exact."""
    x = lam_max * (lam_min / lam_max) ** (np.arange(n_steps + 1) / n_steps)
    x[0], x[-1] = lam_max, lam_min
    return x


def flatten_model(model: Model):
    """Plain arrays of a model, in the order both implementations take them."""
    cell = model.cell
    bonds = np.asarray(cell.bonds, dtype=np.int32).reshape(-1, 5)
    frm = np.asarray([c.frm for c in model.couplings], dtype=np.int32).reshape(-1, 4)
    to = np.asarray([c.to for c in model.couplings], dtype=np.int32).reshape(-1, 4)
    M = np.asarray([c.M for c in model.couplings], dtype=np.float64).reshape(-1, 3, 3)
    return (np.ascontiguousarray(cell.prim), np.ascontiguousarray(cell.basis), bonds, frm, to, M)


def synthetic_state(of, model, seed: int = 0, amp: float = 0.3):
    """A smooth frequency-dependent vertex that respects every symmetry of an SU(2) lattice
    model: a function of the pair's Euclidean distance only, antisymmetric under s <-> u for
    the density part and symmetric for the spin part, plus the bare coupling J/4.  `of` is any
    object with the oracle flow's layout accessors (get_state, block, sites, position,
    coupling, basis, mesh, N, nb); this function only fills values, it evaluates no flow
    equation.  Returns (gamma, Gamma) in that layout."""
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
