"""ctypes wrapper of the plain C FP64 pf-FRG oracle (``pffrg_oracle.c``).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU-baseline leg of
the benchmark.  Builds the C file with gcc into ``oracle/_build`` on first use.

The oracle keeps the vertex in translation-only storage: for every basis site b of the home
cell and every site k within bond distance L of b, the spin-diagonal basis functions
Gamma^{cc}(s, t, u), c = 0..3, on the octant s >= u (layout [b][k][c][pair(s,u)][t]);
`OracleFlowTRI` keeps all 16 Gamma^{mu nu} as complex numbers ([b][k][mu nu][pair][t]).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pffrg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpffrg_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -fopenmp); returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp = C.c_void_p
        lib.or_lattice_new.restype = vp
        lib.or_lattice_new.argtypes = [C.c_int, _dp, _dp, C.c_int, _ip, C.c_int, _ip, _ip, _dp, C.c_int]
        lib.or_lattice_free.argtypes = [vp]
        lib.or_lattice_nsites.restype = C.c_int
        lib.or_lattice_nsites.argtypes = [vp, C.c_int]
        lib.or_lattice_offdiag.restype = C.c_int
        lib.or_lattice_offdiag.argtypes = [vp]
        lib.or_lattice_site.argtypes = [vp, C.c_int, C.c_int, _ip]
        lib.or_lattice_coupling.argtypes = [vp, C.c_int, C.c_int, _dp]
        lib.or_lattice_find.restype = C.c_int
        lib.or_lattice_find.argtypes = [vp, C.c_int, _ip, C.c_int]
        lib.or_state_new.restype = vp
        lib.or_state_new.argtypes = [vp, C.c_int, _dp]
        lib.or_state_free.argtypes = [vp]
        lib.or_state_size.restype = C.c_size_t
        lib.or_state_size.argtypes = [vp]
        lib.or_state_offset.restype = C.c_size_t
        lib.or_state_offset.argtypes = [vp, C.c_int]
        lib.or_state_get.argtypes = [vp, _dp, _dp]
        lib.or_state_set.argtypes = [vp, _dp, _dp]
        lib.or_state_init.argtypes = [vp]
        lib.or_vertex_lookup.argtypes = [vp, C.c_int, _ip, C.c_int, C.c_double, C.c_double, C.c_double, _dp]
        lib.or_sigma_rhs_point.restype = C.c_double
        lib.or_sigma_rhs_point.argtypes = [vp, C.c_int, C.c_double, C.c_double]
        lib.or_rhs.argtypes = [vp, C.c_double, _dp, _dp]
        lib.or_rhs_entries.argtypes = [vp, C.c_double, C.c_int, _ip, _dp]
        lib.or_rhs_prepare.argtypes = [vp, C.c_double, _dp]
        lib.or_rhs_point.argtypes = [vp, C.c_int, _ip, C.c_int, C.c_double, C.c_double, C.c_double, _dp]
        lib.or_channel_nodes.restype = C.c_int
        lib.or_channel_nodes.argtypes = [vp, C.c_int, C.c_double, _dp, _dp]
        lib.or_euler_step.argtypes = [vp, C.c_double, C.c_double]
        lib.or_dp54_step.restype = C.c_double
        lib.or_dp54_step.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double]
        lib.or_chi.argtypes = [vp, C.c_double, _dp]
        lib.or_dp54_tableau.argtypes = [_dp, _dp, _dp, _dp]
        lib.or_mesh_exponential.argtypes = [C.c_int, C.c_double, C.c_double, _dp]
        lib.or_cutoff_exponential.restype = C.c_int
        lib.or_cutoff_exponential.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _dp]
        lib.or_spin_tables.restype = C.c_int
        lib.or_spin_tables.argtypes = [_dp, _dp, _dp, _dp, _dp]
        lib.or_num_threads.restype = C.c_int
        lib.or_set_num_threads.argtypes = [C.c_int]
        lib.or_tri_spin_tables.argtypes = [_dp, _dp, _dp, _dp, _dp]
        lib.or_tri_state_new.restype = vp
        lib.or_tri_state_new.argtypes = [vp, C.c_int, _dp]
        lib.or_tri_state_free.argtypes = [vp]
        lib.or_tri_state_size.restype = C.c_size_t
        lib.or_tri_state_size.argtypes = [vp]
        lib.or_tri_state_offset.restype = C.c_size_t
        lib.or_tri_state_offset.argtypes = [vp, C.c_int]
        lib.or_tri_state_get.argtypes = [vp, _dp, _dp]
        lib.or_tri_state_set.argtypes = [vp, _dp, _dp]
        lib.or_tri_state_init.argtypes = [vp]
        lib.or_tri_lookup.argtypes = [vp, C.c_int, _ip, C.c_int, C.c_double, C.c_double, C.c_double, _dp]
        lib.or_sigma_basis_spread.restype = C.c_double
        lib.or_sigma_basis_spread.argtypes = []
        lib.or_sigma_basis_spread_reset.restype = None
        lib.or_sigma_basis_spread_reset.argtypes = []
        lib.or_tri_sigma_imag.restype = C.c_double
        lib.or_tri_rhs.argtypes = [vp, C.c_double, _dp, _dp]
        lib.or_tri_rhs_prepare.argtypes = [vp, C.c_double, _dp]
        lib.or_tri_rhs_point.argtypes = [vp, C.c_int, _ip, C.c_int, C.c_double, C.c_double, C.c_double, _dp]
        lib.or_tri_euler_step.argtypes = [vp, C.c_double, C.c_double]
        lib.or_tri_rhs_entries.argtypes = [vp, C.c_int, _ip, _dp]
        lib.or_tri_dp54_step.restype = C.c_double
        lib.or_tri_dp54_step.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double]
        lib.or_tri_chi.argtypes = [vp, C.c_double, _dp]
        _lib = lib
        return lib


def mesh_exponential(n: int, wmin: float, wmax: float) -> np.ndarray:
    out = np.zeros(n)
    load().or_mesh_exponential(n, wmin, wmax, out)
    return out


def cutoff_exponential(lmin: float, lmax: float, b: float) -> np.ndarray:
    lib = load()
    cap = 100000
    out = np.zeros(cap)
    n = lib.or_cutoff_exponential(lmin, lmax, b, cap, out)
    return out[:n].copy()


def spin_tables():
    """Coefficient tables generated by the oracle's literal Pauli contraction.
    Returns (coef[5,4,4,4], hartree[4], fock[4], chi_dir[4,4], chi_exc[4,4], closed)."""
    coef = np.zeros(5 * 64)
    h = np.zeros(4)
    f = np.zeros(4)
    cd = np.zeros(16)
    cx = np.zeros(16)
    closed = load().or_spin_tables(coef, h, f, cd, cx)
    return coef.reshape(5, 4, 4, 4), h, f, cd.reshape(4, 4), cx.reshape(4, 4), bool(closed)


def tri_spin_tables():
    """Complex coefficient tables of the TRI core from the oracle's literal Pauli contraction:
    (coef[5,16,16,16], hartree[16], fock[16], chi_dir[16,16], chi_exc[16,16]); component
    index mu * 4 + nu."""
    coef = np.zeros(5 * 4096 * 2)
    h, f = np.zeros(32), np.zeros(32)
    cd, cx = np.zeros(512), np.zeros(512)
    load().or_tri_spin_tables(coef, h, f, cd, cx)
    z = lambda a: a[0::2] + 1j * a[1::2]  # noqa: E731
    return (z(coef).reshape(5, 16, 16, 16), z(h), z(f), z(cd).reshape(16, 16), z(cx).reshape(16, 16))


def dp54_tableau():
    """(c[7], a[7,6], b5[7], b4[7]) of the oracle's Dormand-Prince 5(4) step."""
    c, a, b5, b4 = np.zeros(7), np.zeros(42), np.zeros(7), np.zeros(7)
    load().or_dp54_tableau(c, a, b5, b4)
    return c, a.reshape(7, 6), b5, b4


CH_S, CH_T, CH_U = 0, 1, 2


class OracleFlow:
    """Oracle lattice + vertex state for one model, truncation range and frequency mesh."""

    def __init__(self, model, L: int, mesh: np.ndarray):
        from workloads import flatten_model
        lib = load()
        self.lib = lib
        prim, basis, bonds, frm, to, M = flatten_model(model)
        self.nb = basis.shape[0]
        self.la = lib.or_lattice_new(self.nb, np.ascontiguousarray(prim.reshape(-1)),
                                     np.ascontiguousarray(basis.reshape(-1)), bonds.shape[0],
                                     np.ascontiguousarray(bonds.reshape(-1)), frm.shape[0],
                                     np.ascontiguousarray(frm.reshape(-1)), np.ascontiguousarray(to.reshape(-1)),
                                     np.ascontiguousarray(M.reshape(-1)), L)
        if not self.la:
            raise ValueError("oracle lattice construction failed")
        if lib.or_lattice_offdiag(self.la):
            raise ValueError("oracle stores spin-diagonal vertices only")
        self.mesh = np.ascontiguousarray(mesh, dtype=np.float64)
        self.N = len(self.mesh)
        self.st = lib.or_state_new(self.la, self.N, self.mesh)
        if not self.st:
            raise ValueError("oracle state construction failed")
        self.size = int(lib.or_state_size(self.st))
        self.nsite = [lib.or_lattice_nsites(self.la, b) for b in range(self.nb)]
        self.prim = prim
        self.basis = basis
        self.npair = self.N * (self.N + 1) // 2
        lib.or_state_init(self.st)

    def __del__(self):
        try:
            self.lib.or_state_free(self.st)
            self.lib.or_lattice_free(self.la)
        except Exception:
            pass

    # --- lattice ---
    def sites(self, b: int) -> np.ndarray:
        """(nsite_b, 4) array of (n0, n1, n2, b') for the sites within range of basis b."""
        out = np.zeros((self.nsite[b], 4), dtype=np.int32)
        tmp = np.zeros(4, dtype=np.int32)
        for k in range(self.nsite[b]):
            self.lib.or_lattice_site(self.la, b, k, tmp)
            out[k] = tmp
        return out

    def find(self, b1: int, d, b2: int) -> int:
        return self.lib.or_lattice_find(self.la, b1, np.asarray(d, dtype=np.int32), b2)

    def position(self, site) -> np.ndarray:
        n0, n1, n2, b = site
        return n0 * self.prim[0] + n1 * self.prim[1] + n2 * self.prim[2] + self.basis[b]

    def coupling(self, b: int, k: int) -> np.ndarray:
        out = np.zeros(9)
        self.lib.or_lattice_coupling(self.la, b, k, out)
        return out.reshape(3, 3)

    # --- state ---
    def init(self):
        self.lib.or_state_init(self.st)

    def get_state(self):
        gam = np.zeros(self.N)
        G = np.zeros(self.size)
        self.lib.or_state_get(self.st, gam, G)
        return gam, G

    def set_state(self, gam, G):
        self.lib.or_state_set(self.st, np.ascontiguousarray(gam, dtype=np.float64),
                              np.ascontiguousarray(G, dtype=np.float64))

    def block(self, G: np.ndarray, b: int) -> np.ndarray:
        """View of basis b's block as [k][c][pair][t]."""
        off = int(self.lib.or_state_offset(self.st, b))
        n = self.nsite[b] * 4 * self.npair * self.N
        return G[off:off + n].reshape(self.nsite[b], 4, self.npair, self.N)

    def lookup(self, b1, d, b2, s, t, u) -> np.ndarray:
        out = np.zeros(4)
        self.lib.or_vertex_lookup(self.st, b1, np.asarray(d, dtype=np.int32), b2, s, t, u, out)
        return out

    # --- flow ---
    def rhs(self, lam: float):
        dg = np.zeros(self.N)
        dG = np.zeros(self.size)
        self.lib.or_rhs(self.st, lam, dg, dG)
        return dg, dG

    def rhs_entries(self, lam: float, ent: np.ndarray) -> np.ndarray:
        ent = np.ascontiguousarray(ent, dtype=np.int32).reshape(-1, 5)
        out = np.zeros((ent.shape[0], 4))
        self.lib.or_rhs_entries(self.st, lam, ent.shape[0], ent.reshape(-1), out)
        return out

    def prepare(self, lam: float) -> np.ndarray:
        dg = np.zeros(self.N)
        self.lib.or_rhs_prepare(self.st, lam, dg)
        return dg

    def rhs_point(self, b1, d, b2, s, t, u) -> np.ndarray:
        out = np.zeros(4)
        self.lib.or_rhs_point(self.st, b1, np.asarray(d, dtype=np.int32), b2, s, t, u, out)
        return out

    def sigma_rhs_point(self, w: float, lam: float, b: int = 0) -> float:
        return self.lib.or_sigma_rhs_point(self.st, b, w, lam)

    def channel_nodes(self, ch: int, v: float):
        cap = 2 * self.N + 16
        x = np.zeros(cap)
        W = np.zeros(cap)
        n = self.lib.or_channel_nodes(self.st, ch, v, x, W)
        return x[:n].copy(), W[:n].copy()

    def euler(self, lam: float, lam_next: float):
        self.lib.or_euler_step(self.st, lam, lam_next)

    def dp54(self, lam: float, lam_next: float, rtol: float, atol: float) -> float:
        return self.lib.or_dp54_step(self.st, lam, lam_next, rtol, atol)

    def chi(self, lam: float):
        """Per basis b: array (nsite_b, 4) of chi^{mu mu}_{b k}, mu = 0 (density), x, y, z."""
        tot = sum(self.nsite)
        out = np.zeros(tot * 4)
        self.lib.or_chi(self.st, lam, out)
        out = out.reshape(tot, 4)
        res, o = [], 0
        for b in range(self.nb):
            res.append(out[o:o + self.nsite[b]])
            o += self.nsite[b]
        return res

    def chi_k(self, lam: float, kpts: np.ndarray, chi=None) -> np.ndarray:
        """chi(k) = (1/N_b) sum_b sum_j cos(k (r_b - r_j)) sum_{mu=x,y,z} chi^{mu mu}_{bj}."""
        if chi is None:
            chi = self.chi(lam)
        kpts = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
        acc = np.zeros(kpts.shape[0])
        for b in range(self.nb):
            sites = self.sites(b)
            rb = self.basis[b]
            for k, s in enumerate(sites):
                dr = rb - self.position(s)
                acc += np.cos(kpts @ dr) * chi[b][k, 1:].sum()
        return acc / self.nb

    @staticmethod
    def sigma_basis_spread(reset: bool = False) -> float:
        """Largest relative spread of the self-energy flow across basis sites seen so far
        (the oracle sets dgamma to NaN when it exceeds 1e-10: inequivalent sites)."""
        lib = load()
        v = lib.or_sigma_basis_spread()
        if reset:
            lib.or_sigma_basis_spread_reset()
        return v

    @staticmethod
    def set_threads(n: int):
        load().or_set_num_threads(n)

    @staticmethod
    def threads() -> int:
        return load().or_num_threads()


class OracleFlowTRI(OracleFlow):
    """The oracle's general time-reversal-invariant core: all 16 basis functions
    Gamma^{mu nu} (component mu * 4 + nu) stored as complex numbers, layout
    [b][k][mu nu][pair(s,u)][t].  Accepts couplings with off-diagonal entries."""

    def __init__(self, model, L: int, mesh: np.ndarray):
        from workloads import flatten_model
        lib = load()
        self.lib = lib
        prim, basis, bonds, frm, to, M = flatten_model(model)
        self.nb = basis.shape[0]
        self.la = lib.or_lattice_new(self.nb, np.ascontiguousarray(prim.reshape(-1)),
                                     np.ascontiguousarray(basis.reshape(-1)), bonds.shape[0],
                                     np.ascontiguousarray(bonds.reshape(-1)), frm.shape[0],
                                     np.ascontiguousarray(frm.reshape(-1)), np.ascontiguousarray(to.reshape(-1)),
                                     np.ascontiguousarray(M.reshape(-1)), L)
        if not self.la:
            raise ValueError("oracle lattice construction failed")
        self.mesh = np.ascontiguousarray(mesh, dtype=np.float64)
        self.N = len(self.mesh)
        self.st = lib.or_tri_state_new(self.la, self.N, self.mesh)
        if not self.st:
            raise ValueError("oracle state construction failed")
        self.size = int(lib.or_tri_state_size(self.st))
        self.nsite = [lib.or_lattice_nsites(self.la, b) for b in range(self.nb)]
        self.prim = prim
        self.basis = basis
        self.npair = self.N * (self.N + 1) // 2
        lib.or_tri_state_init(self.st)

    def __del__(self):
        try:
            self.lib.or_tri_state_free(self.st)
            self.lib.or_lattice_free(self.la)
        except Exception:
            pass

    def init(self):
        self.lib.or_tri_state_init(self.st)

    def get_state(self):
        gam = np.zeros(self.N)
        G = np.zeros(2 * self.size)
        self.lib.or_tri_state_get(self.st, gam, G)
        return gam, G[0::2] + 1j * G[1::2]

    def set_state(self, gam, G):
        G = np.asarray(G, dtype=np.complex128)
        buf = np.empty(2 * self.size)
        buf[0::2] = G.real
        buf[1::2] = G.imag
        self.lib.or_tri_state_set(self.st, np.ascontiguousarray(gam, dtype=np.float64), buf)

    def block(self, G: np.ndarray, b: int) -> np.ndarray:
        """View of basis b's block as [k][mu nu][pair][t]."""
        off = int(self.lib.or_tri_state_offset(self.st, b))
        n = self.nsite[b] * 16 * self.npair * self.N
        return G[off:off + n].reshape(self.nsite[b], 16, self.npair, self.N)

    def lookup(self, b1, d, b2, s, t, u) -> np.ndarray:
        out = np.zeros(32)
        self.lib.or_tri_lookup(self.st, b1, np.asarray(d, dtype=np.int32), b2, s, t, u, out)
        return out[0::2] + 1j * out[1::2]

    def rhs(self, lam: float):
        dg = np.zeros(self.N)
        dG = np.zeros(2 * self.size)
        self.lib.or_tri_rhs(self.st, lam, dg, dG)
        return dg, dG[0::2] + 1j * dG[1::2]

    def rhs_entries(self, lam: float, ent: np.ndarray) -> np.ndarray:
        """All 16 functions of selected (b, k, si, ti, ui) entries: complex (n, 16)."""
        self.prepare(lam)
        ent = np.ascontiguousarray(ent, dtype=np.int32).reshape(-1, 5)
        out = np.zeros(ent.shape[0] * 32)
        self.lib.or_tri_rhs_entries(self.st, ent.shape[0], ent.reshape(-1), out)
        out = out.reshape(-1, 32)
        return out[:, 0::2] + 1j * out[:, 1::2]

    def prepare(self, lam: float) -> np.ndarray:
        dg = np.zeros(self.N)
        self.lib.or_tri_rhs_prepare(self.st, lam, dg)
        return dg

    def rhs_point(self, b1, d, b2, s, t, u) -> np.ndarray:
        out = np.zeros(32)
        self.lib.or_tri_rhs_point(self.st, b1, np.asarray(d, dtype=np.int32), b2, s, t, u, out)
        return out[0::2] + 1j * out[1::2]

    @staticmethod
    def sigma_imag() -> float:
        """Largest |Im H| of the self-energy flow seen so far (zero for states of the right
        real / imaginary classes)."""
        return load().or_tri_sigma_imag()

    def sigma_rhs_point(self, w, lam, b=0):  # pragma: no cover - not provided by the TRI core
        raise NotImplementedError

    def euler(self, lam: float, lam_next: float):
        self.lib.or_tri_euler_step(self.st, lam, lam_next)

    def dp54(self, lam: float, lam_next: float, rtol: float, atol: float) -> float:
        return self.lib.or_tri_dp54_step(self.st, lam, lam_next, rtol, atol)

    def chi(self, lam: float):
        """Per basis b: complex array (nsite_b, 16) of chi^{mu nu}_{b k}."""
        tot = sum(self.nsite)
        out = np.zeros(tot * 32)
        self.lib.or_tri_chi(self.st, lam, out)
        out = (out[0::2] + 1j * out[1::2]).reshape(tot, 16)
        res, o = [], 0
        for b in range(self.nb):
            res.append(out[o:o + self.nsite[b]])
            o += self.nsite[b]
        return res

    def chi_k(self, lam: float, kpts: np.ndarray, chi=None) -> np.ndarray:
        """chi(k) with the spin-diagonal components xx, yy, zz (indices 5, 10, 15)."""
        if chi is None:
            chi = self.chi(lam)
        kpts = np.asarray(kpts, dtype=np.float64).reshape(-1, 3)
        acc = np.zeros(kpts.shape[0])
        for b in range(self.nb):
            sites = self.sites(b)
            rb = self.basis[b]
            for k, s in enumerate(sites):
                dr = rb - self.position(s)
                acc += np.cos(kpts @ dr) * chi[b][k, [5, 10, 15]].real.sum()
        return acc / self.nb
