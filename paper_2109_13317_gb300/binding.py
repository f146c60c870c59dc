"""ctypes binding of the C ABI in include/sr.h (argument marshalling only).

Device buffers are PyTorch CUDA tensors (memory and streams only); every step of the flow
runs in the library's kernels.  Names follow the C entry points: ``Lattice`` wraps
``sr_lattice_create`` / ``sr_lattice_info`` / ``sr_lattice_map_pair``; ``Flow`` wraps
``sr_flow_init``, ``sr_flow_rhs``, ``sr_flow_step``, ``sr_measure_susceptibility`` and the
state accessors.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

SR_SU2, SR_XYZ, SR_TRI = 0, 1, 2
SR_FP64, SR_FP32_MIXED = 0, 1
SR_EULER, SR_RK_ADAPTIVE, SR_RK_FIXED = 0, 1, 2
SR_OK, SR_EINVAL, SR_ENOMEM, SR_ECUDA, SR_ESYMMETRY, SR_ENONFINITE, SR_ETIMEOUT, SR_EUNSUPPORTED = range(8)
_STATUS = {0: "SR_OK", 1: "SR_EINVAL", 2: "SR_ENOMEM", 3: "SR_ECUDA", 4: "SR_ESYMMETRY",
           5: "SR_ENONFINITE", 6: "SR_ETIMEOUT", 7: "SR_EUNSUPPORTED"}


class SrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Bond(C.Structure):
    _fields_ = [("from_basis", C.c_int), ("to_basis", C.c_int), ("da", C.c_int * 3)]


class _Coupling(C.Structure):
    _fields_ = [("frm", C.c_int * 4), ("to", C.c_int * 4), ("M", C.c_double * 9)]


class _Desc(C.Structure):
    _fields_ = [("prim", C.c_double * 9), ("n_basis", C.c_int), ("basis_xyz", C.POINTER(C.c_double)),
                ("n_bonds", C.c_int), ("bonds", C.POINTER(_Bond)), ("n_couplings", C.c_int),
                ("couplings", C.POINTER(_Coupling)), ("range_L", C.c_int), ("backend", C.c_int),
                ("eps", C.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load libsr.so (building it first if the sources are newer).  Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        if not os.path.exists(path):
            raise OSError(f"CUDA library not found at {path}")
        lib = C.CDLL(path)
        vp, i, d, l = C.c_void_p, C.c_int, C.c_double, C.c_long
        ip, dp, lp = C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_long)
        sig = {
            "sr_lattice_create": [C.POINTER(_Desc), C.POINTER(vp)],
            "sr_lattice_info": [vp, ip, ip, ip, lp],
            "sr_lattice_representatives": [vp, ip],
            "sr_lattice_map_pair": [vp, ip, ip, ip, ip],
            "sr_lattice_map_pair_components": [vp, ip, ip, ip, ip, ip],
            "sr_lattice_destroy": [vp],
            "sr_frequency_mesh_exponential": [i, d, d, dp],
            "sr_flow_init": [vp, i, dp, d, i, vp, C.POINTER(vp)],
            "sr_flow_init_tangent": [vp, i, dp, d, i, dp, vp, C.POINTER(vp)],
            "sr_flow_tangents": [vp, ip],
            "sr_flow_set_tensor_cores": [vp, i],
            "sr_flow_tensor_cores": [vp, ip],
            "sr_measure_susceptibility_tangent": [vp, i, dp, dp, dp],
            "sr_flow_sizes": [vp, lp, ip, ip],
            "sr_flow_rhs": [vp, d, vp, vp],
            "sr_flow_step": [vp, d, i, d, d, dp],
            "sr_flow_stats": [vp, dp, lp, lp, lp],
            "sr_flow_set_step_limit": [vp, l],
            "sr_measure_susceptibility": [vp, i, dp, dp, vp],
            "sr_flow_chi_sites": [vp, ip],
            "sr_measure_susceptibility_static": [vp, i, vp, vp],
            "sr_flow_get_state": [vp, vp, vp],
            "sr_flow_set_state": [vp, d, vp, vp],
            "sr_flow_lambda": [vp, dp],
            "sr_flow_destroy": [vp],
            "sr_flow_rhs_adjoint": [vp, d, vp, vp, vp, vp],
            "sr_flow_step_adjoint": [vp, d, d, vp, vp, vp, vp],
            "sr_measure_susceptibility_adjoint": [vp, i, dp, dp, vp, vp],
            "sr_couplings_linear": [i, dp, i, dp, dp],
            "sr_flow_rhs_pairs": [vp, d, i, i, vp, vp],
            "sr_flow_advance": [vp, d, vp, vp],
            "sr_flow_initial_vertex_adjoint": [vp, i, dp, vp, dp],
            "sr_flow_profile_enable": [vp, i],
            "sr_flow_profile_read": [vp, dp, lp],
            "sr_flow_node_counts": [vp, ip],
            "sr_flow_lattice_sum_products": [vp, lp],
            "sr_flow_launch_info": [vp, ip],
            "sr_peak_fma": [i, dp],
            "sr_batch_create": [i, C.POINTER(vp), C.POINTER(vp)],
            "sr_batch_run": [vp, i, dp, i, i],
            "sr_batch_info": [vp, ip, ip, dp, dp, lp],
            "sr_batch_destroy": [vp],
            "sr_batch_classes": [vp, ip],
            "sr_batch_class": [vp, i, ip, lp, ip, ip, ip, dp],
            "sr_batch_parallel_classes": [vp, ip],
            "sr_batch_force_launch": [vp, i],
            "sr_batch_class_launch": [vp, i, ip],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        lib.sr_last_error.restype = C.c_char_p
        lib.sr_last_error.argtypes = []
        _lib = lib
        return lib


def _check(st: int):
    if st != 0:
        raise SrError(st, load_library().sr_last_error().decode())


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def sr_peak_fma(precision: int) -> float:
    v = C.c_double()
    _check(load_library().sr_peak_fma(int(precision), C.byref(v)))
    return v.value


def sr_couplings_linear(theta, B) -> np.ndarray:
    """sr_couplings_linear: M_c = sum_p theta_p B[p, c] (B: n_par x n_couplings x 3 x 3)."""
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    Bc = np.ascontiguousarray(B, dtype=np.float64)
    if Bc.ndim != 4 or Bc.shape[0] != th.size or Bc.shape[2:] != (3, 3):
        raise ValueError("B must be n_par x n_couplings x 3 x 3")
    M = np.zeros(Bc.shape[1:])
    _check(load_library().sr_couplings_linear(th.size, _dptr(th), Bc.shape[1], _dptr(Bc), _dptr(M)))
    return M


def sr_frequency_mesh_exponential(n: int, wmin: float, wmax: float) -> np.ndarray:
    out = np.zeros(n)
    _check(load_library().sr_frequency_mesh_exponential(n, wmin, wmax, _dptr(out)))
    return out


class Lattice:
    """sr_lattice_create on plain arrays (prim 3x3, basis nb x 3, bonds (from, to, da0, da1, da2),
    couplings (from[4], to[4], M 3x3))."""

    def __init__(self, prim, basis, bonds, couplings, L: int, backend: int = SR_SU2, eps: float = 1e-5):
        lib = load_library()
        self._lib = lib
        prim = np.ascontiguousarray(prim, dtype=np.float64).reshape(3, 3)
        self._basis = np.ascontiguousarray(basis, dtype=np.float64).reshape(-1, 3)
        self._bonds = (_Bond * len(bonds))()
        for k, (f, t, d0, d1, d2) in enumerate(bonds):
            self._bonds[k].from_basis, self._bonds[k].to_basis = int(f), int(t)
            self._bonds[k].da[:] = [int(d0), int(d1), int(d2)]
        self._coups = (_Coupling * max(1, len(couplings)))()
        for k, (frm, to, M) in enumerate(couplings):
            self._coups[k].frm[:] = [int(x) for x in frm]
            self._coups[k].to[:] = [int(x) for x in to]
            self._coups[k].M[:] = [float(x) for x in np.asarray(M, dtype=np.float64).reshape(9)]
        desc = _Desc()
        desc.prim[:] = list(prim.reshape(9))
        desc.n_basis = self._basis.shape[0]
        desc.basis_xyz = _dptr(self._basis)
        desc.n_bonds = len(bonds)
        desc.bonds = self._bonds
        desc.n_couplings = len(couplings)
        desc.couplings = self._coups
        desc.range_L = int(L)
        desc.backend = int(backend)
        desc.eps = float(eps)
        h = C.c_void_p()
        _check(lib.sr_lattice_create(C.byref(desc), C.byref(h)))
        self.h = h
        self.backend = backend
        self.prim = prim
        self.basis = self._basis
        ns, nt, nb, P = C.c_int(), C.c_int(), C.c_int(), C.c_long()
        _check(lib.sr_lattice_info(h, C.byref(ns), C.byref(nt), C.byref(nb), C.byref(P)))
        self.N_s, self.N_tot, self.N_basis, self.P = ns.value, nt.value, nb.value, P.value

    @classmethod
    def from_model(cls, model, L: int, backend=None, eps: float = 1e-5) -> "Lattice":
        cell = model.cell
        coups = [(c.frm, c.to, c.M) for c in model.couplings]
        be = backend if backend is not None else {"XYZ": SR_XYZ, "TRI": SR_TRI}.get(getattr(model, "backend", "SU2"), SR_SU2)
        return cls(cell.prim, cell.basis, cell.bonds, coups, L, be, eps)

    def representatives(self) -> np.ndarray:
        out = np.zeros((self.N_s, 4), dtype=np.int32)
        _check(self._lib.sr_lattice_representatives(self.h, _iptr(out)))
        return out

    def map_pair(self, i1, i2):
        a = np.ascontiguousarray(i1, dtype=np.int32)
        b = np.ascontiguousarray(i2, dtype=np.int32)
        r = C.c_int()
        perm = np.zeros(4, dtype=np.int32)
        _check(self._lib.sr_lattice_map_pair(self.h, _iptr(a), _iptr(b), C.byref(r), _iptr(perm)))
        return r.value, perm

    @property
    def n_comp(self) -> int:
        return {SR_SU2: 2, SR_XYZ: 4, SR_TRI: 16}[int(self.backend)]

    def map_pair_components(self, i1, i2):
        """(r, comp, sign): component c of the pair (i1, i2) is sign[c] * stored component
        comp[c] of irreducible site r (r = -1 beyond range)."""
        a = np.ascontiguousarray(i1, dtype=np.int32)
        b = np.ascontiguousarray(i2, dtype=np.int32)
        r = C.c_int()
        comp = np.zeros(self.n_comp, dtype=np.int32)
        sign = np.zeros(self.n_comp, dtype=np.int32)
        _check(self._lib.sr_lattice_map_pair_components(self.h, _iptr(a), _iptr(b), C.byref(r), _iptr(comp), _iptr(sign)))
        return r.value, comp, sign

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self._lib.sr_lattice_destroy(self.h)
                self.h = None
        except Exception:
            pass


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Flow:
    """sr_flow_init: a flow on the current CUDA device and PyTorch stream."""

    def __init__(self, lattice: Lattice, mesh, lambda_init: float, precision: int = SR_FP64, stream=None,
                 tangents=None):
        """tangents: optional (n_par, n_couplings, 3, 3) derivatives of the coupling matrices
        (sr_flow_init_tangent): the flow then carries d/dtheta_p of every value."""
        import torch
        lib = load_library()
        self._lib = lib
        self.lattice = lattice
        self.mesh = np.ascontiguousarray(mesh, dtype=np.float64)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        if tangents is None:
            _check(lib.sr_flow_init(lattice.h, len(self.mesh), _dptr(self.mesh), float(lambda_init), int(precision),
                                    C.c_void_p(stream.cuda_stream), C.byref(h)))
            self.n_tan = 0
            self.ts = 1
        else:
            dM = np.ascontiguousarray(tangents, dtype=np.float64)
            npar = dM.shape[0]
            _check(lib.sr_flow_init_tangent(lattice.h, len(self.mesh), _dptr(self.mesh), float(lambda_init), npar,
                                            _dptr(dM.reshape(-1)), C.c_void_p(stream.cuda_stream), C.byref(h)))
            self.n_tan = npar
            self.ts = 3      # (value, d/dtheta_1, d/dtheta_2) per state scalar
        self.h = h
        ng, nf, nc = C.c_long(), C.c_int(), C.c_int()
        _check(lib.sr_flow_sizes(h, C.byref(ng), C.byref(nf), C.byref(nc)))
        self.n_gamma, self.N, self.n_comp = ng.value, nf.value, nc.value
        self.npair = self.N * (self.N + 1) // 2

    # state layout: [pair][t][c][site]
    def shape(self):
        return (self.npair, self.N, self.n_comp, self.lattice.N_s)

    def rhs(self, lam: float, dsigma=None, dgamma=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if dsigma is None:
            dsigma = torch.empty(self.N * self.ts, dtype=torch.float64, device=dev)
        if dgamma is None:
            dgamma = torch.empty(self.n_gamma * self.ts, dtype=torch.float64, device=dev)
        _check(self._lib.sr_flow_rhs(self.h, float(lam), _ptr(dsigma), _ptr(dgamma)))
        return dsigma, dgamma

    @property
    def entries_per_pair(self) -> int:
        """State doubles of one stored (s, u) pair: all t, components and sites (with tangents)."""
        return self.N * self.n_comp * self.lattice.N_s * self.ts

    def rhs_pairs(self, lam: float, pair_begin: int, pair_end: int, dsigma, dgamma):
        """sr_flow_rhs_pairs: dgamma/dLambda into dsigma, and dGamma/dLambda of the stored pairs
        [pair_begin, pair_end) into their slice of dgamma (state layout; the rest untouched)."""
        if dsigma.numel() < self.N * self.ts or dgamma.numel() < self.n_gamma * self.ts:
            raise ValueError("dsigma / dgamma smaller than the state")
        _check(self._lib.sr_flow_rhs_pairs(self.h, float(lam), int(pair_begin), int(pair_end), _ptr(dsigma), _ptr(dgamma)))
        return dsigma, dgamma

    def advance(self, lam_next: float, dsigma, dgamma):
        """sr_flow_advance: Euler step to lam_next with a supplied right-hand side."""
        if dsigma.numel() < self.N * self.ts or dgamma.numel() < self.n_gamma * self.ts:
            raise ValueError("dsigma / dgamma smaller than the state")
        _check(self._lib.sr_flow_advance(self.h, float(lam_next), _ptr(dsigma), _ptr(dgamma)))

    def step(self, lam_next: float, method: int = SR_EULER, rtol: float = 1e-6, atol: float = 1e-10) -> float:
        reached = C.c_double()
        _check(self._lib.sr_flow_step(self.h, float(lam_next), int(method), float(rtol), float(atol), C.byref(reached)))
        return reached.value

    @property
    def tensor_cores(self) -> bool:
        """Whether the SU2 lattice sum of this FP32-mixed flow runs on the tensor cores."""
        v = C.c_int()
        _check(self._lib.sr_flow_tensor_cores(self.h, C.byref(v)))
        return bool(v.value)

    @tensor_cores.setter
    def tensor_cores(self, on: bool):
        _check(self._lib.sr_flow_set_tensor_cores(self.h, 1 if on else 0))

    def set_step_limit(self, n: int):
        _check(self._lib.sr_flow_set_step_limit(self.h, int(n)))

    def stats(self):
        e, n, a, r = C.c_double(), C.c_long(), C.c_long(), C.c_long()
        _check(self._lib.sr_flow_stats(self.h, C.byref(e), C.byref(n), C.byref(a), C.byref(r)))
        return {"last_err": e.value, "n_rhs": n.value, "n_accept": a.value, "n_reject": r.value}

    @property
    def lam(self) -> float:
        v = C.c_double()
        _check(self._lib.sr_flow_lambda(self.h, C.byref(v)))
        return v.value

    def measure(self, kpts=None, want_ij: bool = True):
        """chi(k) at the given momenta (host numpy) and chi_ij (CUDA tensor [b][j][c])."""
        import torch
        nk = 0 if kpts is None else len(kpts)
        kp = np.ascontiguousarray(np.zeros((0, 3)) if kpts is None else kpts, dtype=np.float64).reshape(-1, 3)
        chik = np.zeros(max(nk, 1))
        chi_ij = None
        if want_ij:
            n = self.lattice.N_basis * self.lattice.N_tot * self.n_comp
            chi_ij = torch.empty(n, dtype=torch.float64, device="cuda")
        _check(self._lib.sr_measure_susceptibility(self.h, nk, _dptr(kp), _dptr(chik) if nk else None,
                                                   _ptr(chi_ij)))
        if chi_ij is not None:
            chi_ij = chi_ij.view(self.lattice.N_basis, self.lattice.N_tot, self.n_comp)
        return (chik[:nk] if nk else None), chi_ij

    def measure_static(self, k_dev, out_dev):
        """sr_measure_susceptibility_static: chi(k) from device momenta (n_k x 3 float64) into a
        device output (n_k float64), allocating nothing."""
        n = out_dev.numel()
        if k_dev.numel() != 3 * n:
            raise ValueError("k_dev must hold 3 values per output")
        _check(self._lib.sr_measure_susceptibility_static(self.h, int(n), _ptr(k_dev), _ptr(out_dev)))
        return out_dev

    def measure_tangent(self, kpts):
        """(chi(k), d chi(k) / d theta) of a tangent flow: arrays (n_k,), (n_k, n_par)."""
        kp = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
        nk = kp.shape[0]
        chik = np.zeros(nk)
        d = np.zeros(nk * 2)
        _check(self._lib.sr_measure_susceptibility_tangent(self.h, nk, _dptr(kp), _dptr(chik), _dptr(d)))
        return chik, d.reshape(nk, 2)[:, :self.n_tan]

    def chi_sites(self) -> np.ndarray:
        out = np.zeros((self.lattice.N_basis * self.lattice.N_tot, 4), dtype=np.int32)
        _check(self._lib.sr_flow_chi_sites(self.h, _iptr(out)))
        return out.reshape(self.lattice.N_basis, self.lattice.N_tot, 4)

    def get_state(self):
        """(sigma, gamma) as CUDA tensors; tangent flows interleave (value, d1, d2)."""
        import torch
        g = torch.empty(self.N * self.ts, dtype=torch.float64, device="cuda")
        G = torch.empty(self.n_gamma * self.ts, dtype=torch.float64, device="cuda")
        _check(self._lib.sr_flow_get_state(self.h, _ptr(g), _ptr(G)))
        return g, G

    def set_state(self, lam: float, sigma=None, gamma=None):
        _check(self._lib.sr_flow_set_state(self.h, float(lam), _ptr(sigma), _ptr(gamma)))

    # ---- adjoint (FP64 plain flows) ----
    def rhs_adjoint(self, lam: float, fbar_sigma, fbar_gamma):
        """sr_flow_rhs_adjoint: (J^T fbar) of the right-hand side at the current state, as new
        CUDA tensors (sigma part, gamma part)."""
        import torch
        gs = torch.empty(self.N, dtype=torch.float64, device="cuda")
        gG = torch.empty(self.n_gamma, dtype=torch.float64, device="cuda")
        _check(self._lib.sr_flow_rhs_adjoint(self.h, float(lam), _ptr(fbar_sigma), _ptr(fbar_gamma), _ptr(gs),
                                             _ptr(gG)))
        return gs, gG

    def step_adjoint(self, lam_from: float, lam_to: float, bar_sigma, bar_gamma, out_sigma=None, out_gamma=None):
        """sr_flow_step_adjoint: the adjoint of one Euler step from lam_from (the flow's state)
        to lam_to.  Outputs may alias the inputs."""
        if out_sigma is None:
            out_sigma = bar_sigma
        if out_gamma is None:
            out_gamma = bar_gamma
        _check(self._lib.sr_flow_step_adjoint(self.h, float(lam_from), float(lam_to), _ptr(bar_sigma), _ptr(bar_gamma),
                                              _ptr(out_sigma), _ptr(out_gamma)))
        return out_sigma, out_gamma

    def measure_adjoint(self, kpts, chi_bar):
        """sr_measure_susceptibility_adjoint: d (sum_k chi_bar_k chi(k)) / d state, as new CUDA
        tensors (sigma part, gamma part)."""
        import torch
        kp = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
        cb = np.ascontiguousarray(chi_bar, dtype=np.float64).reshape(-1)
        if cb.shape[0] != kp.shape[0]:
            raise ValueError("one chi_bar value per momentum")
        gs = torch.empty(self.N, dtype=torch.float64, device="cuda")
        gG = torch.empty(self.n_gamma, dtype=torch.float64, device="cuda")
        _check(self._lib.sr_measure_susceptibility_adjoint(self.h, kp.shape[0], _dptr(kp), _dptr(cb), _ptr(gs),
                                                           _ptr(gG)))
        return gs, gG

    def initial_vertex_adjoint(self, dM, bar_gamma) -> np.ndarray:
        """sr_flow_initial_vertex_adjoint: grad_p = <d Gamma_init / d theta_p, bar_gamma> for
        coupling derivatives dM (n_par x n_couplings x 3 x 3); returns an array (n_par,)."""
        d = np.ascontiguousarray(dM, dtype=np.float64)
        grad = np.zeros(d.shape[0])
        _check(self._lib.sr_flow_initial_vertex_adjoint(self.h, d.shape[0], _dptr(d), _ptr(bar_gamma), _dptr(grad)))
        return grad

    def profile_enable(self, on: bool = True):
        _check(self._lib.sr_flow_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """(ms[3], launches[3]) of the self-energy, node and vertex kernels."""
        ms = np.zeros(3)
        n = (C.c_long * 3)()
        _check(self._lib.sr_flow_profile_read(self.h, _dptr(ms), n))
        return ms, np.array(list(n))

    def lattice_sum_products(self) -> int:
        n = C.c_long()
        _check(self._lib.sr_flow_lattice_sum_products(self.h, C.byref(n)))
        return n.value

    def launch_info(self) -> dict:
        out = np.zeros(4, dtype=np.int32)
        _check(self._lib.sr_flow_launch_info(self.h, _iptr(out)))
        return {"tc_grid": int(out[0]), "tc_smem": int(out[1]), "tc_occupancy_runtime": int(out[2]),
                "smem": int(out[3])}

    def node_counts(self) -> np.ndarray:
        out = np.zeros(3 * self.N, dtype=np.int32)
        _check(self._lib.sr_flow_node_counts(self.h, _iptr(out)))
        return out.reshape(3, self.N)

    def close(self):
        if getattr(self, "h", None):
            self._lib.sr_flow_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """sr_batch_create / sr_batch_run: FP32-mixed flows integrated together (persistent vertex
    kernel over all instances, CUDA-graph-captured Euler loop, autotuned launch shape)."""

    def __init__(self, flows):
        lib = load_library()
        self._lib = lib
        self.flows = list(flows)
        arr = (C.c_void_p * len(self.flows))(*[f.h.value for f in self.flows])
        h = C.c_void_p()
        _check(lib.sr_batch_create(len(self.flows), arr, C.byref(h)))
        self.h = h

    def run(self, lambdas, use_graph: bool = True, autotune: bool = True):
        lams = np.ascontiguousarray(lambdas, dtype=np.float64)
        _check(self._lib.sr_batch_run(self.h, len(lams), _dptr(lams), 1 if use_graph else 0, 1 if autotune else 0))

    def info(self):
        qc, ct, tm, rm, u = C.c_int(), C.c_int(), C.c_double(), C.c_double(), C.c_long()
        _check(self._lib.sr_batch_info(self.h, C.byref(qc), C.byref(ct), C.byref(tm), C.byref(rm), C.byref(u)))
        return {"qc": qc.value, "ctas_per_sm": ct.value, "tune_ms": tm.value, "run_ms": rm.value, "units": u.value}

    def classes(self):
        n = C.c_int()
        _check(self._lib.sr_batch_classes(self.h, C.byref(n)))
        out = []
        for k in range(n.value):
            ni, u, sm, qc, ct, ms = C.c_int(), C.c_long(), C.c_int(), C.c_int(), C.c_int(), C.c_double()
            _check(self._lib.sr_batch_class(self.h, k, C.byref(ni), C.byref(u), C.byref(sm), C.byref(qc), C.byref(ct),
                                            C.byref(ms)))
            out.append({"instances": ni.value, "units": u.value, "smem_bytes": sm.value, "node_block": qc.value,
                        "ctas_per_sm": ct.value, "tuned_ms": ms.value})
        return out

    @property
    def parallel_classes(self) -> bool:
        v = C.c_int()
        _check(self._lib.sr_batch_parallel_classes(self.h, C.byref(v)))
        return bool(v.value)

    def force_launch(self, mode: int):
        """0: autotuned launch form per class, 1: persistent kernels, 2: per-instance kernels."""
        _check(self._lib.sr_batch_force_launch(self.h, int(mode)))

    def class_launches(self):
        """Per class: True if it runs its instances' own kernels, False if its persistent kernel."""
        n = C.c_int()
        _check(self._lib.sr_batch_classes(self.h, C.byref(n)))
        out = []
        for k in range(n.value):
            v = C.c_int()
            _check(self._lib.sr_batch_class_launch(self.h, k, C.byref(v)))
            out.append(bool(v.value))
        return out

    def close(self):
        if getattr(self, "h", None):
            self._lib.sr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
