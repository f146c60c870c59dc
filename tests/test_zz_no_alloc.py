"""The allocation-free correlation entry point (sr_measure_susceptibility_static).

It serves callers that cannot allocate device memory while they run -- hosts whose device
memory belongs entirely to another framework's pool or to a fixed budget -- by keeping its
intermediate chi_ij table in a static device array.  These tests call it through the C ABI and
check it, on two calls in a row at two different states, against the regular (allocating)
entry point and against the oracle's chi(k), for the SU(2), XYZ and TRI cores, and check that
a table above the static limit is rejected without touching the output.  The file is
collected last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests.helpers import oracle_to_gpu, tri_oracle_to_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402

CASES = [
    ("su2_square_j1j2", lambda: W.square_j1j2(1.0, 0.5), 3, False),
    ("xyz_honeycomb_kitaev", lambda: W.honeycomb_kitaev(0.2, -1.0), 2, False),
    ("tri_kagome_dm", lambda: W.kagome_dm(1.0, 0.5), 2, True),
]


def _kgrid(n=9):
    ks = np.linspace(-math.pi, math.pi, n)
    return np.array([[a, b, 0.0] for a in ks for b in ks])


def _static(lib, fl, k_dev, out):
    st = lib.sr_measure_susceptibility_static(fl.h, out.numel(), C.c_void_p(k_dev.data_ptr()),
                                              C.c_void_p(out.data_ptr()))
    return st


@pytest.mark.parametrize("name,mk,L,tri", CASES, ids=[c[0] for c in CASES])
def test_static_chi_matches_allocating_entry_point_and_oracle_twice(name, mk, L, tri):
    lib = sr.load_library()
    model = mk()
    mesh = O.mesh_exponential(7, 0.02, 20.0)
    of = (O.OracleFlowTRI if tri else O.OracleFlow)(model, L, mesh)
    lat = sr.Lattice.from_model(model, L)
    fl = sr.Flow(lat, mesh, 10.0, sr.SR_FP64)
    kpts = _kgrid()
    k_dev = torch.tensor(kpts.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.full((len(kpts),), float("nan"), dtype=torch.float64, device="cuda")
    lams = [10.0, 4.0, 1.5]
    for a, b in zip(lams[:-1], lams[1:]):   # two calls in a row, at two different states
        of.euler(a, b)
        gam, G = of.get_state()
        Gg = tri_oracle_to_gpu(of, lat, G) if tri else oracle_to_gpu(of, lat, G, fl.n_comp)
        fl.set_state(b, torch.tensor(gam, device="cuda"), torch.tensor(Gg.reshape(-1), device="cuda"))
        ref, _ = fl.measure(kpts, want_ij=False)
        st = _static(lib, fl, k_dev, out)
        assert st == 0, lib.sr_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-14)
        exp = of.chi_k(b, kpts)
        assert np.abs(got - exp).max() <= 1e-10 * np.abs(exp).max()
    fl.close()


def _square_supercell(k):
    """The square lattice described with a k x k supercell: k^2 equivalent basis sites, so the
    correlation table (basis sites x sites in range) grows with k^2 while the irreducible
    vertex stays that of the square lattice."""
    basis = [[i, j, 0] for j in range(k) for i in range(k)]
    bonds = []
    for j in range(k):
        for i in range(k):
            b = j * k + i
            bonds.append((b, j * k + (i + 1) % k, 1 if i + 1 == k else 0, 0, 0))
            bonds.append((b, ((j + 1) % k) * k + i, 0, 1 if j + 1 == k else 0, 0))
    return W.UnitCell(f"square_{k}x{k}", np.diag([k, k, 1.0]), np.array(basis, dtype=float), bonds)


def test_static_chi_rejects_tables_above_the_limit():
    """The square lattice as a 16 x 16 supercell at range 16: 256 basis sites x 545 sites x 2
    components = 279,040 chi_ij values, above the static array's 262,144: the call fails with
    SR_EINVAL before any launch and the caller's output keeps its contents."""
    lib = sr.load_library()
    lat = sr.Lattice.from_model(W.nn_heisenberg(_square_supercell(16)), 16)
    assert lat.N_basis * lat.N_tot * 2 > 262144
    fl = sr.Flow(lat, O.mesh_exponential(2, 0.1, 1.0), 5.0, sr.SR_FP64)
    kpts = _kgrid(3)
    k_dev = torch.tensor(kpts.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.full((len(kpts),), 123.25, dtype=torch.float64, device="cuda")
    st = _static(lib, fl, k_dev, out)
    torch.cuda.synchronize()
    assert st == sr.SR_EINVAL
    assert "static limit" in lib.sr_last_error().decode()
    assert torch.all(out == 123.25)
    fl.close()
