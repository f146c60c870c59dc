"""The allocation-free correlation entry point (sr_measure_susceptibility_static).

It serves callers that cannot allocate device memory while they run -- code inside a CUDA
stream capture, or hosts whose device memory belongs to another framework's pool -- by
keeping its intermediate chi_ij table in a static device array.  This test calls it through
the C ABI and checks it against the regular entry point on two calls in a row.  The file
is collected last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402


def test_static_chi_matches_allocating_entry_point_twice():
    lib = sr.load_library()
    model = W.square_j1j2(1.0, 0.5)
    mesh = O.mesh_exponential(8, 0.02, 20.0)
    lat = sr.Lattice.from_model(model, 3)
    fl = sr.Flow(lat, mesh, 10.0, sr.SR_FP64)
    ks = np.linspace(-math.pi, math.pi, 9)
    kpts = np.array([[a, b, 0.0] for a in ks for b in ks])
    k_dev = torch.tensor(kpts.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.full((len(kpts),), float("nan"), dtype=torch.float64, device="cuda")
    for lam in (4.0, 1.5):   # two calls in a row, at two different states
        fl.step(lam, sr.SR_EULER)
        ref, _ = fl.measure(kpts, want_ij=False)
        st = lib.sr_measure_susceptibility_static(fl.h, len(kpts), C.c_void_p(k_dev.data_ptr()),
                                                   C.c_void_p(out.data_ptr()))
        assert st == 0, lib.sr_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-14)
    fl.close()
