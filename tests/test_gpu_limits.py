"""The largest frequency mesh the library accepts (256 positive frequencies) on the first
right-hand side of the flow, whose value at the bare vertex is known in closed form: gamma = 0
and Gamma = J/4 make the Katanin part vanish, the delta parts of the three bubbles integrate
exactly, and the lattice sum reduces to sum_j J_1j J_j2.  The closed form is written here from
the flow equations, independently of the oracle and of the library.  Also the rejection of a
larger mesh."""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_13317_gb300 as sr  # noqa: E402

NMAX = 256


def _bubble(lam, v):
    """delta-part integral of G(w)S(v-w) + G(v-w)S(w) at gamma = 0 (s channel); the t and u
    channels carry the opposite sign."""
    th = v - 2 * lam >= 0
    return (2.0 / lam) * (1.0 / (v + lam) - (1.0 / (v - lam) if th else 0.0))


@pytest.mark.parametrize("prec,tol", [(sr.SR_FP64, 1e-12), (sr.SR_FP32_MIXED, 2e-5)])
def test_largest_mesh_first_rhs_closed_form(prec, tol):
    model = W.nn_heisenberg(W.square(), 1.0)    # J1 only: J_ii = 0, on-site terms vanish
    lat = sr.Lattice.from_model(model, 1)       # the reference site and its 4 neighbours
    mesh = sr.sr_frequency_mesh_exponential(NMAX, 0.01, 50.0)
    lam = 3.7
    fl = sr.Flow(lat, mesh, lam, prec)
    dg, dG = fl.rhs(lam)
    torch.cuda.synchronize()
    assert float(dg.abs().max()) == 0.0
    G = dG.view(fl.npair, fl.N, 2, lat.N_s).cpu().numpy()
    reps = lat.representatives()
    N = NMAX
    si = np.array([s for s in range(N) for u in range(s + 1)])
    ui = np.array([u for s in range(N) for u in range(s + 1)])
    Is = np.array([_bubble(lam, mesh[i]) for i in range(N)])
    for r, rep in enumerate(reps):
        d = tuple(int(x) for x in rep[:3])
        J12 = 1.0 if sum(abs(x) for x in d) == 1 else 0.0
        # lattice sum over j within range 1 of both sites: only the on-site ends contribute
        # J_1j J_j2 with j a common neighbour; for range 1 the common neighbours of i1 and a
        # neighbour i2 are none, of i1 with itself the four neighbours
        rpa = 4.0 if d == (0, 0, 0) else 0.0
        e0 = 3 * (J12 / 4) ** 2 * (Is[si] - Is[ui]) / (2 * math.pi)
        ez = (-2 * (J12 / 4) ** 2 * Is[si] - 2 * (J12 / 4) ** 2 * Is[ui]) / (2 * math.pi)
        scale = max(np.abs(e0).max(), np.abs(ez).max(), 1e-300)
        for ti in range(0, N, 17):
            It = -Is[ti]
            ezt = ez - 2 * It * rpa / 16 / (2 * math.pi)
            got0 = G[:, ti, 0, r]
            got1 = G[:, ti, 1, r]
            sc = max(scale, abs(2 * It * rpa / 16 / (2 * math.pi)))
            assert np.abs(got0 - e0).max() <= tol * sc
            assert np.abs(got1 - ezt).max() <= tol * sc
    fl.close()


def test_mesh_larger_than_the_limit_is_rejected():
    lat = sr.Lattice.from_model(W.nn_heisenberg(W.square(), 1.0), 1)
    mesh = sr.sr_frequency_mesh_exponential(NMAX + 1, 0.01, 50.0)
    with pytest.raises(sr.SrError) as e:
        sr.Flow(lat, mesh, 3.0, sr.SR_FP64)
    assert e.value.status == sr.SR_EINVAL
