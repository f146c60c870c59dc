"""One right-hand side of a named workload, for profiler captures of the vertex kernels.

    python -m paper_2109_13317_gb300.profile_case --workload kagome_dm_L7 --n-freq 48 --precision fp64

builds the flow of the configuration (optionally with another number of frequencies), takes
two Euler steps (Lambda_max -> 0.4 Lambda_max -> 0.16 Lambda_max, two vertex-kernel launches)
and evaluates one right-hand side at 0.1 Lambda_max (the third launch), so that a capture
skips two launches of the vertex kernel and takes one.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True)
    ap.add_argument("--n-freq", type=int, default=0, help="override the configuration's frequency count")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import workloads as W
    from . import binding as sr
    cfg = W.config(a.workload)
    n = a.n_freq or cfg.n_freq
    lat = sr.Lattice.from_model(cfg.model, cfg.L)
    mesh = sr.sr_frequency_mesh_exponential(n, cfg.w_min, cfg.w_max)
    prec = sr.SR_FP64 if a.precision == "fp64" else sr.SR_FP32_MIXED
    fl = sr.Flow(lat, mesh, cfg.lam_max, prec)
    fl.step(0.4 * cfg.lam_max, sr.SR_EULER)
    fl.step(0.16 * cfg.lam_max, sr.SR_EULER)
    fl.rhs(0.1 * cfg.lam_max)
    torch.cuda.synchronize()
    print(f"{cfg.name}: N_s={lat.N_s} P={lat.P} n_freq={n} entries={fl.n_gamma} precision={a.precision}")
    fl.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
