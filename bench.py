"""Benchmark of the pf-FRG flow step on GB300.

Workload: square-lattice J1-J2 Heisenberg model (J1 = 1, J2 = 0.5), truncation range 7
bonds (N_s = 20 irreducible sites, N_tot = 113), 48 log-spaced frequencies 0.001..100,
SU(2) core; 2,257,920 stored vertex entries.  One step = one full pass of the hot path:
self-energy flow, integration nodes, vertex flow (s, t, u channels with the lattice sum),
Euler update and the susceptibility chi(k) on a 64 x 64 momentum grid.  The flow is first
advanced (untimed) from Lambda = 100 to mid-flow (Lambda ~ 1) so every step carries the
full regular (Katanin) integration work.

Metric: RHS vertex entries per second (stored Gamma entries x right-hand-side evaluations
/ time).  ``--impl reference`` times the CPU oracle on the machine's host cores on a bounded
sample of entries of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOAD = "square_j1j2_L7"
METRIC = "RHS vertex entries/s"
UNIT = "entries/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-mixed side measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-flow", action="store_true", help="skip the full adaptive Lambda flow")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched coupling sweep")
    ap.add_argument("--profile-rhs", action="store_true",
                    help="profiling case: two Euler steps of the workload, then one right-hand side, and exit")
    ap.add_argument("--n-freq", type=int, default=0, help="profiling case: override the frequency count")
    ap.add_argument("--oracle-flow", action="store_true",
                    help="time the CPU oracle's whole Euler flow of the workload (all host cores), print one "
                         "JSON line and exit; --oracle-budget bounds it (the rest is extrapolated per step)")
    ap.add_argument("--oracle-budget", type=float, default=600.0, help="seconds for --oracle-flow")
    ap.add_argument("--profile-lambda", type=float, default=0.0,
                    help="profiling case: cutoff of the profiled right-hand side (default 0.1 Lambda_max)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["square_j1j2_L7", "square_j1_L3", "pyrochlore_L6", "honeycomb_hk_L5", "kagome_dm_L7"],
                    help="configuration to measure (the default is the headline workload)")
    return ap.parse_args()


def _describe(cfg):
    """Lattice, couplings and spin core of a configuration, for the JSON line."""
    m = cfg.model
    js = sorted({round(float(c.M[2, 2]), 6) for c in m.couplings})
    return {"lattice": f"{m.cell.name}, couplings zz in {js}", "core": m.backend}


def _oracle_fits(cfg, limit_bytes: float = 1e9) -> bool:
    """Whether the oracle's translation-only vertex of the configuration stays below limit_bytes
    (the TRI oracle keeps 16 complex functions: 4 GB)."""
    from oracle import oracle as O
    tri = cfg.model.backend == "TRI"
    of = (O.OracleFlowTRI if tri else O.OracleFlow)(cfg.model, cfg.L, O.mesh_exponential(2, cfg.w_min, cfg.w_max))
    n = cfg.n_freq
    per = 16 * 16 if tri else 8 * 4
    return per * sum(of.nsite) * n * n * (n + 1) / 2 <= (4 * limit_bytes if tri else limit_bytes)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms during the timed region (the
    sampler is running before the region starts; samples taken before it are dropped)."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.samples and time.time() - t0 < 5.0:
            time.sleep(0.01)
        self.samples.clear()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _sync_all(torch, ws: int, cuda: bool = True):
    """Barrier over the ranks (one flow replica per GPU) and a device synchronize."""
    if ws > 1:
        torch.distributed.barrier()
    if cuda:
        torch.cuda.synchronize()


def _max_over_ranks(torch, value: float, ws: int, device="cuda") -> float:
    """The largest per-rank value (the job's time is its slowest rank's)."""
    if ws == 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_throughput(units_per_rank: float, ws: int, t_ms: float) -> float:
    """Whole-job units per second: every rank processed units_per_rank in t_ms (the max)."""
    return units_per_rank * ws / (t_ms * 1e-3)


def _algorithmic_flops(counts: np.ndarray, N: int, Ns: int, nc: int, P: int, nprod: int) -> float:
    """Floating-point operations of one vertex-flow launch, counted as the natural evaluation
    of the flow equations (an FMA = 2 flop).  Per stored triple (s, t, u) and integration node:
    every vertex row the equations need is interpolated over all irreducible sites and
    components; one of the three frequency arguments of every row is a mesh frequency, so an
    interpolated value is 4 corners = 4 FMA = 8 flop, and the node weight multiplies one row
    (1 flop per value).  s and u channels: two rows and the projected product (SU2 11 flop per
    site: A1 B1, its multiples and three FMAs plus two accumulations; XYZ 32).  t channel: two
    rows, two on-site rows (n_c values each), the on-site terms (SU2 6 flop per site and
    component, XYZ 7) and the lattice sum as one FMA (2 flop) per distinct product of table
    rows.  Per triple, the lattice sum's table gather adds P n_c flop.  TRI (n_c = 16): the
    s / u products are 256 FMA per site (512 flop), the two on-site terms 1024 flop per site
    (64 per value), and the lattice sum 64 FMA per table entry (nprod = 64 P), summed in
    place."""
    row = Ns * nc
    prod = {2: 11, 4: 32, 16: 512}[nc]
    onsite = {2: 6, 4: 7, 16: 64}[nc]
    per_s = 2 * row * 8 + row + Ns * prod
    per_u = per_s
    per_t = (2 * row + 2 * nc) * 8 + row + nc + 2 * nprod + onsite * row
    ns, nt, nu = counts[0].astype(np.float64), counts[1].astype(np.float64), counts[2].astype(np.float64)
    cs = np.arange(1, N + 1, dtype=np.float64)   # number of u_i <= s_i
    tot = N * float(np.sum(ns * cs)) * per_s                   # s channel: node count depends on s_i
    tot += (N * (N + 1) / 2) * float(np.sum(nt)) * per_t       # t channel: on t_i
    tot += N * float(np.sum(nu * (N - np.arange(N)))) * per_u  # u channel: on u_i
    if nc != 16:                                               # (the TRI kernel sums in place)
        tot += (N * N * (N + 1) / 2) * P * nc                  # lattice-sum gather per triple
    return tot


def _kernel_hash() -> str:
    """Hash of the device code of the vertex kernels: kernels.cuh, tc.cuh, su2f.cuh and flow.cu
    up to its host-side objects (changes to host code leave committed ncu figures valid)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2109_13317_gb300", "csrc")
    for f in ("kernels.cuh", "tc.cuh", "su2f.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "flow.cu"), "rb") as fh:
        src = fh.read()
    h.update(src.split(b'#include "adjoint.cuh"')[0])
    return h.hexdigest()[:16]


def _traffic(precision: str):
    """DRAM bytes per vertex-flow launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "gamma_rhs_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(precision)
        if e and e.get("kernel_hash") == _kernel_hash():
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


def _kgrid(n=64):
    ks = np.linspace(-2 * math.pi, 2 * math.pi, n)
    kx, ky = np.meshgrid(ks, ks, indexing="ij")
    return np.stack([kx.ravel(), ky.ravel(), np.zeros(n * n)], axis=1)


def _oracle_sampler(cfg, seed: int):
    """The oracle on the workload and a function timing its right-hand side on m random stored
    entries: returns (run(m) -> (entries, seconds), description of the state).  SU2 / XYZ:
    synthetic symmetric state at Lambda = 0.9, one stored entry per call of the oracle.  TRI:
    the initial vertex J/4 with a synthetic self-energy (the work per entry does not depend on
    the values), all 16 functions of a site pair and frequency triple per call."""
    from oracle import oracle as O
    mesh = O.mesh_exponential(cfg.n_freq, cfg.w_min, cfg.w_max)
    rng = np.random.default_rng(seed)
    N = cfg.n_freq
    if cfg.model.backend == "TRI":
        of = O.OracleFlowTRI(cfg.model, cfg.L, mesh)
        gam = 0.2 * np.tanh(mesh) + 0.05 * mesh / (1 + mesh)
        _, G = of.get_state()
        of.set_state(gam, G)

        def run(m):
            ent = []
            for _ in range(m):
                si = int(rng.integers(0, N))
                ent.append((0, int(rng.integers(0, of.nsite[0])), si, int(rng.integers(0, N)), int(rng.integers(0, si + 1))))
            ent = np.array(ent, dtype=np.int32)
            t0 = time.perf_counter()
            of.rhs_entries(0.9, ent)
            return 16 * m, time.perf_counter() - t0
        return run, "initial vertex J/4 with a synthetic self-energy at Lambda=0.9 (16 functions per sampled pair and triple)"
    of = O.OracleFlow(cfg.model, cfg.L, mesh)
    gam, G = W.synthetic_state(of, cfg.model, seed=3)
    of.set_state(gam, G)

    def run(m):
        ent = []
        for _ in range(m):
            si = int(rng.integers(0, N))
            ui = int(rng.integers(0, si + 1))
            ti = int(rng.integers(0, N))
            k = int(rng.integers(0, of.nsite[0]))
            ent.append((0, k, si, ti, ui))
        ent = np.array(ent, dtype=np.int32)
        t0 = time.perf_counter()
        of.rhs_entries(0.9, ent)
        return m, time.perf_counter() - t0
    return run, "synthetic symmetric state at Lambda=0.9"


def _cpu_baseline(cfg, target_s: float = 12.0):
    """The oracle as it stands, on the host's cores, on a bounded random sample of stored
    entries of the same workload."""
    from oracle import oracle as O
    run, state = _oracle_sampler(cfg, 5)
    run(4)
    n0 = 32
    e0, dt = run(n0)
    m = max(n0, int(n0 * target_s / max(dt, 1e-3)))
    e, dt = run(m)
    cores = O.OracleFlow.threads()
    # the same oracle on one core (a smaller sample of the same kind, ~target_s / 3)
    O.OracleFlow.set_threads(1)
    try:
        m1 = max(8, int(m * (target_s / 3) / target_s / max(cores, 1)))
        e1, dt1 = run(m1)
    finally:
        O.OracleFlow.set_threads(cores)
    # the oracle evaluates every symmetry-equivalent pair; a stored entry of the oracle's
    # translation-only vertex is one equation, as for the GPU's reduced vertex
    return {"value": e / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{e} random stored vertex entries (RHS of each, incl. self-energy flow) of the "
                      f"{cfg.name} workload, {state}; {dt:.1f} s",
            "single_thread": {"value": e1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{e1} random stored entries of the same kind; {dt1:.1f} s"}}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    cfg = W.config(args.workload)
    from oracle import oracle as O
    if args.workload != WORKLOAD and not _oracle_fits(cfg):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle's unreduced vertex of {cfg.name} exceeds 1 GB"}))
        return
    run, state = _oracle_sampler(cfg, 7)
    m = 256 if cfg.model.backend != "TRI" else 64
    for _ in range(args.warmup):
        run(m)
    tot, ent = 0.0, 0
    for _ in range(args.steps):
        e, dt = run(m)
        tot += dt
        ent += e
    val = ent / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg.name, "sample_entries_per_step": ent // args.steps, "lambda": 0.9},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": O.OracleFlow.threads(), "kind": "oracle",
                             "sample": f"{ent // args.steps} random stored entries per step of {cfg.name}, {state}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _measure_precision(sr, torch, cfg, lat, mesh, prec, steps, warmup, lams, flush, kgrid, sampler=None, sync=None):
    """Advance to mid-flow, warm up, then time `steps` Euler steps (+ chi) with CUDA events.
    From Lambda ~ 1 on, the steps follow a fine log grid (2000 steps per four decades), so any
    number of timed steps stays mid-flow."""
    fl = sr.Flow(lat, mesh, lams[0], prec)
    i = 0
    # untimed advance to mid-flow
    while lams[i] > 1.0:
        fl.step(lams[i + 1], sr.SR_EULER)
        i += 1
    n_adv = i
    ratio = (cfg.lam_min / cfg.lam_max) ** (1.0 / 2000)
    lams = [lams[i] * ratio ** k for k in range(warmup + steps + 1)]
    i = 0
    for _ in range(warmup):
        fl.step(lams[i + 1], sr.SR_EULER)
        fl.measure(kgrid, want_ij=False)
        i += 1
    stream = torch.cuda.current_stream()
    fl.profile_enable(True)
    ev = []
    if sync:
        sync()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    lam_start = lams[i]
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fl.step(lams[i + 1], sr.SR_EULER)
        fl.measure(kgrid, want_ij=False)
        b.record(stream)
        ev.append((a, b))
        i += 1
    torch.cuda.synchronize()
    if sync:
        sync()
    if sampler:
        sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    kms, kn = fl.profile_read()
    counts = fl.node_counts()
    fl.profile_enable(False)
    return fl, ms, kms, kn, counts, (lam_start, lams[i]), n_adv + i


def _full_flow(sr, torch, cfg, lat, mesh, prec, kgrid, method="euler", n_steps=200, n_out=50, budget_s=40.0):
    """The whole flow of the workload from Lambda = 100 to 0.01 with chi(k) on the k-grid at
    n_out log-spaced output cutoffs: Euler on n_steps log steps (the paper's scheme), or
    adaptive Dormand-Prince 5(4) (rtol 1e-6, atol 1e-10) stopped after budget_s seconds.
    Timed with CUDA events on the flow's stream."""
    fl = sr.Flow(lat, mesh, cfg.lam_max, prec)
    out_grid = W.lambda_list(cfg.lam_max, cfg.lam_min, n_out)
    if method == "euler":
        lams = W.lambda_list(cfg.lam_max, cfg.lam_min, n_steps)
        per_out = n_steps // n_out
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    a.record(stream)
    chimax = []
    reached = cfg.lam_max
    complete = True
    for k, lam in enumerate(out_grid[1:]):
        if method == "euler":
            try:
                for j in range(k * per_out, (k + 1) * per_out):
                    fl.step(float(lams[j + 1]), sr.SR_EULER)
                reached = float(lams[(k + 1) * per_out])
            except sr.SrError as e:   # the vertex overflowed (a flow breakdown): stop, no output
                if e.status != 5:
                    raise
                reached = fl.lam
                complete = False
                break
        else:
            fl.set_step_limit(500)
            try:
                reached = fl.step(float(lam), sr.SR_RK_ADAPTIVE, cfg.rtol, cfg.atol)
            except sr.SrError as e:
                if e.status != 6:
                    raise
                reached = fl.lam
                complete = False
        ck, _ = fl.measure(kgrid, want_ij=False)
        chimax.append(float(ck.max()))
        if not complete or time.perf_counter() - t0 > budget_s:
            complete = complete and reached <= cfg.lam_min * (1 + 1e-12)
            break
    b.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = fl.stats()
    ck, _ = fl.measure(kgrid, want_ij=False)
    fl.close()
    res = {"method": "Euler, %d log steps" % n_steps if method == "euler" else
           "adaptive Dormand-Prince 5(4), rtol %g, atol %g, normwise error" % (cfg.rtol, cfg.atol),
           "seconds": a.elapsed_time(b) * 1e-3, "wall_seconds": wall, "rhs_evaluations": st["n_rhs"],
           "accepted": st["n_accept"], "rejected": st["n_reject"], "lambda_reached": reached,
           "complete": bool(complete), "chi_max_final": chimax[-1] if chimax else None}
    return res, np.array(chimax), ck


def _batched_sweep(sr, torch, steps=20):
    """The batched coupling sweep: 64 seeded instances (square J1-J2 with J2/J1 ~ U[0,1] and
    range 5..9, kagome J1 with range 4..8, 32..64 frequencies), FP32-mixed, Euler steps on a
    common log cutoff list 50 -> 0.05 (100 steps).  The flows are advanced untimed to mid-flow
    by the batch itself, then `steps` Euler steps are timed (a) batched: all instances per step
    in one CUDA graph (replays timed, capture excluded), per size class the autotuner's choice of
    a persistent vertex kernel or the instances' own kernels, and (b) one flow after another with
    sr_flow_step, from the same saved states."""
    insts = W.batched_instances(0)
    lams = W.lambda_list(50.0, 0.05, 100)
    flows = []
    for c in insts:
        lat = sr.Lattice.from_model(c.model, c.L)
        mesh = sr.sr_frequency_mesh_exponential(c.n_freq, c.w_min, c.w_max)
        flows.append(sr.Flow(lat, mesh, lams[0], sr.SR_FP32_MIXED))
    n_ent = sum(f.n_gamma for f in flows)
    b = sr.Batch(flows)
    mid = 50
    b.run(lams[:mid + 1], use_graph=True, autotune=False)
    saved = [f.get_state() for f in flows]
    window = lams[mid:mid + steps + 1]
    b.run(window, use_graph=True, autotune=True)
    info = b.info()
    classes = b.classes()
    for c, per in zip(classes, b.class_launches()):
        c["launch"] = "per-instance kernels" if per else "persistent kernel"
    parallel = b.parallel_classes
    batched_ms = info["run_ms"]
    after_b = [f.get_state()[1] for f in flows]
    # each launch form on its own over the same window (the persistent form tuned for itself)
    forms = {}
    for mode, name in ((1, "persistent_kernels"), (2, "per_instance_kernels")):
        for f, (g, G) in zip(flows, saved):
            f.set_state(float(window[0]), g, G)
        b.force_launch(mode)
        b.run(window, use_graph=True, autotune=True)
        forms[name] = {"ms_per_step": b.info()["run_ms"] / steps, "parallel_classes": b.parallel_classes}
    b.force_launch(0)
    for f, (g, G) in zip(flows, saved):
        f.set_state(float(window[0]), g, G)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record()
    for f in flows:
        for lam in window[1:]:
            f.step(float(lam), sr.SR_EULER)
    e.record()
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(e)
    diff = max(float((f.get_state()[1] - Gb).abs().max() / Gb.abs().max()) for f, Gb in zip(flows, after_b))
    b.close()
    for f in flows:
        f.close()
    return {"workload": "64 seeded instances (48 square J1-J2, 16 kagome), FP32-mixed, Euler",
            "entries": n_ent, "steps_timed": steps, "lambda_window": [float(window[0]), float(window[-1])],
            "batched_ms_per_step": batched_ms / steps, "batched_entries_per_s": n_ent * steps / (batched_ms * 1e-3),
            "sequential_ms_per_step": seq_ms / steps, "sequential_entries_per_s": n_ent * steps / (seq_ms * 1e-3),
            "speedup": seq_ms / batched_ms, "size_classes": classes, "parallel_classes": parallel,
            "launch_forms": forms,
            "max_rel_diff_batched_vs_sequential": diff}


def _tensor_core_variant(sr, torch, fl):
    """The vertex kernel with the SU2 lattice sum on the tensor cores (3xTF32 tcgen05 MMAs) on
    the flow's current state, against the default CUDA-core kernel: kernel times (CUDA events,
    5 launches each after 2 warm-up launches) and the normwise difference of dGamma."""
    if fl.n_comp != 2:
        return None
    lam = fl.lam
    out = {}
    res = {}
    for tc in (False, True):
        fl.tensor_cores = tc
        for _ in range(2):
            fl.rhs(lam)
        torch.cuda.synchronize()
        fl.profile_enable(False)
        fl.profile_enable(True)
        for _ in range(5):
            _, dG = fl.rhs(lam)
        torch.cuda.synchronize()
        kms, kn = fl.profile_read()
        out["tensor_cores_ms" if tc else "cuda_cores_ms"] = float(kms[2] / max(kn[2], 1))
        res[tc] = dG.clone()
    fl.tensor_cores = False
    fl.profile_enable(False)
    out["rel_diff"] = float((res[True] - res[False]).abs().max() / res[False].abs().max())
    out["default"] = "cuda_cores"
    return out


def _gradient_timing(sr, torch, cfg, mesh):
    """d chi(k_max, Lambda_min) / d(J, K) of the Heisenberg-Kitaev flow (200 Euler steps): the
    reverse-mode adjoint with a checkpoint every 20 steps, the tangent-linear flow, and central
    finite differences (h = 1e-5) of the FP64 flow; wall times and the agreement."""
    import math
    from paper_2109_13317_gb300.autograd import susceptibility, susceptibility_adjoint
    cell, sites, B = W.honeycomb_kitaev_linear()
    theta0 = np.array([0.2, -1.0])
    lams = W.lambda_list(cfg.lam_max, cfg.lam_min, cfg.n_steps)
    kmax = np.array([[0.0, 4.0 * math.pi / 3.0, 0.0]])

    def grad(fn):
        th = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        chi = fn(th)
        (g,) = torch.autograd.grad(chi[0], th)
        torch.cuda.synchronize()
        return g.numpy(), time.perf_counter() - t0

    ga, ta = grad(lambda th: susceptibility_adjoint(th, cell, sites, B, cfg.L, mesh, lams, kmax, sr.SR_XYZ, every=20))
    gt, tt = grad(lambda th: susceptibility(th, cell, sites, B, cfg.L, mesh, lams, kmax, sr.SR_XYZ))

    def chi_at(theta):
        lat = sr.Lattice.from_model(W.linear_model(cell, sites, B, theta), cfg.L)
        fl = sr.Flow(lat, mesh, lams[0], sr.SR_FP64)
        for lam in lams[1:]:
            fl.step(float(lam), sr.SR_EULER)
        c, _ = fl.measure(kmax, want_ij=False)
        fl.close()
        return float(c[0])
    t0 = time.perf_counter()
    h = 1e-5
    gf = np.array([(chi_at(theta0 + h * e) - chi_at(theta0 - h * e)) / (2 * h) for e in np.eye(2)])
    tf = time.perf_counter() - t0
    return {"quantity": "d chi(k) / d(J, K) at k = (0, 4pi/3, 0), Lambda = 0.05, theta = (0.2, -1)",
            "adjoint": {"grad": ga.tolist(), "seconds": ta, "checkpoint_every": 20},
            "tangent": {"grad": gt.tolist(), "seconds": tt},
            "central_fd": {"grad": gf.tolist(), "seconds": tf, "h": h},
            "adjoint_vs_tangent_rel": float(np.abs(ga - gt).max() / np.abs(gt).max()),
            "adjoint_vs_fd_rel": float(np.abs(ga - gf).max() / np.abs(gf).max())}


def run_ours(args):
    import torch
    import paper_2109_13317_gb300 as sr
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    cfg = W.config(args.workload)
    headline = args.workload == WORKLOAD
    mesh = sr.sr_frequency_mesh_exponential(cfg.n_freq, cfg.w_min, cfg.w_max)
    lat = sr.Lattice.from_model(cfg.model, cfg.L)
    lams = W.lambda_list(cfg.lam_max, cfg.lam_min, cfg.n_steps)
    while len(lams) < 200:
        lams = W.lambda_list(cfg.lam_max, cfg.lam_min, 2 * (len(lams) - 1))
    kgrid = _kgrid(64)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2
    prec = sr.SR_FP64 if args.precision == "fp64" else sr.SR_FP32_MIXED
    sampler = ClockSampler(local) if rank == 0 else None

    # the timed steps are bracketed by a barrier over the ranks and a synchronize on both sides
    fl, ms, kms, kn, counts, lam_rng, i_end = _measure_precision(sr, torch, cfg, lat, mesh, prec, args.steps,
                                                                 args.warmup, lams, flush, kgrid, sampler,
                                                                 sync=lambda: _sync_all(torch, ws))
    t_step = _max_over_ranks(torch, sum(ms) / len(ms), ws)  # ms
    n_ent = fl.n_gamma
    value = _job_throughput(n_ent, ws, t_step)

    # roofline of the dominant kernel (vertex flow)
    flops = _algorithmic_flops(counts, fl.N, lat.N_s, fl.n_comp, lat.P, fl.lattice_sum_products())
    k_ms = kms[2] / max(kn[2], 1)
    achieved = flops / (k_ms * 1e-3) / 1e12
    peak_fp64_nominal = 1.25     # TFLOP/s, recipe table
    peak_fp32_units = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
    peak = peak_fp64_nominal if prec == sr.SR_FP64 else peak_fp32_units
    measured_peak = sr.sr_peak_fma(prec) / 1e12

    extra = {}
    if not args.no_fp32 and prec == sr.SR_FP64:
        fl2, ms2, kms2, kn2, counts2, _, _ = _measure_precision(sr, torch, cfg, lat, mesh, sr.SR_FP32_MIXED,
                                                                 args.steps, args.warmup, lams, flush, kgrid)
        # accuracy of the mixed flow after the same Euler steps: chi(k) and Gamma vs the FP64 flow
        assert abs(fl.lam - fl2.lam) <= 1e-12 * fl.lam
        ck64, _ = fl.measure(kgrid, want_ij=False)
        ck32, _ = fl2.measure(kgrid, want_ij=False)
        _, G64 = fl.get_state()
        _, G32 = fl2.get_state()
        flops2 = _algorithmic_flops(counts2, fl2.N, lat.N_s, fl2.n_comp, lat.P, fl2.lattice_sum_products())
        k2 = kms2[2] / max(kn2[2], 1)
        tcv = _tensor_core_variant(sr, torch, fl2)
        extra["fp32_mixed"] = {"value": n_ent * ws / (sum(ms2) / len(ms2) * 1e-3), "unit": UNIT,
                               "ms_per_step": sum(ms2) / len(ms2), "dtype": "f32-mixed",
                               "gamma_rhs_ms": k2,
                               "gamma_rhs_tflops": flops2 / (k2 * 1e-3) / 1e12,
                               "frac_of_fp32_peak": flops2 / (k2 * 1e-3) / 1e12 / (152 * 128 * 2 * 2.07e9 / 1e12),
                               "chi_rel_err_vs_fp64": float(np.abs(ck32 - ck64).max() / np.abs(ck64).max()),
                               "gamma_rel_err_vs_fp64": float((G32 - G64).abs().max() / G64.abs().max()),
                               "lambda": fl.lam,
                               "note": f"both flows integrated with the same {i_end} Euler steps from Lambda=100",
                               "tensor_core_lattice_sum": tcv}
        fl2.close()

    # end to end through the public API: state in from pinned host memory, step, state out
    g_h = torch.empty(fl.N, dtype=torch.float64).pin_memory()
    G_h = torch.empty(fl.n_gamma, dtype=torch.float64).pin_memory()
    g_d, G_d = fl.get_state()
    g_h.copy_(g_d)
    G_h.copy_(G_d)
    torch.cuda.synchronize()
    lam = fl.lam
    e2e_t = []
    for k in range(max(3, min(args.steps, 5))):
        t0 = time.perf_counter()
        g_dev = g_h.to("cuda", non_blocking=True)
        G_dev = G_h.to("cuda", non_blocking=True)
        fl.set_state(lam, g_dev, G_dev)
        fl.step(lam * 0.95, sr.SR_EULER)
        g_o, G_o = fl.get_state()
        G_h.copy_(G_o, non_blocking=True)
        g_h.copy_(g_o, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        lam = lam * 0.95
    e2e_val = n_ent * ws / statistics.median(e2e_t)
    bytes_state = 8 * (fl.N + fl.n_gamma)

    if not args.no_flow and prec == sr.SR_FP64:
        ff = {"lambda": [cfg.lam_max, cfg.lam_min], "outputs": 50}
        n_eu = 200 if cfg.method == "rk" else cfg.n_steps   # the configuration's Euler steps
        # Euler flows run to the end (their cost is fixed by the configuration's steps)
        e64, cm64, ck64 = _full_flow(sr, torch, cfg, lat, mesh, sr.SR_FP64, kgrid, "euler", n_steps=n_eu, budget_s=1e9)
        e32, cm32, ck32 = _full_flow(sr, torch, cfg, lat, mesh, sr.SR_FP32_MIXED, kgrid, "euler", n_steps=n_eu,
                                     budget_s=1e9)
        if e32["complete"] and e64["complete"]:
            e32["chi_rel_err_vs_fp64_final"] = float(np.abs(ck32 - ck64).max() / np.abs(ck64).max())
        n_cmp = min(len(cm32), len(cm64))   # outputs both flows reached
        e32["chi_max_rel_err_vs_fp64_all_outputs"] = float(np.abs(cm32[:n_cmp] - cm64[:n_cmp]).max() /
                                                           np.abs(cm64[:n_cmp]).max())
        e32["speedup_vs_fp64"] = e64["seconds"] / e32["seconds"]
        ff["euler"] = {"fp64": e64, "fp32_mixed": e32}
        if cfg.method == "rk":
            a64, cma, cka = _full_flow(sr, torch, cfg, lat, mesh, sr.SR_FP64, kgrid, "rk", budget_s=110.0)
            a32, _, _ = _full_flow(sr, torch, cfg, lat, mesh, sr.SR_FP32_MIXED, kgrid, "rk", budget_s=30.0)
            ff["adaptive"] = {"fp64": a64, "fp32_mixed": a32}
            # what the adaptive flow's accuracy buys: the Euler flows' distance from it (chi_max at
            # every output cutoff both reached, chi(k) at the end); Euler's error falls with the step
            e4, cm4, ck4 = _full_flow(sr, torch, cfg, lat, mesh, sr.SR_FP64, kgrid, "euler", n_steps=4 * n_eu,
                                      budget_s=1e9)
            acc = {"reference": "adaptive Dormand-Prince FP64 flow (rtol %g)" % cfg.rtol,
                   "euler_4x_steps_fp64_seconds": e4["seconds"]}
            for name, cm, ck in (("euler_fp64", cm64, ck64), ("euler_fp32_mixed", cm32, ck32),
                                 ("euler_4x_steps_fp64", cm4, ck4)):
                n_cmp = min(len(cm), len(cma))
                acc[name] = {"chi_max_rel_diff_all_outputs": float(np.abs(cm[:n_cmp] - cma[:n_cmp]).max() / np.abs(cma[:n_cmp]).max()),
                             "chi_k_rel_diff_final": float(np.abs(ck - cka).max() / np.abs(cka).max())
                             if a64["complete"] else None}
            ff["accuracy_vs_adaptive"] = acc
        extra["full_flow"] = ff
        if cfg.name == "honeycomb_hk_L5":
            extra["gradient"] = _gradient_timing(sr, torch, cfg, mesh)

    if not args.no_batch and rank == 0 and headline:
        extra["batched_sweep"] = _batched_sweep(sr, torch)

    clocks = sampler.summary() if sampler else None
    cpu = None
    if rank == 0 and not args.no_cpu and (headline or _oracle_fits(cfg)):
        try:
            cpu = _cpu_baseline(cfg)
        except Exception as e:  # the oracle is a baseline, never the product path
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {e}"}

    launches_per_step = 5 + 1 + (1 if prec == sr.SR_FP32_MIXED else 0)  # sigma, nodes, gamma, 2 axpy, chi (+1 shadow)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == sr.SR_FP64 else "f32-mixed", "data": "synthetic",
            "config": {"workload": cfg.name, **_describe(cfg), "range_L": cfg.L,
                       "N_s": lat.N_s, "N_tot": lat.N_tot, "P": lat.P, "lattice_sum_products": fl.lattice_sum_products(),
                       "n_freq": cfg.n_freq,
                       "freq_range": [cfg.w_min, cfg.w_max], "entries": n_ent,
                       "step": "Euler step (self-energy + vertex flow + update) + chi(k) on 64x64 k-grid",
                       "lambda_range_timed": [float(lam_rng[0]), float(lam_rng[1])],
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": {"bound": "alu", "kernel": "k_gamma_rhs_tri" if fl.n_comp == 16 else "k_gamma_rhs",
                         "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "peak_source": "FP64 nominal 1.25 TFLOP/s (recipe table)" if prec == sr.SR_FP64 else
                         "FP32 from unit counts: 152 SMs x 128 lanes x 2 flop x 2.07 GHz",
                         "peak_measured_fma": measured_peak, "frac_of_measured_fma": achieved / measured_peak,
                         "algorithmic_flop_per_launch": flops, "launch_ms": k_ms,
                         "traffic": _traffic(args.precision) if headline else None},
            "kernels_ms_per_step": {"sigma_rhs": kms[0] / max(kn[0], 1), "channel_nodes": kms[1] / max(kn[1], 1),
                                    "gamma_rhs": k_ms},
            "clocks": clocks,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": bytes_state,
                    "d2h_bytes_per_step": bytes_state},
            "gpu_launches": launches_per_step * args.steps,
            "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    fl.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def profile_rhs(args):
    """One right-hand side of the workload, for profiler captures of the vertex kernels: the
    flow (optionally with another number of frequencies) takes two Euler steps (two
    vertex-kernel launches) and evaluates one right-hand side (the third launch), so that a
    capture skips two launches of the vertex kernel and takes one.  The right-hand side is at
    --profile-lambda (default 0.1 Lambda_max), the steps at 4 and 1.6 times that cutoff (the
    work per launch depends on the cutoff through the integration nodes, not on the state)."""
    import torch
    import paper_2109_13317_gb300 as sr
    cfg = W.config(args.workload)
    n = args.n_freq or cfg.n_freq
    lat = sr.Lattice.from_model(cfg.model, cfg.L)
    mesh = sr.sr_frequency_mesh_exponential(n, cfg.w_min, cfg.w_max)
    prec = sr.SR_FP64 if args.precision == "fp64" else sr.SR_FP32_MIXED
    lam = args.profile_lambda or 0.1 * cfg.lam_max
    fl = sr.Flow(lat, mesh, 10.0 * lam, prec)
    fl.step(4.0 * lam, sr.SR_EULER)
    fl.step(1.6 * lam, sr.SR_EULER)
    fl.rhs(lam)
    torch.cuda.synchronize()
    print(f"{cfg.name}: N_s={lat.N_s} P={lat.P} n_freq={n} entries={fl.n_gamma} precision={args.precision} "
          f"Lambda={lam}")
    fl.close()


def oracle_flow(args):
    """The CPU oracle's own Euler flow of the workload on all host cores (the configuration's
    log-spaced cutoff steps from Lambda_max to Lambda_min, chi(k) on the 64 x 64 grid at the
    end): whole-flow seconds when it fits the budget, else the seconds per step of the steps
    taken and the whole flow extrapolated from them (stated in the line)."""
    from oracle import oracle as O
    cfg = W.config(args.workload)
    mesh = O.mesh_exponential(cfg.n_freq, cfg.w_min, cfg.w_max)
    tri = cfg.model.backend == "TRI"
    of = (O.OracleFlowTRI if tri else O.OracleFlow)(cfg.model, cfg.L, mesh)
    n_steps = cfg.n_steps if cfg.method == "euler" else 200
    lams = W.lambda_list(cfg.lam_max, cfg.lam_min, n_steps)
    t0 = time.perf_counter()
    done = 0
    for a, b in zip(lams[:-1], lams[1:]):
        of.euler(float(a), float(b))
        done += 1
        if time.perf_counter() - t0 > args.oracle_budget:
            break
    dt = time.perf_counter() - t0
    line = {"impl": "oracle", "workload": cfg.name, "metric": "full Lambda-flow time", "unit": "s",
            "method": f"Euler, {n_steps} log steps {cfg.lam_max} -> {cfg.lam_min}", "cores": O.OracleFlow.threads(),
            "steps_done": done, "seconds": dt, "seconds_per_step": dt / done,
            "complete": done == n_steps, "full_flow_seconds": dt if done == n_steps else dt / done * n_steps,
            "full_flow_seconds_kind": "measured" if done == n_steps else "extrapolated from the steps done",
            "entries": int(of.size)}
    if done == n_steps:
        line["chi_max_final"] = float(np.max(of.chi_k(float(lams[-1]), _kgrid(64))))
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    if args.oracle_flow:
        oracle_flow(args)
    elif args.profile_rhs:
        profile_rhs(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
