"""Benchmark of the projection solve on GB300: prints ONE JSON line (rank 0).

Workload (default): 3-D 256^3 plane-parallel stratified atmosphere (density
contrast 1e3, Gaussian random velocity sigma_U = 1e-2, Gaussian heating blob of
amplitude 1 and width 0.1), MIXED precision.  One step is one pass of the whole
hot path over one input: coefficient setup on every level (step a1), the MAC
projection and the nodal projection (steps a2-a10) to relative residual 1e-10.
A step therefore holds two projection solves; the metric counts both.  The
velocity inputs are restored from a resident copy at the start of every step
(device-to-device copies inside the timed region: a projected field would
otherwise be projected again).

Timing: W untimed warm-up steps, then exactly K steps bracketed by a barrier and
a device synchronisation, timed with CUDA events on the solver stream; every
input array (134 MB in FP64 at 256^3) is larger than the 129 MB L2, so no L2
flush is needed between steps.  Under torchrun every rank solves its own copy of
the workload (independent solves: weak scaling, no collective on the data path)
and rank 0 reports the whole-job throughput over the slowest rank's time.

--impl reference times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import math
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "projection solves/s (MAC + nodal per step), mixed precision, rel. residual 1e-10"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cells per axis of the stratified workload")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="stratified", choices=["stratified", "batch", "serve", "config1", "config2", "step"],
                    help="stratified: the default 256^3 MAC + nodal mixed step; batch: 64 uneven MAC solves in "
                         "one graph launch; serve: Poisson stream of polytrope-star projections (p50/p99); "
                         "config1: 2-D 64^2 manufactured solve; config2: 128^3 FP64 MAC + nodal step; "
                         "step: the time step around the two projections (face velocities, MAC projection, "
                         "advection with rotation, nodal projection), mixed, on the stratified workload")
    ap.add_argument("--batch-branches", action="store_true",
                    help="batch: run every solve as its own graph branch instead of the shared batched loop")
    ap.add_argument("--parity", action="store_true",
                    help="also solve the MAC system of the workload with the CPU oracle and report rel-L2 of phi")
    ap.add_argument("--budget-gb", type=float, default=24.0, help="serve: device-memory budget of the slots")
    ap.add_argument("--inflight", type=int, default=8, help="serve: concurrent solves")
    ap.add_argument("--serve-count", type=int, default=256, help="serve: requests per arrival rate")
    ap.add_argument("--sweep", default="v4", choices=["v4", "pipe", "tma", "legs"],
                    help="FP32 cell smoother: two vectorised colour passes (v4), the pipelined one-launch "
                         "sweep (pipe, MG_FLAG_SWEEP_PIPE), the TMA-staged one-pass sweep (tma, MG_FLAG_SWEEP_TMA) "
                         "or whole V-cycle legs of the finest level as one L2-pipelined launch each (legs, "
                         "MG_FLAG_CELL_PIPE)")
    ap.add_argument("--inner-mac", type=int, default=0,
                    help="FP32 V-cycles per FP64 refinement step of the MAC solve (0: the library's choice)")
    ap.add_argument("--nu", default="2,1",
                    help="pre,post smoothing sweeps of the MAC V-cycle (nodal: --nu-nodal)")
    ap.add_argument("--nu-nodal", default="2,2", help="pre,post smoothing sweeps of the nodal V-cycle")
    ap.add_argument("--omega-nodal", type=float, default=0.9, help="damping of the nodal Jacobi smoother")
    ap.add_argument("--autotune", action="store_true",
                    help="time the smoother kernels of both hierarchies at setup (MG_FLAG_AUTOTUNE) and report "
                         "the choices")
    ap.add_argument("--inner-nodal", type=int, default=0,
                    help="FP32 V-cycles per FP64 refinement step of the nodal solve (0: the library's choice)")
    ap.add_argument("--coarsest", type=int, default=0,
                    help="largest coarsest-level size handed to the dense solve (0: the library's default)")
    ap.add_argument("--only-mixed", action="store_true",
                    help="time only the mixed-precision step (no graph-path, FP64, e2e or CPU legs): the "
                         "command used for ncu captures")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1948.1), "measured"
    return 6800.0, 1900.0, "fallback"


def fp64_peak_measured(dev, index):
    """FP64 FMA throughput of this GPU, measured: independent FMA chains in
    every thread, four 256-thread blocks per SM, CUDA events on the launching
    stream, median of seven launches after two warm-ups, with the SM clock
    sampled meanwhile.  Returns (TFLOP/s, clocks record)."""
    import torch
    from paper_1910_12979_gb300 import native as N
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.Stream(device=dev)
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    iters = 4096
    for _ in range(2):
        N.mg_fp64_fma_probe(4 * sms, iters, sink.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    ck = Clocks(index)
    ck.start()
    rates = []
    for _ in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = N.mg_fp64_fma_probe(4 * sms, iters, sink.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        rates.append(fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return statistics.median(rates), ck.stop()


def workload_config(n, tol):
    return {"workload": f"stratified atmosphere {n}^3, MAC + nodal projection, mixed precision",
            "grid": [n, n, n], "density_contrast": 1e3, "u_sigma": 1e-2, "blob_width": 0.1,
            "bc": "periodic x,y; slip wall z=0; outflow (phi=0) z=1", "tol": tol, "solves_per_step": 2,
            "precision": "FP32 V-cycles in FP64 iterative refinement; FP64 residual, update, bottom solve",
            "l2": "inputs larger than L2 (each FP64 field 134 MB > 129 MB L2); no flush",
            "seed": 3}


# --------------------------------------------------------------------- oracle

def oracle_sample(n_sample, seed=3):
    """Time the oracle's MAC + nodal projection on an n_sample^3 instance of the
    same recipe; returns (seconds, relres list)."""
    import inputs as I
    import oracle as O
    O.build()
    p = I.stratified(n_sample, seed=seed, contrast=1e3)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
    t0 = time.perf_counter()
    a = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-10)
    b = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=1e-10)
    return time.perf_counter() - t0, [a["relres"], b["relres"]]


def oracle_cpu_leg(n_full, n_small=48, n_large=128, seed=3, tol=1e-10):
    """The FP64 oracle timed on this host, one thread: a full MAC + nodal
    projection of the stratified recipe at n_small^3 and at n_large^3, each to
    the workload's tolerance.  The n_large^3 time is the baseline (scaled to
    n_full^3 by the cell count); the two per-cell times check that the work is
    linear in the cells.  The n_large^3 solutions are then carried on, untimed,
    to the oracle's round-off floor and returned as the reference for the GPU's
    error at that size."""
    import inputs as I
    import oracle as O
    O.build()
    times, ref = {}, None
    for n in (n_small, n_large):
        p = I.stratified(n, seed=seed, contrast=1e3)
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        t0 = time.perf_counter()
        a = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=tol)
        b = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=tol)
        times[n] = time.perf_counter() - t0
        if n == n_large:
            fm = O.mac_rhs(g, p["beta0"], p["beta0_face"], p["U_mac"], p["S"])
            phm, _ = O.mac_solve_mg(g, O.mac_faces(g, p["sigma"]), fm, tol=1e-13, phi0=a["phi"])
            fn = O.nodal_rhs(g, p["beta0"], p["U_cell"], p["S"])
            phn, _ = O.nodal_solve_mg(g, p["sigma"], fn, tol=1e-13, phi0=b["phi"])
            ref = {"p": p, "g": g, "mac_phi": phm, "nodal_phi": phn, "live": ~g.dirichlet_node_mask()}
    # the all-core build of the oracle (colour-ordered smoothers, OpenMP loops): its result must
    # not depend on the thread count (checked at n_small^3), then it is timed at n_large^3
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    par = None
    try:
        p = I.stratified(n_small, seed=seed, contrast=1e3)
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        outs = []
        for th in (1, cores):
            with O.all_cores(th):
                a = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=tol)
                b = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=tol)
            outs.append((a["phi"], b["phi"]))
        same = bool(all((x == y).all() for x, y in zip(outs[0], outs[1])))
        p = I.stratified(n_large, seed=seed, contrast=1e3)
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        with O.all_cores(cores):
            t0 = time.perf_counter()
            O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=tol)
            O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=tol)
            tp = time.perf_counter() - t0
        par = {"value": 2.0 / (tp * (n_full / n_large) ** 3), "unit": UNIT, "cores": cores,
               "kind": "oracle, all cores (colour-ordered Gauss-Seidel, OpenMP)",
               "sample": f"one MAC + nodal projection at {n_large}^3 ({tp:.1f} s, measured) scaled by "
                         f"{(n_full / n_large) ** 3:.0f} to {n_full}^3",
               "bitwise_equal_1_vs_all_threads": same}
    except Exception as e:  # no OpenMP toolchain on this host: report why
        par = {"unavailable": repr(e)[:200]}
    scale = (n_full / n_large) ** 3
    per_cell = {n: times[n] / n ** 3 for n in times}
    base = {"value": 2.0 / (times[n_large] * scale), "unit": UNIT, "cores": 1, "kind": "oracle",
            "all_cores": par,
            "sample": f"one full MAC + nodal oracle projection of the same recipe at {n_large}^3 "
                      f"({times[n_large]:.1f} s, measured) scaled by the cell-count ratio {scale:.0f} to "
                      f"{n_full}^3; at {n_small}^3 it took {times[n_small]:.2f} s: "
                      f"{1e6 * per_cell[n_small]:.2f} vs {1e6 * per_cell[n_large]:.2f} us per cell "
                      f"(ratio {per_cell[n_large] / per_cell[n_small]:.2f}), so the scaling is checked, not assumed",
            "measured_s": {f"{n}^3": times[n] for n in times}}
    return base, ref


def gpu_error_vs_oracle(ref, dev, tol):
    """The GPU's mixed MAC and nodal projections of the oracle's reference
    problem, in the benchmark's solver configuration, against the oracle's
    solutions: rel-L2 of phi (nodal: over the unknown nodes)."""
    import numpy as np
    import torch
    from paper_1910_12979_gb300 import ProjectionSolver
    from paper_1910_12979_gb300 import native as N
    p = ref["p"]
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    mac = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed", flags=N.MG_FLAG_ZERO_GUESS,
                           nu1=2, nu2=1)
    nod = ProjectionSolver(p["geom"], T(p["sigma"]), loc="nodal", prec="mixed", flags=N.MG_FLAG_ZERO_GUESS)
    phim = torch.zeros(mac.vec_shape, dtype=torch.float64, device=dev)
    phin = torch.zeros(nod.vec_shape, dtype=torch.float64, device=dev)
    mac.project([T(u) for u in p["U_mac"]], T(p["beta0"]), T(p["S"]), beta0_face=[T(b) for b in p["beta0_face"]],
                phi=phim, tol=tol, allow_not_converged=True)
    nod.project([T(u) for u in p["U_cell"]], T(p["beta0"]), T(p["S"]), phi=phin, tol=tol, allow_not_converged=True)
    pm, pn = phim.cpu().numpy(), phin.cpu().numpy()
    mac.close()
    nod.close()
    live = ref["live"]
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"grid": f"{p['geom']['n'][0]}^3 (the benchmark's recipe and solver settings at the size the oracle "
                    f"solves within the run; the GPU to the workload's tol {tol:g}, the oracle to its floor)",
            "mac_phi_rel_l2_vs_oracle": rel(pm, ref["mac_phi"]),
            "nodal_phi_rel_l2_vs_oracle": rel(pn[live], ref["nodal_phi"][live]), "bound": 1e-8}


def run_reference(args, rank):
    """The reference arm: the FP64 oracle, as it stands, on this host's cores.
    Each step is one MAC + nodal oracle projection of a 32^3 instance of the
    same recipe (a bounded sample of the 256^3 workload: 1/512 of its cells).
    ms_per_step is the measured time of such a step, so steps x ms_per_step is
    the time this run spent; value is the throughput on the workload's size,
    the sample's time scaled by the cell-count ratio (multigrid work is linear
    in the cells at a fixed iteration count -- the default GPU line's
    cpu_baseline checks that with a 48^3 and a 128^3 run)."""
    if rank != 0:
        return
    n_sample = 32
    for _ in range(args.warmup):
        oracle_sample(n_sample)
    times = []
    for _ in range(args.steps):
        dt, _ = oracle_sample(n_sample)
        times.append(dt)
    scale = (args.n / n_sample) ** 3
    total = sum(times) * scale
    value = 2.0 * args.steps / total
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "ms_per_step_at_workload_size": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.n, args.tol),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "host_cores_available": cores,
                             "sample": f"each step: one MAC + nodal oracle projection at {n_sample}^3 of the same "
                                       f"recipe (measured: ms_per_step), scaled by the cell-count ratio "
                                       f"{scale:.0f} to {args.n}^3 for value"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# the source files whose change invalidates a kernel class's ncu counters
PROF_SOURCES = {"cell_smooth_fine": ["mg_gsrb_tma.cu", "mg_gsrb4.cu", "mg_sweep.cu", "mg_cell.cu"],
                "node_smooth_fine": ["mg_nodal4.cu", "mg_nodal.cu", "mg_nodal.cuh"],
                "cell_restrict_fine": ["mg_gsrb4.cu", "mg_cell.cu"], "cell_resid64": ["mg_cell.cu"],
                "node_resid64": ["mg_nodal.cu", "mg_nodal.cuh"]}


def source_hash(kernel_class):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1910_12979_gb300", "csrc")
    for f in sorted(PROF_SOURCES.get(kernel_class, []) + ["mg_device.cuh", "mg_internal.cuh"]):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(kernel_class)
    if not e or e.get("source_hash") != source_hash(kernel_class):
        return None
    return e.get("bytes_per_launch")


def run_batch(args, dev, world, dist):
    """64 independent MAC solves of uneven size (32-128^3), one graph launch per step."""
    import numpy as np
    import torch

    import inputs as I
    from paper_1910_12979_gb300 import ProjectionSolver, solve_batch
    from paper_1910_12979_gb300 import native as N

    specs = I.batch_specs(64, seed=4)
    stream = torch.cuda.Stream(device=dev)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    solvers, rhs, phis, cells = [], [], [], 0
    with torch.cuda.stream(stream):
        for sp in specs:
            p = I.batch_problem(sp)
            s = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed", stream=stream,
                                 flags=N.MG_FLAG_AUTOTUNE | N.MG_FLAG_ZERO_GUESS |
                                 (N.MG_FLAG_BATCH_BRANCHES if args.batch_branches else 0))
            f = s.rhs([T(u) for u in p["U_mac"]], T(p["beta0"]), T(p["S"]), beta0_face=[T(b) for b in p["beta0_face"]])
            solvers.append(s)
            rhs.append(f)
            phis.append(torch.zeros_like(f))
            cells += sp["n"] ** 3
    stream.synchronize()
    tols = [args.tol] * len(solvers)
    kind_names = {0: "default", 1: "4-cell passes, 8 quads/row", 2: "4-cell passes, 16 quads/row",
                  3: "4-cell passes, 32 quads/row", 4: "pipelined one-launch sweep",
                  5: "4-node passes, 8 quads/row, 4 planes/thread", 6: "4-node passes, 16 quads/row, 4 planes/thread",
                  7: "4-node passes, 32 quads/row, 4 planes/thread", 8: "TMA-staged one-pass sweep"}
    tuned = {}
    for sp, s in zip(specs, solvers):
        tuned.setdefault(f"{sp['n']}^3", [kind_names.get(N.mg_smoother_kind(s.handle, l), "?")
                                          for l in range(8) if N.mg_smoother_kind(s.handle, l) >= 0])

    def step():
        with torch.cuda.stream(stream):
            for ph in phis:
                ph.zero_()
        return solve_batch(solvers, rhs, phis, tols, allow_not_converged=True)

    for _ in range(args.warmup):
        st = step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    l0 = N.mg_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st = step()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    launches = N.mg_launch_count() - l0
    # the same solves one after another (one graph launch and one sync per solve)
    t_seq = 0.0
    for s, f, ph in zip(solvers, rhs, phis):
        ph.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            s.solve(f, ph, tol=args.tol, allow_not_converged=True)
        b.record(stream)
        b.synchronize()
        t_seq += a.elapsed_time(b)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = len(solvers) * args.steps * world / (ms / 1e3)
    errs = None
    if not args.no_cpu:
        # three entries (the first 32^3, 96^3 and 128^3 of the batch) against oracle solves of their systems;
        # the solves of the last timed launch are re-run to leave their phi in place
        import oracle as O
        st = step()
        errs = {"quantity": f"rel-L2 of phi, GPU at tol {args.tol:g} (batch launch), oracle to its floor"}
        for n in (32, 96, 128):
            i = next(k for k, sp in enumerate(specs) if sp["n"] == n)
            p = I.batch_problem(specs[i])
            g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
            fo = O.mac_rhs(g, p["beta0"], p["beta0_face"], p["U_mac"], p["S"])
            ref, _ = O.mac_solve_mg(g, O.mac_faces(g, p["sigma"]), fo, tol=1e-13)
            ph = phis[i].cpu().numpy()
            errs[f"entry {i} ({n}^3)"] = float(np.linalg.norm(ph - ref) / np.linalg.norm(ref))
    return {"metric": "independent projection solves/s, uneven batch in one graph launch", "value": value,
            "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": "batch of 64 MAC solves, n in {32,64,96,128} (seed 4), contrast log-uniform "
                                   "in [1e1,1e4], one graph launch per step", "cells": cells, "tol": args.tol,
                       "loop": ("per-solve graph branches" if args.batch_branches else
                                "the solves of at most 64^3 cells (32 of 64) in one batched loop -- each step of all "
                                "of them one launch driven by per-solve work items -- the larger ones as concurrent "
                                "graph branches"),
                       "rhs": "each solve's right-hand side formed before the timed region (mg_rhs); the timed "
                              "step is the 64 solves",
                       "l2": "aggregate inputs larger than L2",
                       "autotuned_smoother_per_level": tuned},
            "gpu_launches": launches,
            "iters": {"min": min(x["iters"] for x in st), "max": max(x["iters"] for x in st)},
            "worst_rel_resid": max(x["rel_resid"] for x in st),
            "sequential": {"value": len(solvers) / (t_seq / 1e3), "unit": "solves/s",
                           "note": "the same 64 solves issued one mg_solve at a time"},
            "rel_l2_vs_oracle": errs,
            "small_batch": small_batch_compare(dev, stream, args.tol)}


def small_batch_compare(dev, stream, tol, n=32, count=64):
    """count solves of n^3 (the batch recipe at one size): the batched loop
    against per-solve graph branches, CUDA events over 5 launches after 3."""
    import numpy as np
    import torch

    import inputs as I
    from paper_1910_12979_gb300 import ProjectionSolver, solve_batch
    from paper_1910_12979_gb300 import native as N

    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    specs = I.batch_specs(count, seed=4, sizes=(n,))
    out = {"workload": f"{count} MAC solves of {n}^3 (batch recipe, seed 4)", "unit": "solves/s"}
    for name, extra in (("batched_loop", 0), ("graph_branches", N.MG_FLAG_BATCH_BRANCHES)):
        solvers, rhs = [], []
        with torch.cuda.stream(stream):
            for sp in specs:
                p = I.batch_problem(sp)
                s = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec="mixed", stream=stream,
                                     flags=N.MG_FLAG_ZERO_GUESS | extra)
                rhs.append(s.rhs([T(u) for u in p["U_mac"]], T(p["beta0"]), T(p["S"]),
                                 beta0_face=[T(b) for b in p["beta0_face"]]))
                solvers.append(s)
        phis = [torch.zeros_like(f) for f in rhs]
        for _ in range(3):
            solve_batch(solvers, rhs, phis, [tol] * count, allow_not_converged=True)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = N.mg_launch_count()
        e0.record(stream)
        for _ in range(5):
            solve_batch(solvers, rhs, phis, [tol] * count, allow_not_converged=True)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 5
        out[name] = {"value": count / (ms / 1e3), "ms_per_batch": ms, "gpu_launches_per_batch": (N.mg_launch_count() - l0) / 5}
        for s in solvers:
            s.close()
    return out


def run_serve(args, dev, rank, world, dist):
    """Poisson stream of polytrope-star MAC projections, sizes 64..256^3."""
    import numpy as np
    import torch

    import inputs as I
    from paper_1910_12979_gb300 import native as N
    from paper_1910_12979_gb300.serve import GpuBackend, Scheduler, host_problem, latency_stats, make_requests, shard

    sizes = (64, 96, 128, 192, 256)
    per_size = 3   # distinct problems per size, in pinned host memory; requests cycle through them
    raw = {n: [I.polytrope_star(n, seed=500 + n + k) for k in range(per_size)] for n in sizes}
    problems = {n: [host_problem(p) for p in raw[n]] for n in sizes}
    budget = int(args.budget_gb * 2 ** 30)
    l0 = N.mg_launch_count()

    # one serving process: the scheduler and its resident slots (hierarchies, captured graphs) persist
    # from the warm-up through the saturation and the arrival-rate streams
    sch = Scheduler(GpuBackend(problems, device=str(dev), tol=args.tol), budget, max_inflight=args.inflight)

    def serve(reqs):
        done = sch.run_stream(reqs, timeout=900)
        return done, sch.evictions, list(sch.batches)

    rng = np.random.default_rng(5)
    # saturation: every request present at t = 0
    sat_n = args.serve_count // 4
    ns = [int(x) for x in rng.choice(sizes, size=sat_n)]
    # warm-up: the slots of every size, as many as can be in flight, and their graphs
    serve(make_requests([0.0] * (len(sizes) * args.inflight), [n for n in sizes for _ in range(args.inflight)],
                        per_size))
    serve(make_requests([0.0] * sat_n, ns, per_size))   # and the saturation stream once, untimed
    n_warm = len(sizes) * args.inflight + sat_n
    done, _, _ = serve(shard(make_requests([0.0] * sat_n, ns, per_size), rank, world))
    mu = latency_stats(done)["solves_per_s"]
    rates = {}
    for frac in (0.5, 0.8, 0.95):
        t, ns2 = I.poisson_arrivals(frac * mu * world, args.serve_count, seed=5, sizes=sizes)
        reqs = shard(make_requests(t, ns2, per_size, seed=5), rank, world)
        done, ev, batches = serve(reqs)
        bad = sum(isinstance(r.status, Exception) for r in done)
        rates[str(frac)] = dict(latency_stats(done), evictions=ev, failed=bad,
                                batched_requests=sum(b for b in batches if b > 1), mean_batch=float(np.mean(batches)))
    slots = {str(n): sum(1 for s_ in sch.slots if s_.n == n) for n in sizes}
    sch.close()
    launches = N.mg_launch_count() - l0
    head = rates["0.8"]
    out = {"metric": "serving: projection solves/s and p50/p99 latency at 0.8 x saturation", "value":
           head["solves_per_s"] * world, "unit": "solves/s", "n_gpus": world, "steps": args.serve_count,
           "warmup": n_warm, "ms_per_step": 1e3 / head["solves_per_s"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
           "config": {"workload": "Poisson arrivals of polytrope (n=3) star MAC projections, Dirichlet, "
                                  "sizes {64,96,128,192,256}^3 (seed 5)", "budget_gb": args.budget_gb,
                      "max_inflight": args.inflight, "tol": args.tol,
                      "slots": "one scheduler for the warm-up, saturation and rate streams: hierarchies and their "
                               "captured graphs stay resident between requests (resident slots per size at the "
                               f"end: {slots})",
                      "io": f"every request uploads its problem (sigma, beta0 at cells and faces, S, U) from pinned "
                            f"host memory and reads the projected U back: latency includes both; {per_size} "
                            f"distinct problems per size", "batching": "requests admitted together run as one "
                                                                     "mg_project_batch (solves in one graph launch)"},
           "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "saturation_solves_per_s": mu * world,
           "rates": rates, "gpu_launches": launches}
    if rank == 0 and not args.no_cpu:
        out["rel_l2_vs_oracle"] = served_error_vs_oracle(raw, dev, args.tol)
    return out


def served_error_vs_oracle(raw, dev, tol):
    """Two served requests (64^3 and 128^3 polytrope stars) through the serving
    backend, their projected velocities against oracle projections."""
    import numpy as np
    import oracle as O
    from paper_1910_12979_gb300.serve import GpuBackend, Request, Scheduler, host_problem
    out = {}
    for n in (64, 128):
        p = raw[n][0]
        sch = Scheduler(GpuBackend({n: [host_problem(p)]}, device=str(dev), tol=tol), 8 * 2 ** 30, max_inflight=1)
        r = sch.run_stream([Request(0, n, 0.0, (n, 0), keep=True)], timeout=600)[0]
        sch.close()
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        ref = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-13)
        num = math.sqrt(sum(float(np.sum((u.numpy() - v) ** 2)) for u, v in zip(r.result, ref["U"])))
        den = math.sqrt(sum(float(np.sum(v ** 2)) for v in ref["U"]))
        out[f"{n}^3"] = num / den
    out["quantity"] = f"rel-L2 of the projected face velocity, GPU at tol {tol:g}, oracle to its floor"
    return out


def _timed_solves(fn, K, W, stream):
    import torch
    for _ in range(W):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def run_config1(args, dev):
    """2-D 64^2 manufactured solve, FP64 and mixed, against the oracle and the exact phi."""
    import numpy as np
    import torch

    import inputs as I
    import oracle as O
    from paper_1910_12979_gb300 import ProjectionSolver
    from paper_1910_12979_gb300 import native as N

    p = I.manufactured_2d(64)
    g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
    ref, _ = O.mac_solve_mg(g, O.mac_faces(g, p["sigma"]), p["f"])
    ref = ref - ref.mean()
    stream = torch.cuda.Stream(device=dev)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    res = {}
    for prec in ("fp64", "mixed"):
        with torch.cuda.stream(stream):
            s = ProjectionSolver(p["geom"], T(p["sigma"]), loc="cell", prec=prec, stream=stream,
                                 flags=N.MG_FLAG_ZERO_GUESS)
            f = T(p["f"])
            phi = torch.zeros_like(f)

        def solve():
            with torch.cuda.stream(stream):
                phi.zero_()
                return s.solve(f, phi, tol=1e-12)
        ms, st = _timed_solves(solve, args.steps, args.warmup, stream)
        ph = phi.cpu().numpy()
        ph = ph - ph.mean()
        ex = p["phi_exact"] - p["phi_exact"].mean()
        res[prec] = {"solves_per_s": args.steps / (ms / 1e3), "iters": st["iters"], "rel_resid": st["rel_resid"],
                     "rel_l2_vs_oracle": float(np.linalg.norm(ph - ref) / np.linalg.norm(ref)),
                     "rms_error_vs_exact_phi": float(np.sqrt(np.mean((ph - ex) ** 2)))}
    return {"metric": "2-D 64^2 manufactured MAC-type solve, solves/s", "value": res["fp64"]["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / res["fp64"]["solves_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "2-D 64x64 stratified rho = exp(-y/0.25), beta0 = rho^(3/5), manufactured "
                                   "phi = cos(2 pi x) cos(2 pi y); periodic x, Neumann y; tol 1e-12"},
            "fp64": res["fp64"], "mixed": res["mixed"]}


def run_step(args, dev, world, dist):
    """Time steps around the two projections (mg_step) on the stratified workload, mixed precision."""
    import numpy as np
    import torch

    import inputs as I
    from paper_1910_12979_gb300 import ProjectionSolver
    from paper_1910_12979_gb300 import native as N
    from paper_1910_12979_gb300.solver import time_step

    n = args.n
    p = I.stratified(n, seed=3, contrast=1e3, mac=False)
    stream = torch.cuda.Stream(device=dev)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with torch.cuda.stream(stream):
        sigma, beta0, S = T(p["sigma"]), T(p["beta0"]), T(p["S"])
        b0f = [T(b) for b in p["beta0_face"]]
        U0 = [T(u) for u in p["U_cell"]]
        fl = N.MG_FLAG_ZERO_GUESS
        mac = ProjectionSolver(p["geom"], sigma, loc="cell", prec="mixed", stream=stream, flags=fl)
        nod = ProjectionSolver(p["geom"], sigma, loc="nodal", prec="mixed", stream=stream, flags=fl)
        Un = [torch.empty_like(u) for u in U0]
        Ua = [torch.empty(mac.face_shape(d), dtype=torch.float64, device=dev) for d in range(3)]
    stream.synchronize()
    dt, omega, centre = 0.01, (0.0, 0.0, 2.0), (0.5, 0.5, 0.5)

    def step():
        with torch.cuda.stream(stream):
            mac.update_coeff(sigma)
            nod.update_coeff(sigma)
            return time_step(mac, nod, U0, Un, Ua, beta0, b0f, S, dt, omega=omega, center=centre, centrifugal=True,
                             tol=args.tol, allow_not_converged=True)

    for _ in range(args.warmup):
        st = step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    l0 = N.mg_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st = step()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    launches = N.mg_launch_count() - l0
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return {"metric": "time steps/s around the two projections", "value": args.steps * world / (ms / 1e3),
            "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": f"stratified atmosphere {n}^3: face velocities, MAC projection, upwind advection "
                                   f"with Coriolis and centrifugal terms (Omega = {omega}), nodal projection",
                       "dt": dt, "tol": args.tol, "coefficient_update_per_step": True},
            "gpu_launches": launches,
            "solver": {"mac": {k: st[0][k] for k in ("iters", "rel_resid", "rel_constraint")},
                       "nodal": {k: st[1][k] for k in ("iters", "rel_resid", "rel_constraint")}}}


def run_config2(args, dev):
    """128^3 stratified MAC + nodal step in FP64 (and the MAC rel-L2 against the oracle)."""
    import numpy as np
    import torch

    import inputs as I
    from paper_1910_12979_gb300 import ProjectionSolver
    from paper_1910_12979_gb300 import native as N

    p = I.stratified(128, seed=2, contrast=1e3)
    stream = torch.cuda.Stream(device=dev)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with torch.cuda.stream(stream):
        sigma, beta0, S = T(p["sigma"]), T(p["beta0"]), T(p["S"])
        b0f = [T(b) for b in p["beta0_face"]]
        U0m, U0c = [T(u) for u in p["U_mac"]], [T(u) for u in p["U_cell"]]
        Um, Uc = [u.clone() for u in U0m], [u.clone() for u in U0c]
        out = {}
        for prec in ("fp64", "mixed"):
            mac = ProjectionSolver(p["geom"], sigma, loc="cell", prec=prec, stream=stream, flags=N.MG_FLAG_ZERO_GUESS)
            nod = ProjectionSolver(p["geom"], sigma, loc="nodal", prec=prec, stream=stream, flags=N.MG_FLAG_ZERO_GUESS)
            phim = torch.zeros_like(sigma)
            phin = torch.zeros(nod.vec_shape, dtype=torch.float64, device=dev)

            def step():
                with torch.cuda.stream(stream):
                    mac.update_coeff(sigma)
                    nod.update_coeff(sigma)
                    for a, b in zip(Um + Uc, U0m + U0c):
                        a.copy_(b)
                    a = mac.project(Um, beta0, S, beta0_face=b0f, phi=phim, tol=args.tol, allow_not_converged=True)
                    b = nod.project(Uc, beta0, S, phi=phin, tol=args.tol, allow_not_converged=True)
                    return a, b
            ms, (a, b) = _timed_solves(step, args.steps, args.warmup, stream)
            out[prec] = {"solves_per_s": 2 * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                         "mac": {k: a[k] for k in ("iters", "rel_resid", "rel_constraint")},
                         "nodal": {k: b[k] for k in ("iters", "rel_resid", "rel_constraint")},
                         "phi_mac": phim.cpu().numpy(), "phi_nodal": phin.cpu().numpy()}
    line = {"metric": "128^3 MAC + nodal projection step, FP64 plain multigrid, solves/s",
            "value": out["fp64"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["fp64"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "stratified atmosphere 128^3 (contrast 1e3, seed 2), MAC + nodal, tol %g" % args.tol},
            "mixed_vs_fp64": out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]}
    check = not args.no_cpu
    if check:
        import oracle as O
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        ref = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-13)
        refn = O.nodal_project(g, p["sigma"], p["beta0"], p["U_cell"], p["S"], tol=1e-13)
        live = ~g.dirichlet_node_mask()
    for prec in ("fp64", "mixed"):
        ph, pn = out[prec].pop("phi_mac"), out[prec].pop("phi_nodal")
        if check:
            out[prec]["mac"]["rel_l2_vs_oracle"] = float(np.linalg.norm(ph - ref["phi"]) / np.linalg.norm(ref["phi"]))
            out[prec]["nodal"]["rel_l2_vs_oracle"] = float(np.linalg.norm(pn[live] - refn["phi"][live]) /
                                                           np.linalg.norm(refn["phi"][live]))
        line[prec] = out[prec]
    return line


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gb300" else "gloo"
        if args.impl == "gb300":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    import numpy as np
    import torch

    import inputs as I
    from paper_1910_12979_gb300 import ProjectionSolver
    from paper_1910_12979_gb300 import native as N

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.workload != "stratified":
        if args.workload == "batch":
            line = run_batch(args, dev, world, dist)
        elif args.workload == "serve":
            line = run_serve(args, dev, rank, world, dist)
        elif args.workload == "config1":
            line = run_config1(args, dev)
        elif args.workload == "step":
            line = run_step(args, dev, world, dist)
        else:
            line = run_config2(args, dev)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    stream = torch.cuda.Stream(device=dev)
    n = args.n
    p = I.stratified(n, seed=3, contrast=1e3)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with torch.cuda.stream(stream):
        sigma, beta0, S = T(p["sigma"]), T(p["beta0"]), T(p["S"])
        b0f = [T(b) for b in p["beta0_face"]]
        U0m = [T(u) for u in p["U_mac"]]
        U0c = [T(u) for u in p["U_cell"]]
        Um = [u.clone() for u in U0m]
        Uc = [u.clone() for u in U0c]
    stream.synchronize()

    def make(prec):
        # every step starts the solves from phi = 0 (the step zeroes phi anyway)
        fl = N.MG_FLAG_ZERO_GUESS | {"v4": 0, "pipe": N.MG_FLAG_SWEEP_PIPE, "tma": N.MG_FLAG_SWEEP_TMA,
                                     "legs": N.MG_FLAG_CELL_PIPE}[args.sweep]
        cm = {"coarsest_max": args.coarsest} if args.coarsest > 0 else {}
        nu_c = [int(v) for v in args.nu.split(",")]
        nu_n = [int(v) for v in args.nu_nodal.split(",")]
        if args.autotune:
            fl |= N.MG_FLAG_AUTOTUNE
        mac = ProjectionSolver(p["geom"], sigma, loc="cell", prec=prec, stream=stream, flags=fl,
                               inner_cycles=args.inner_mac, nu1=nu_c[0], nu2=nu_c[1], **cm)
        nod = ProjectionSolver(p["geom"], sigma, loc="nodal", prec=prec, stream=stream,
                               flags=N.MG_FLAG_ZERO_GUESS | (N.MG_FLAG_AUTOTUNE if args.autotune else 0),
                               inner_cycles=args.inner_nodal, nu1=nu_n[0], nu2=nu_n[1], omega=args.omega_nodal,
                               **cm)
        phim = torch.zeros(mac.vec_shape, dtype=torch.float64, device=dev)
        phin = torch.zeros(nod.vec_shape, dtype=torch.float64, device=dev)
        return mac, nod, phim, phin

    stats = {}

    def step(solvers):
        mac, nod, phim, phin = solvers
        with torch.cuda.stream(stream):
            mac.update_coeff(sigma)
            nod.update_coeff(sigma)
            for a, b in zip(Um, U0m):
                a.copy_(b)
            for a, b in zip(Uc, U0c):
                a.copy_(b)
            stats["mac"] = mac.project(Um, beta0, S, beta0_face=b0f, phi=phim, tol=args.tol,
                                       allow_not_converged=True)
            stats["nodal"] = nod.project(Uc, beta0, S, phi=phin, tol=args.tol, allow_not_converged=True)

    def timed(solvers, K, W, prof=False, clocks=None):
        for _ in range(W):
            step(solvers)
        if dist is not None:
            dist.barrier()
        stream.synchronize()
        torch.cuda.synchronize(dev)
        if clocks:
            clocks.start()
        if prof:
            N.mg_prof_enable(True)
        l0 = N.mg_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step(solvers)
        e1.record(stream)
        e1.synchronize()
        launches = N.mg_launch_count() - l0
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        prof_out = None
        if prof:
            prof_out = {N.PROF_NAMES[k]: N.mg_prof_query(k) for k in N.PROF_NAMES}
            N.mg_prof_enable(False)
        ck = clocks.stop() if clocks else None
        if dist is not None:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            dist.barrier()
        return ms, launches, prof_out, ck

    mixed = make("mixed")
    ms, launches, prof, clocks = timed(mixed, args.steps, args.warmup, prof=True, clocks=Clocks(local))
    ms_step = ms / args.steps
    value = 2.0 * args.steps * world / (ms / 1e3)
    st_mac, st_nod = dict(stats["mac"]), dict(stats["nodal"])

    # roofline of the dominant (largest total time) instrumented kernel class;
    # the FP64 residuals are bound by the FP64 pipe, the FP32 sweeps by HBM
    hbm, bf16, src = peaks()
    # the FP64 classes are judged against the FP64 FMA rate measured here, on this GPU
    fp64_peak, fp64_clocks = fp64_peak_measured(dev, local)
    fp64_src = ("measured in this run: FP64 FMA probe (mg_fp64_fma_probe), median of 7 launches, "
                f"SM clock median {fp64_clocks['sm_mhz'] if fp64_clocks else 'n/a'} MHz")

    def roof(name):
        k = prof[name]
        n = max(k["launches"], 1)
        t = k["ms"] / n * 1e-3
        if name in N.PROF_FP64_BOUND:
            ach = k["flops"] / n / t / 1e12
            return {"kernel": name, "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": ach / fp64_peak, "traffic": ncu_traffic(name), "peak_source": fp64_src,
                    "algorithmic_flops_per_launch": k["flops"] / n, "algorithmic_bytes_per_launch": k["bytes"] / n,
                    "hbm_GBps": k["bytes"] / n / t / 1e9, "avg_launch_ms": t * 1e3, "launches": k["launches"],
                    "share_of_step": k["ms"] / ms if ms > 0 else None}
        ach = k["bytes"] / n / t / 1e9
        tr = ncu_traffic(name)
        out = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
               "traffic": tr, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
               "algorithmic_bytes_per_launch": k["bytes"] / n, "avg_launch_ms": t * 1e3,
               "launches": k["launches"], "share_of_step": k["ms"] / ms if ms > 0 else None}
        if tr:
            # the DRAM bytes the kernel actually moves (ncu, per launch) over this run's event-timed
            # launch duration: the kernel's fraction of the HBM peak on its own traffic
            out["dram_GBps"] = tr / t / 1e9
            out["dram_frac"] = tr / t / 1e9 / hbm
        return out

    live = [k for k in prof if prof[k]["launches"] > 0]
    dom = max(live, key=lambda k: prof[k]["ms"])
    roof_line = roof(dom)
    hbm_classes = [k for k in live if k not in N.PROF_FP64_BOUND]
    roof_line["hbm_kernel"] = roof(max(hbm_classes, key=lambda k: prof[k]["ms"])) if hbm_classes else None
    roof_line["all"] = {k: roof(k) for k in live}
    for v in roof_line["all"].values():
        v.pop("traffic", None)
        v.pop("peak_source", None)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": dict(workload_config(n, args.tol), parallelism=f"independent solves x{world}",
                           cell_smoother=args.sweep, smoothing={"mac": args.nu, "nodal": args.nu_nodal},
                           nodal_jacobi_omega=args.omega_nodal,
                           **({"autotuned_kinds": {nm: [N.mg_smoother_kind(sv.handle, l) for l in range(10)
                                                        if N.mg_smoother_kind(sv.handle, l) >= 0]
                                                   for nm, sv in (("mac", mixed[0]), ("nodal", mixed[1]))}}
                              if args.autotune else {})),
            "clocks": clocks, "gpu_launches": launches, "roofline": roof_line,
            "fp64_tflops_measured": fp64_peak, "fp64_probe_clocks": fp64_clocks,
            "solver": {nm: dict({k: st[k] for k in ("iters", "vcycles", "rel_resid", "rel_constraint")},
                                rel_constraint_before=st["rhs_norm"] / st["src_norm"] if st["src_norm"] > 0 else None)
                       for nm, st in (("mac", st_mac), ("nodal", st_nod))}}

    if args.only_mixed:
        args.no_fp64 = args.no_e2e = args.no_cpu = True
    # the same step with the graph-resident solve loop (no per-kernel events)
    msg, launches_g, _, _ = (0.0, 0, None, None) if args.only_mixed else timed(mixed, args.steps, 1)
    value_graph = 2.0 * args.steps * world / (msg / 1e3) if msg > 0 else None
    if not args.only_mixed:
        line["graph_path"] = {"value": value_graph, "unit": UNIT, "ms_per_step": msg / args.steps,
                              "gpu_launches": launches_g,
                              "note": "same step, iterations driven by CUDA-graph conditional nodes; the headline "
                                      "value uses the host-driven loop so that per-kernel CUDA events can be "
                                      "recorded"}

    # end to end through the public API with host buffers: every step copies its inputs from pinned
    # host memory and reads its projected velocities back.  Two device input and output sets, an
    # upload stream and a read-back stream (the two copy directions run concurrently) let the copies
    # of step k+1 and the read-back of step k-1 overlap the solves of step k.
    if not args.no_e2e:
        mac, nod, phim, phin = mixed
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        # the base state of the plane-parallel atmosphere depends on height only: it is uploaded as
        # radial tables every half cell (so every cell and face centre is a table point) and expanded
        # to sigma, beta0 at cells and beta0 at faces on the device by mg_base_state_map
        hz = p["geom"]["h"][2]
        nr = 2 * n + 1
        z_r = 0.5 * hz * np.arange(nr)
        rho_r = np.exp(-math.log(1e3) * z_r)
        beta_r = rho_r ** (1.0 / I.GAMMA1)
        geo = N.mg_geometry(3, (n, n, n), tuple(p["geom"]["h"]), N.MG_LOC_CELL)
        h_in = [pin(beta_r), pin(rho_r), pin(p["S"])] + [pin(u) for u in p["U_mac"]] + [pin(u) for u in p["U_cell"]]
        h2d = sum(t.numel() * t.element_size() for t in h_in)
        ustream = torch.cuda.Stream(device=dev)   # host -> device
        dstream = torch.cuda.Stream(device=dev)   # device -> host
        with torch.cuda.stream(stream):
            d_sets = [[torch.empty(nr, dtype=torch.float64, device=dev) for _ in range(2)] + [torch.empty_like(sigma)] +
                      [torch.empty_like(u) for u in U0m] + [torch.empty_like(u) for u in U0c] for _ in range(2)]
            m_sig, m_b0 = torch.empty_like(sigma), torch.empty_like(sigma)
            m_b0f = [torch.empty_like(b) for b in b0f]
        h_out = [[torch.empty_like(u, device="cpu").pin_memory() for u in Um + Uc] for _ in range(2)]
        d2h = sum(t.numel() * t.element_size() for t in h_out[0])
        h2d_done = [torch.cuda.Event() for _ in range(2)]
        comp_done = [torch.cuda.Event() for _ in range(2)]
        d2h_done = [torch.cuda.Event() for _ in range(2)]

        issue_ms = {"upload": 0.0, "download": 0.0, "calls": 0}   # host time spent issuing the copies
        tl = []   # (stage, event) of the first timed steps: where the device spends each step

        def mark(st_, name):
            if tl is not None and len(tl) < 36:
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(st_)
                tl.append((name, ev))

        def upload(i):
            t_issue = time.perf_counter()
            with torch.cuda.stream(ustream):
                ustream.wait_event(comp_done[i])   # the solves that used set i are done
                ustream.wait_event(d2h_done[i])    # and its projected velocities have been read back
                mark(ustream, f"upload{i}-start")
                for d, hsrc in zip(d_sets[i], h_in):
                    d.copy_(hsrc, non_blocking=True)
                h2d_done[i].record(ustream)
                mark(ustream, f"upload{i}-end")
            issue_ms["upload"] = max(issue_ms["upload"], (time.perf_counter() - t_issue) * 1e3)

        def compute(i):
            br, rr, Sv = d_sets[i][0], d_sets[i][1], d_sets[i][2]
            um, uc = d_sets[i][3:6], d_sets[i][6:9]   # projected in place
            stream.wait_event(h2d_done[i])
            mark(stream, f"step{i}-start")
            with torch.cuda.stream(stream):
                N.mg_base_state_map(geo, 0, (0.5, 0.5, 0.5), 0.0, 0.5 * hz, nr, br.data_ptr(), rr.data_ptr(),
                                    m_sig.data_ptr(), m_b0.data_ptr(), [b.data_ptr() for b in m_b0f],
                                    stream.cuda_stream)
                sg, b0, bf = m_sig, m_b0, m_b0f
                mac.update_coeff(sg)
                nod.update_coeff(sg)
                mac.project(um, b0, Sv, beta0_face=bf, phi=phim, tol=args.tol, allow_not_converged=True)
                nod.project(uc, b0, Sv, phi=phin, tol=args.tol, allow_not_converged=True)
                comp_done[i].record(stream)
                mark(stream, f"step{i}-end")

        def download(i):
            t_issue = time.perf_counter()
            with torch.cuda.stream(dstream):
                dstream.wait_event(comp_done[i])
                mark(dstream, f"readback{i}-start")
                for hd, d in zip(h_out[i], d_sets[i][3:9]):
                    hd.copy_(d, non_blocking=True)
                d2h_done[i].record(dstream)
                mark(dstream, f"readback{i}-end")
            issue_ms["download"] = max(issue_ms["download"], (time.perf_counter() - t_issue) * 1e3)

        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)

        def run(K, timed=False):
            torch.cuda.synchronize(dev)
            if timed:
                e0.record(stream)
            for i in range(2):   # fresh events (after e0): nothing to wait for at the start
                comp_done[i].record(stream)
                d2h_done[i].record(stream)
            upload(0)
            if K > 1:
                upload(1)
            for k in range(K):
                compute(k % 2)
                download(k % 2)
                if k + 2 < K:
                    upload(k % 2)   # after this step's solves (event): input set k % 2 is free
            stream.wait_event(d2h_done[(K - 1) % 2])
            stream.wait_event(h2d_done[(K - 1) % 2])
            if timed:
                e1.record(stream)
            torch.cuda.synchronize(dev)

        tl = None
        run(2)
        Ke = max(2, args.steps)
        if dist is not None:
            dist.barrier()
        tl = []
        run(Ke, timed=True)
        mse = e0.elapsed_time(e1)
        timeline = [(name, round(e0.elapsed_time(ev), 3)) for name, ev in tl]
        tl = None
        if dist is not None:
            t = torch.tensor([mse], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            mse = float(t.item())
        # the parts of a step timed one at a time (after the pipelined run; inputs resident):
        # the upload alone, the read-back alone, and the device work of one step alone
        def alone(st_, fn, reps=3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(st_)
            for _ in range(reps):
                fn()
            b.record(st_)
            b.synchronize()
            return a.elapsed_time(b) / reps

        def up_only():
            with torch.cuda.stream(ustream):
                for d, hsrc in zip(d_sets[0], h_in):
                    d.copy_(hsrc, non_blocking=True)

        def down_only():
            with torch.cuda.stream(dstream):
                for hd, d in zip(h_out[0], d_sets[0][3:9]):
                    hd.copy_(d, non_blocking=True)

        def compute_only(reps=3):
            # each projection starts from the step's inputs again (restored outside the timed part)
            tot = 0.0
            for _ in range(reps):
                with torch.cuda.stream(stream):
                    for d, u in zip(d_sets[0][3:9], U0m + U0c):
                        d.copy_(u)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                compute(0)
                b.record(stream)
                b.synchronize()
                tot += a.elapsed_time(b)
            return tot / reps

        t_up, t_down, t_comp = alone(ustream, up_only), alone(dstream, down_only), compute_only()
        torch.cuda.synchronize(dev)
        breakdown = {"h2d_ms": t_up, "h2d_gbs": h2d / (t_up * 1e6), "d2h_ms": t_down, "d2h_gbs": d2h / (t_down * 1e6),
                     "device_ms": t_comp, "pipelined_ms_per_step": mse / Ke,
                     "hidden_copy_ms": t_up + t_down + t_comp - mse / Ke,
                     "host_buffers_pinned": all(t.is_pinned() for t in h_in + h_out[0] + h_out[1]),
                     "max_host_issue_ms": {"upload": issue_ms["upload"], "download": issue_ms["download"]},
                     "timeline_ms": timeline,
                     "note": "each part timed alone with CUDA events on its own stream (the device part: the "
                             "base-state expansion, both coefficient rebuilds and both projections of one "
                             "step); hidden_copy_ms = the parts' sum minus the pipelined step time"}
        line["e2e"] = {"value": 2.0 * Ke * world / (mse / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": mse / Ke, "breakdown": breakdown,
                       "note": "pinned host inputs copied and results read back every step on an upload and "
                               "a read-back stream, overlapping the solves of the neighbouring steps "
                               "(double-buffered device inputs and outputs). The height-dependent base state "
                               "travels as its radial beta0 and rho0 tables (every half cell) and is expanded "
                               "to sigma and beta0 at cells and faces on the device (mg_base_state_map); each "
                               "step then rebuilds both hierarchies' coefficients from that sigma"}

    # plain FP64 GPU multigrid on the same workload (graph path, like graph_path above)
    if not args.no_fp64:
        f64 = make("fp64")
        K64 = max(1, min(args.steps, 3))
        ms64, _, _, _ = timed(f64, K64, 1)
        v64 = 2.0 * K64 * world / (ms64 / 1e3)
        line["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / K64,
                        "mac_iters": stats["mac"]["iters"], "nodal_iters": stats["nodal"]["iters"]}
        line["mixed_vs_fp64"] = value_graph / v64
        for s in f64[:2]:
            s.close()

    if args.parity and rank == 0:
        import oracle as O
        g = O.Grid.make(p["geom"]["n"], p["geom"]["bclo"], p["geom"]["bchi"])
        ref = O.mac_project(g, p["sigma"], p["beta0"], p["beta0_face"], p["U_mac"], p["S"], tol=1e-13)
        mixed[0].update_coeff(sigma)
        for a, b in zip(Um, U0m):
            a.copy_(b)
        phim = mixed[2]
        phim.zero_()
        mixed[0].project(Um, beta0, S, beta0_face=b0f, phi=phim, tol=args.tol, allow_not_converged=True)
        ph = phim.cpu().numpy()
        line["parity"] = {"mac_phi_rel_l2_vs_oracle": float(np.linalg.norm(ph - ref["phi"]) / np.linalg.norm(ref["phi"])),
                          "oracle_relres": ref["relres"], "tol": args.tol}

    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"], ref = oracle_cpu_leg(n)
        line["parity"] = dict(line.get("parity", {}), **gpu_error_vs_oracle(ref, dev, args.tol))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
