"""Benchmark: batched mixed-precision minimisation throughput (solves/s) on GB300.

Workload (default): 64 independent minimisation problems on one 60 nm cube
(30^3 cells, 6 Kuhn tetrahedra per cell, 29 791 nodes, 5 402 surface nodes),
Nd2Fe14B, applied fields U[-8,0] T along z and easy-axis tilts U[0,5] deg drawn
from seed 4, m0 = +z perturbed; each solve runs the curvilinear steepest-descent
minimiser to max|m x h_eff|/Js < 1e-6.  One step = set m0 (device resident) and
minimise the whole batch.  Inputs are synthetic (seeded), shaped like the
paper's permanent-magnet grain workload.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on
the host cores instead (bounded sample per step, same metric).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")          # the CPU oracle legs run on one core

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth.inputs import A_JM, JS_T, K1_JM3, batched_case  # noqa: E402

METRIC = "solves/s, batched mixed-prec vs plain FP64 on GB300 at <=1e-6 rel energy; p50/p99 ms"
N_CELLS = 30
BATCH = 64


def batched_config() -> dict:
    """The benchmark workload (identical on both arms)."""
    N = (N_CELLS + 1) ** 3
    nb = N - (N_CELLS - 1) ** 3
    return {"workload": f"batched same-mesh: {BATCH} instances on a {N_CELLS}^3-cell (60 nm) Kuhn cube, "
                        f"{N} nodes, {nb} surface nodes",
            "n": N_CELLS, "batch": BATCH, "tol": 1e-6, "l2": "flushed between timed steps (512 MB write)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_tc", choices=["mixed", "mixed_tc", "fp64"])
    ap.add_argument("--fp64-sample", type=int, default=4,
                    help="instances of the plain-FP64 single-instance comparison arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-s", type=float, default=20.0)
    ap.add_argument("--ref-step-s", type=float, default=0.0,
                    help="seconds of oracle work per step of the reference arm (0: 5-30 s by step count)")
    ap.add_argument("--ref-cores", type=int, default=0,
                    help="host processes of the reference arm (0: all cores, capped by memory)")
    ap.add_argument("--workload", default="batched", choices=["batched", "served", "large", "shell"],
                    help="batched: 64 same-mesh instances (default); served: Poisson request stream; "
                         "large: one instance on an n^3 cube (n = 80: 531 441 nodes, 5.9 GB FP32 BEM matrix); "
                         "shell: the batched workload with the space-transformation boundary")
    ap.add_argument("--n", type=int, default=80, help="cells per side of the large workload")
    ap.add_argument("--shell-a", type=int, default=4, help="air cells of the shell workload")
    ap.add_argument("--shell-s", type=int, default=8, help="shell cells of the shell workload")
    ap.add_argument("--no-shell", action="store_true",
                    help="skip the space-transformation leg (the bench batch with the shell boundary)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the single-instance 80^3-cell leg of the default line")
    ap.add_argument("--large-hm-eps", type=float, default=1e-6,
                    help="tolerance of the H-matrix variant of the large leg (0: dense only)")
    ap.add_argument("--max-iter", type=int, default=100000, help="iteration cap of the large workload")
    ap.add_argument("--pcg-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="potential-solve kernel (lbm_solve_opts.pcg_kernel): 0 choose, 1 grid-wide, 2 clusters")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--rate", type=float, default=0.0, help="arrivals/s (0: 0.8 x calibrated capacity)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank: int) -> int:
    """Seed of the independent batch a rank solves: rank 0 solves the seed-4
    batch (the one the parity tests pin); rank r > 0 an independent batch of the
    same distribution.  The problems are independent, so ranks share nothing on
    the data path (weak scaling: BATCH solves per rank per step)."""
    return 4 if rank == 0 else 4 + 7919 * rank


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """Whole-job time: the slowest rank's seconds (all-reduce MAX over the
    initialised process group; the identity for one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(solves_per_rank: int, seconds: float, ws: int) -> float:
    """solves/s of the whole job: every rank's solves over the slowest rank's time."""
    return ws * solves_per_rank / seconds


def _oracle_proc(k, n_windows, budget_s, q_ready, go, q_out):
    """One host core (a spawned process): build the oracle problem of instance k
    (set-up, not timed), report ready, then for each window, when `go[w]` is
    set, run minimiser steps for budget_s seconds and report (w, evaluations,
    seconds)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from oracle.micromag import CubeProblem
    from oracle.minimise import minimise
    inst = batched_case(N_CELLS, BATCH, seed=4)[k]
    p = CubeProblem(inst.n, inst.Js, inst.A, inst.K1, inst.axis)
    q_ready.put(k)
    m = inst.m0
    for w in range(n_windows):
        go[w].wait()
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < budget_s:
            r = minimise(p, m, inst.h_ext, tol=1e-6, max_iter=8)
            done += r.evaluations
            m = inst.m0 if r.status == 0 else r.m
        q_out.put((w, done, time.perf_counter() - t0))


def host_cores(max_workers=None):
    """Worker processes for the all-cores oracle timing: the host's cores, capped
    by memory (~1.5 GB per worker for the 30^3-cell problem)."""
    n = os.cpu_count() or 1
    try:
        mem = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        n = max(1, min(n, int(mem // 1.5e9)))
    except (ValueError, OSError, AttributeError):
        pass
    return min(n, max_workers) if max_workers else n


def oracle_all_cores(budget_s, cores, n_windows=1, setup_timeout_s=300.0):
    """Oracle throughput with `cores` processes at once, each on its own instance
    of the workload; all start every timed window together.  Returns, per
    window, (evaluations per second, evaluations, seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q_ready, q_out = ctx.Queue(), ctx.Queue()
    go = [ctx.Event() for _ in range(n_windows)]
    procs = [ctx.Process(target=_oracle_proc, args=(k % BATCH, n_windows, budget_s, q_ready, go, q_out))
             for k in range(cores)]
    for pr in procs:
        pr.start()
    try:
        for _ in range(cores):
            q_ready.get(timeout=setup_timeout_s)
        out = []
        for w in range(n_windows):
            go[w].set()
            res = [q_out.get(timeout=budget_s + 300.0) for _ in range(cores)]
            evals = sum(r[1] for r in res)
            secs = max(r[2] for r in res)
            out.append((evals / secs, evals, secs))
        return out
    finally:
        for pr in procs:
            pr.join(timeout=30)
            if pr.is_alive():
                pr.terminate()


def golden_evals_per_solve():
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "batched_n30.json")))
    return float(np.mean([r["evaluations"] for r in gold["results"]]))


def cpu_oracle_sample(insts, evals_per_solve_gpu, budget_s):
    """Time the FP64 oracle on one instance of the workload: field evaluations
    and steps for about `budget_s` seconds (set-up -- assembly, BEM, LU -- is
    excluded, as in the paper's CPU timings), scaled to solves/s with the
    evaluations per solve measured on the GPU."""
    from oracle.micromag import CubeProblem
    from oracle.minimise import minimise
    inst = insts[0]
    p = CubeProblem(inst.n, inst.Js, inst.A, inst.K1, inst.axis)
    t0 = time.perf_counter()
    done_evals = 0
    chunk = 8
    m = inst.m0
    while time.perf_counter() - t0 < budget_s:
        r = minimise(p, m, inst.h_ext, tol=1e-6, max_iter=chunk)
        done_evals += r.evaluations
        m = r.m
        if r.status == 0:
            m = inst.m0
    dt = time.perf_counter() - t0
    per_eval = dt / max(done_evals, 1)
    try:
        evals_per_solve = golden_evals_per_solve()
        src = "the oracle's own mean over the 64 instances"
    except Exception:
        evals_per_solve, src = evals_per_solve_gpu, "the GPU run"
    out = {"value": 1.0 / (per_eval * evals_per_solve), "unit": "solves/s", "cores": 1,
           "kind": "oracle",
           "sample": (f"FP64 numpy/scipy oracle (one thread), instance 0 of the {N_CELLS}^3-cell "
                      f"workload: {done_evals} energy-gradient evaluations in {dt:.1f} s "
                      f"({per_eval * 1e3:.1f} ms each, set-up excluded), scaled by "
                      f"{evals_per_solve:.0f} evaluations per solve ({src})")}
    # the same oracle on all host cores at once (one process per core, each on
    # its own instance): the host's full throughput
    try:
        cores = host_cores()
        rate, ev, secs = oracle_all_cores(budget_s, cores)[0]
        out["all_cores"] = {"value": rate / evals_per_solve, "unit": "solves/s", "cores": cores,
                            "sample": f"{cores} processes, one instance each, {ev} evaluations in {secs:.1f} s "
                                      f"(set-up excluded)"}
    except Exception as exc:   # the single-core figure stands on its own
        out["all_cores"] = {"error": repr(exc)[:200]}
    return out


def _single_core_rate(per_step, n_windows):
    """Oracle evaluations per second on this process's one core, per window."""
    from oracle.micromag import CubeProblem
    from oracle.minimise import minimise
    inst = batched_case(N_CELLS, BATCH, seed=4)[0]
    p = CubeProblem(inst.n, inst.Js, inst.A, inst.K1, inst.axis)
    out, m = [], inst.m0
    for _ in range(n_windows):
        t0 = time.perf_counter()
        ev = 0
        while time.perf_counter() - t0 < per_step:
            r = minimise(p, m, inst.h_ext, tol=1e-6, max_iter=8)
            ev += r.evaluations
            m = r.m if r.status != 0 else inst.m0
        dt = time.perf_counter() - t0
        out.append((ev / dt, ev, dt))
    return out


def run_reference(args, ws, rank):
    """The oracle as it stands on the host's cores: one process per core, each on
    its own instance of the workload, all timed together for a bounded window per
    step (set-up excluded); evaluations per solve from the oracle's own runs."""
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    per_step = args.ref_step_s if args.ref_step_s > 0 else max(5.0, min(30.0, 120.0 / max(1, args.steps + args.warmup)))
    n_windows = args.warmup + args.steps
    evals_per_solve = golden_evals_per_solve()
    cores = host_cores(args.ref_cores if args.ref_cores > 0 else None)
    how = f"{cores} processes (one per core), one instance each"
    try:
        windows = oracle_all_cores(per_step, cores, n_windows=n_windows)
    except Exception as exc:   # fall back to this process's one core
        cores = 1
        how = f"one core (the all-core run failed: {repr(exc)[:120]})"
        windows = _single_core_rate(per_step, n_windows)
    timed = windows[args.warmup:]
    rate = float(np.mean([w[0] for w in timed]))
    total_evals = sum(w[1] for w in timed)
    value = rate / evals_per_solve
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean([w[2] for w in timed])) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": batched_config(),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"FP64 numpy/scipy oracle on {how}: {total_evals} energy-gradient "
                                       f"evaluations over {args.steps} windows of {per_step:.0f} s (set-up "
                                       f"excluded), scaled by {evals_per_solve:.0f} evaluations per solve"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes (read + write) per millisecond of kernel time of the potential-solve
# kernels, from one ncu capture each of the batched workload (profiles/), used to
# report the roofline's measured traffic per launch: (bytes/ms) x average launch ms.
PROFILED_DRAM_BYTES_PER_MS = {
    "fp32": (1109.2e6 / 6.216, "profiles/k_pcg_cluster_fp32_batched64_n30.md"),
}


def pinned_copy(a: np.ndarray):
    """A float64 copy of `a` in page-locked host memory, for the end-to-end leg's
    host<->device copies: (array, owner, "pinned"), the owner keeping the memory
    alive; (array, None, "pageable") when page-locked memory is refused."""
    try:
        import torch
        t = torch.empty(tuple(a.shape), dtype=torch.float64, pin_memory=True)
        out = t.numpy()
        out[...] = a
        return out, t, "pinned"
    except Exception:
        return np.array(a, dtype=np.float64, order="C"), None, "pageable"


def pcg_bytes_per_row(kind):
    """Algorithmic bytes of one PCG iteration per row and system: z gather, p rw,
    q rw (phase A); x rw, r rw, p and q read, z write (phase B) = 12 vector
    words.  FP32 solves: 12 x 4 B; plain FP64: 12 x 8 B; FP64 solves iterated in
    FP32: 12 x 4 B (the FP32 correction takes x's place; it is folded into the
    FP64 x once per restart cycle, not counted).  The int8 stiffness tables are
    shared by all systems and not counted."""
    return {"fp32": 48, "fp64": 96, "fp64_fp32iter": 48}[kind]


# Algorithmic bytes of one unit of each kernel kind on a single instance (B = 1),
# FP32 work vectors: every array a kernel must touch read or written once (the
# mesh tables included -- with one instance they are not shared):
#   trial update, per node: m and grad phi at the base point (2 x 24 B), the
#     trial m (24 B) and, in the FP32 phase, its FP32 copy (12 B);
#   field, per node: the CSR row (column, {K, G}, G^T words: 12 B per entry),
#     the node word (4 B), the trial point (24 B FP64 + 12 B FP32 copy in the
#     FP32 phase, or 24 B), the base point and its gradient (48 B), three
#     potential columns (12 or 24 B), the new gradient (24 B);
#   potential solves, per row and sweep of the two systems (forward, adjoint):
#     12 FP32 words per system (z, p, q; x or d, r, p, q, z) and the row's
#     stiffness entries, pointer and node word (36 B);
#   BEM products, per evaluation: the forward and the transposed product each
#     read the matrix once (4 or 8 B per entry; with B_H its stored values).
def large_leg(local, n, hm_eps, max_iter=100000, warmup=1):
    """One instance on an n^3-cell cube (random start, -3 T, mixed precision):
    time to solution and per-kernel achieved bandwidth against the measured HBM
    peak, with the dense boundary matrix and (hm_eps > 0) with B_H."""
    import torch
    import paper_1309_5796_gb300 as lbm
    from synth.inputs import large_case
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    stream = torch.cuda.current_stream()
    ctx = lbm.Context(local, stream=stream.cuda_stream)
    case = large_case(n)
    t0 = time.perf_counter()
    mesh = ctx.mesh_cube(2e-9, n)
    setup_s = time.perf_counter() - t0
    info = ctx.mesh_info(mesh)
    N, nb, nnz = info["N"], info["nb"], info["nnz"]
    m0 = torch.from_numpy(np.ascontiguousarray(case.m0)).to(f"cuda:{local}")
    out = {"workload": f"one instance on a {n}^3-cell Kuhn cube ({N} nodes, {nb} surface nodes), random start "
                       "on the sphere (seed 3), -3 T along z, mixed precision; BEM matrix "
                       f"{4 * nb * nb / 1e9:.2f} GB in FP32 (> L2)",
           "mesh_setup_s": round(setup_s, 2), "peak_GB_s": hbm_peak,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    variants = [("dense", 0.0)] + ([("hmatrix", hm_eps)] if hm_eps > 0 else [])
    for name, eps in variants:
        stored = nb * nb
        if eps > 0:
            t0 = time.perf_counter()
            hinfo = ctx.mesh_hmatrix(mesh, eps)
            stored = hinfo["stored"]
            build_s = time.perf_counter() - t0
        inst = ctx.instance_create(mesh, 1, lbm.LBM_MIXED)
        inst.set_material(JS_T, A_JM, K1_JM3, case.axis)
        inst.set_field(case.h_ext)
        opts = lbm.default_opts(lbm.LBM_MIXED, max_iter=max_iter)
        for _ in range(warmup):
            inst.set_m_device(m0.data_ptr())
            inst.minimise(opts)
        ctx.profile_read(reset=True)
        ctx.profile_enable(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst.set_m_device(m0.data_ptr())
        r = inst.minimise(opts)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = ctx.profile_read(reset=True)
        ctx.profile_enable(False)
        inst.destroy()
        n32, n64 = prof["pcg1_fp32"]["launches"], prof["pcg1_fp64"]["launches"]
        sweeps = sum(prof["cg_sweeps"])
        kern = {
            "trial_update": (prof["trial_update"], (n32 * 84 + n64 * 72) * N),
            "field": (prof["field"], (n32 + n64) * (12 * nnz + 124 * N)),
            "potential_solves": ({"ms": sum(prof[k]["ms"] for k in ("pcg1_fp32", "pcg2_fp32", "pcg1_fp64", "pcg2_fp64")),
                                  "launches": sum(prof[k]["launches"] for k in ("pcg1_fp32", "pcg2_fp32", "pcg1_fp64",
                                                                                "pcg2_fp64"))},
                                 sweeps * N * (2 * 48 + 36)),
            "bem_products": (prof["bem_product"], (n32 * 2 * 4 + n64 * 2 * 8) * stored),
        }
        per = {}
        for k, (p, by) in kern.items():
            gbs = by / (p["ms"] / 1e3) / 1e9 if p["ms"] > 0 else None
            per[k] = {"ms": round(p["ms"], 3), "launches": p["launches"], "bytes": int(by),
                      "GB_s": round(gbs, 1) if gbs else None,
                      "frac": round(gbs / hbm_peak, 4) if gbs else None}
        v = {"ms_to_solution": round(ms, 1), "status": r["status"], "iterations": r["iterations"],
             "evaluations": r["evaluations"], "torque": r["torque"], "energy_J": r["energy"][4],
             "cg_sweeps": prof["cg_sweeps"], "kernels": per}
        if eps > 0:
            v.update({"eps": eps, "stored_values": stored, "stored_fraction": round(stored / (nb * nb), 4),
                      "build_s": round(build_s, 2)})
        out[name] = v
    ctx.mesh_destroy(mesh)
    ctx.close()
    return out


# DRAM bytes per ms of k_shell_pcg kernel time from the ncu capture in
# profiles/k_shell_pcg_fp32_batched64_n30_shell4x8.md (185.02 GB in 37.659 ms)
PROFILED_SHELL_DRAM_BYTES_PER_MS = 185.02e9 / 37.659


def shell_leg(ctx, local, insts, a=4, s=8, precision="mixed"):
    """The bench's batch (64 instances on the 30^3-cell cube, same materials,
    fields and starts) with the open boundary by space transformation (Sec. 3.1:
    the paper's own solver) instead of FEM/BEM: air a cells, shell s cells, one
    grid of (30 + 2(a + s))^3 cells.  Time to solution of the batch and the
    shell solve kernel's achieved bandwidth against the measured HBM peak.
    Algorithmic bytes of one CG iteration per grid row off the outer face: 12
    work-vector words per instance (z, p, q read and p, q written in the stencil
    pass; d, p, r, q read and d, r, z written in the update pass: FP32 words in
    the FP32 phase and in the mixed-iteration FP64 phase) and the row's stencil
    record read twice (64 B + 4 B FP32), shared by the instances."""
    import torch
    import paper_1309_5796_gb300 as lbm
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    stream = torch.cuda.current_stream()
    prec = {"mixed": lbm.LBM_MIXED, "fp64": lbm.LBM_FP64}[precision]
    B = len(insts)
    mesh = ctx.mesh_cube(2e-9, N_CELLS)
    t0 = time.perf_counter()
    info = ctx.mesh_shell(mesh, a, s)
    setup_s = time.perf_counter() - t0
    nt = N_CELLS + 2 * (a + s)
    rows = info["grid_nodes"] - (6 * nt * nt + 2)          # grid rows off the outer face
    inst = ctx.instance_create(mesh, B, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, np.stack([i.axis for i in insts]))
    inst.set_field(np.stack([i.h_ext for i in insts]))
    m0 = torch.from_numpy(np.stack([i.m0 for i in insts])).to(f"cuda:{local}")
    opts = lbm.default_opts(prec)
    inst.set_m_device(m0.data_ptr())
    inst.evaluate(opts, want_h=False, want_u=False)          # one-time set-up (attributes, occupancy)
    ctx.profile_read(reset=True)
    ctx.profile_enable(True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    inst.set_m_device(m0.data_ptr())
    res = inst.minimise(opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    inst.destroy()
    ctx.mesh_destroy(mesh)
    sw = prof["cg_sweeps"]
    word = 4 if (precision == "mixed" or opts.cg_mixed_iter) else 8
    rec = 68 if word == 4 else 136
    solve_ms = prof["pcg1_fp32"]["ms"] + prof["pcg1_fp64"]["ms"]
    by = (sw[0] + sw[2]) * rows * (12 * word * B + rec)
    gbs = by / (solve_ms / 1e3) / 1e9 if solve_ms > 0 else None
    nlaunch = prof["pcg1_fp32"]["launches"] + prof["pcg1_fp64"]["launches"]
    avg_ms = solve_ms / max(1, nlaunch)
    return {"workload": f"the bench batch ({B} instances, {N_CELLS}^3-cell cube) with the space-transformation "
                        f"boundary: air {a}, shell {s} cells, grid {nt}^3 cells ({info['grid_nodes']} nodes, "
                        f"{info['shell_tets']} shell tetrahedra), {precision} precision",
            "setup_s": round(setup_s, 3), "ms_to_solution": round(ms, 1),
            "solves_per_s": B / (ms / 1e3), "statuses_nonzero": [r["status"] for r in res if r["status"]],
            "evaluations_per_solve": float(np.mean([r["evaluations"] for r in res])),
            "cg_sweeps": sw,
            "shell_solve": {"kernel": "k_shell_pcg", "ms": round(solve_ms, 2),
                            "launches": prof["pcg1_fp32"]["launches"] + prof["pcg1_fp64"]["launches"],
                            "us_per_sweep": round(1e3 * solve_ms / max(1, sw[0] + sw[2]), 1),
                            "bytes": int(by), "GB_s": round(gbs, 1) if gbs else None,
                            "frac": round(gbs / hbm_peak, 4) if gbs else None,
                            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                            "algorithmic_bytes_per_sweep": rows * (12 * word * B + rec),
                            "avg_launch_ms": round(avg_ms, 3),
                            "bytes_per_launch": by / max(1, nlaunch),
                            "traffic": PROFILED_SHELL_DRAM_BYTES_PER_MS * avg_ms if word == 4 else None,
                            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per ms of kernel "
                                               "time (profiles/k_shell_pcg_fp32_batched64_n30_shell4x8.md) x "
                                               "average launch duration") if word == 4 else None},
            "kernel_ms": {k: round(v["ms"], 2) for k, v in prof.items()
                          if isinstance(v, dict) and v.get("launches")}}


def run_ours(args, ws, rank, local):
    import torch
    import paper_1309_5796_gb300 as lbm
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = {"mixed": lbm.LBM_MIXED, "mixed_tc": lbm.LBM_MIXED_TC, "fp64": lbm.LBM_FP64}[args.precision]
    stream = torch.cuda.current_stream()
    ctx = lbm.Context(local, stream=stream.cuda_stream)
    insts = batched_case(N_CELLS, BATCH, seed=rank_seed(rank))
    mesh = ctx.mesh_cube(2e-9, N_CELLS)
    info = ctx.mesh_info(mesh)
    N = info["N"]
    inst = ctx.instance_create(mesh, BATCH, prec)
    axes = np.stack([i.axis for i in insts])
    fields = np.stack([i.h_ext for i in insts])
    inst.set_material(JS_T, A_JM, K1_JM3, axes)
    inst.set_field(fields)
    m0_host = np.stack([i.m0 for i in insts])
    m0_dev = torch.from_numpy(m0_host).to(f"cuda:{local}")
    opts = lbm.default_opts(prec, pcg_kernel=args.pcg_kernel)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    def step():
        inst.set_m_device(m0_dev.data_ptr())
        return inst.minimise(opts)

    res = []
    for _ in range(args.warmup):
        res = step()
    bad = [r["status"] for r in res if r["status"] != 0]
    ctx.profile_read(reset=True)
    ctx.profile_enable(True)
    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    step_ms = []
    evals = []
    for _ in range(args.steps):
        flush.zero_()                                 # L2 flush between timed steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        evals.extend(r["evaluations"] for r in res)
        bad.extend(r["status"] for r in res if r["status"] != 0)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = ctx.launch_count() - launches0
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    clocks = sampler.stop()
    total_s = max_over_ranks(sum(step_ms) / 1e3, ws, device=f"cuda:{local}")
    value = whole_job_value(BATCH * args.steps, total_s, ws)
    final_res = res

    # end to end through the public API with host buffers (H2D of m0, D2H of m),
    # both in page-locked memory
    m0_e2e, _m0_owner, host_mem = pinned_copy(m0_host)
    m_out, _mo_owner, _ = pinned_copy(np.zeros_like(m0_host))
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        inst.set_m(m0_e2e)
        inst.minimise(opts)
        inst.get_m(out=m_out)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_s = max_over_ranks(statistics.mean(e2e_ms) / 1e3, ws, device=f"cuda:{local}")
    e2e_value = whole_job_value(BATCH, e2e_s, ws)

    if rank != 0:
        return
    # roofline of the dominant kernel: the potential solves (k_pcg).  Algorithmic
    # bytes per system-iteration and row: z gather, p rw, q rw (phase A), x rw,
    # r rw, p, q read, z write (phase B) = 12 vector words; the int8 matrix and
    # the row tables are shared by all 2B systems and not counted.
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    kinds = {k: v for k, v in prof.items() if k not in ("cg_iters", "cg_sweeps")}
    total_kernel_ms = sum(v["ms"] for v in kinds.values())
    pcg = {}
    fp64_kind = "fp64_fp32iter" if opts.cg_mixed_iter and prec != lbm.LBM_FP64 else "fp64"
    for name, idx, kind in (("fp32", 0, "fp32"), ("fp64", 1, fp64_kind)):
        ms = kinds[f"pcg1_{name}"]["ms"] + kinds[f"pcg2_{name}"]["ms"]
        nl = kinds[f"pcg1_{name}"]["launches"] + kinds[f"pcg2_{name}"]["launches"]
        by = prof["cg_iters"][idx] * pcg_bytes_per_row(kind) * N
        pcg[name] = dict(ms=ms, launches=nl, bytes=by, kind=kind)
    dom = max(pcg, key=lambda k: pcg[k]["ms"])
    d = pcg[dom]
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] > 0 else 0.0
    avg_ms = d["ms"] / max(d["launches"], 1)
    traffic, traffic_src = None, None
    if d["kind"] in PROFILED_DRAM_BYTES_PER_MS and args.workload == "batched":
        rate, traffic_src = PROFILED_DRAM_BYTES_PER_MS[d["kind"]]
        traffic = rate * avg_ms
    roofline = {"bound": "hbm", "kernel": f"k_pcg_cluster ({d['kind']} potential solves, forward + adjoint)",
                "bytes_per_row_system_iteration": pcg_bytes_per_row(d["kind"]),
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum per ms of kernel time "
                                   f"({traffic_src}) x average launch duration") if traffic_src else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "bytes_per_launch": d["bytes"] / max(d["launches"], 1),
                "avg_launch_ms": avg_ms,
                "share_of_kernel_time": d["ms"] / total_kernel_ms if total_kernel_ms else None,
                "other": {k: {"ms": round(v["ms"], 2), "GB_s": (v["bytes"] / (v["ms"] / 1e3) / 1e9
                                                                 if v["ms"] > 0 else None)}
                          for k, v in pcg.items()}}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(insts, statistics.mean(evals), args.cpu_sample_s)

    fp64_arm = None
    if args.fp64_sample > 0 and prec != lbm.LBM_FP64:
        single = ctx.instance_create(mesh, 1, lbm.LBM_FP64)
        o64 = lbm.default_opts(lbm.LBM_FP64)
        t_fp64, e_err = [], []
        Kd = JS_T ** 2 / (2 * 4e-7 * math.pi)
        for b in range(args.fp64_sample):
            single.set_material(JS_T, A_JM, K1_JM3, axes[b])
            single.set_field(fields[b])
            single.set_m(m0_host[b])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r64 = single.minimise(o64)[0]
            t_fp64.append(time.perf_counter() - t0)
            Eref = r64["energy"][4]
            scale = max(abs(Eref), Kd * (N_CELLS * 2e-9) ** 3)
            e_err.append(abs(final_res[b]["energy"][4] - Eref) / scale)
        fp64_arm = {"solves_per_s": 1.0 / statistics.mean(t_fp64), "instances_timed": args.fp64_sample,
                    "ms_per_solve": 1e3 * statistics.mean(t_fp64),
                    "speedup_of_batched_mixed": value / (1.0 / statistics.mean(t_fp64)),
                    "max_rel_energy_err_batched_mixed_vs_fp64": max(e_err)}
        single.destroy()

    shell = None
    if not args.no_shell:
        try:
            shell = shell_leg(ctx, local, insts, a=args.shell_a, s=args.shell_s)
        except Exception as exc:   # the headline stands on its own
            shell = {"error": repr(exc)[:300]}

    large = None
    if not args.no_large:
        try:
            large = large_leg(local, 80, args.large_hm_eps, warmup=1)
        except Exception as exc:   # the headline stands on its own
            large = {"error": repr(exc)[:300]}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "mixed_tc": "f32+tf32x3+f64", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": batched_config(), "precision": args.precision,
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "statuses_nonzero": bad,
        "evaluations_per_solve": statistics.mean(evals),
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roofline,
        "kernel_ms": {k: round(v["ms"], 3) for k, v in kinds.items()},
        "cpu_baseline": cpu,
        "fp64_single_instance": fp64_arm,
        "large_single_instance_n80": large,
        "shell_boundary_batched64_n30": shell,
        "e2e": {"value": e2e_value, "unit": "solves/s",
                "h2d_bytes_per_step": int(m0_e2e.nbytes), "d2h_bytes_per_step": int(m_out.nbytes),
                "host_memory": host_mem},
    }
    print(json.dumps(line), flush=True)


def run_served(args, ws, rank, local):
    """Served stream: Poisson arrivals of minimisation requests on cubes of
    10^3..50^3 cells (random field and tilt), continuous batching in the
    library's server; p50/p99 latency (submit -> result) and solves/s."""
    import torch
    import paper_1309_5796_gb300 as lbm
    from synth.inputs import served_stream
    torch.cuda.set_device(local)
    ctx = lbm.Context(local)
    ctx.serve_start(slots=16, chunk=8)
    rate = args.rate
    calib = None
    if rate <= 0:
        # closed-loop burst of 48 requests of the same distribution -> capacity
        burst = served_stream(48, 1.0, seed=55)
        t0 = time.perf_counter()
        ts = [ctx.submit(r.inst.n, 2e-9, JS_T, A_JM, K1_JM3, r.inst.axis, r.inst.h_ext, r.inst.m0)
              for r in burst]
        for t in ts:
            ctx.wait(t, None, timeout_s=900)
        cap = len(burst) / (time.perf_counter() - t0)
        rate = 0.8 * cap
        calib = {"burst_requests": len(burst), "capacity_solves_per_s": cap}
    reqs = served_stream(args.requests, rate, seed=5)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.launch_count()
    t_start = time.perf_counter()
    tickets = []
    for r in reqs:
        delay = r.arrival_s - (time.perf_counter() - t_start)
        if delay > 0:
            time.sleep(delay)
        tickets.append(ctx.submit(r.inst.n, 2e-9, JS_T, A_JM, K1_JM3, r.inst.axis, r.inst.h_ext, r.inst.m0))
    results = [ctx.wait(t, None, timeout_s=1800)[0] for t in tickets]
    makespan = time.perf_counter() - t_start
    clocks = sampler.stop()
    stats = ctx.serve_stats()
    launches = ctx.launch_count() - launches0
    ctx.serve_stop()
    lat = np.array([r["wall_ms"] for r in results])
    ok = sum(r["status"] == 0 for r in results)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": ok / makespan, "unit": "solves/s", "n_gpus": ws, "steps": 1,
            "warmup": 0, "ms_per_step": makespan * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"served stream: {args.requests} Poisson requests at {rate:.2f}/s, "
                                   "cubes of 10^3..50^3 cells, mixed precision, 16 slots per cube size",
                       "rate_per_s": rate, "calibration": calib},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "completed_ok": ok, "stats": stats, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_large(args, ws, rank, local):
    """One instance on a large cube (random start on the sphere, -3 T along z,
    mixed precision): time to solution and the roofline of the BEM products,
    the kernels whose operand (the FP32 matrix, 4 nb^2 bytes) exceeds L2."""
    import torch
    import paper_1309_5796_gb300 as lbm
    from synth.inputs import large_case
    torch.cuda.set_device(local)
    prec = {"mixed": lbm.LBM_MIXED, "mixed_tc": lbm.LBM_MIXED, "fp64": lbm.LBM_FP64}[args.precision]
    stream = torch.cuda.current_stream()
    ctx = lbm.Context(local, stream=stream.cuda_stream)
    case = large_case(args.n)
    t0 = time.perf_counter()
    mesh = ctx.mesh_cube(2e-9, args.n)
    setup_s = time.perf_counter() - t0
    info = ctx.mesh_info(mesh)
    N, nb = info["N"], info["nb"]
    inst = ctx.instance_create(mesh, 1, prec)
    inst.set_material(JS_T, A_JM, K1_JM3, case.axis)
    inst.set_field(case.h_ext)
    opts = lbm.default_opts(prec, max_iter=args.max_iter)
    m0 = torch.from_numpy(np.ascontiguousarray(case.m0)).to(f"cuda:{local}")
    for _ in range(args.warmup):
        inst.set_m_device(m0.data_ptr())
        inst.minimise(opts)
    sampler = ClockSampler(local)
    sampler.start()
    ctx.profile_read(reset=True)
    ctx.profile_enable(True)
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    ms, res = [], None
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst.set_m_device(m0.data_ptr())
        res = inst.minimise(opts)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    clocks = sampler.stop()
    launches = ctx.launch_count() - launches0
    if rank != 0:
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # one evaluation = one forward and one transposed product: the FP32 matrix in
    # the FP32 phase, the FP64 matrix in FP64 runs and in the FP64 phase of mixed
    # runs (one BEM scope per evaluation: as many as first-stage solves)
    word = 8 if prec == lbm.LBM_FP64 else 4
    bem = prof["bem_product"]
    n32, n64 = prof["pcg1_fp32"]["launches"], prof["pcg1_fp64"]["launches"]
    bem_bytes = (n32 * 2 * 4 + n64 * 2 * 8) * nb * nb if n32 + n64 == bem["launches"] else \
        bem["launches"] * 2 * word * nb * nb
    achieved = bem_bytes / (bem["ms"] / 1e3) / 1e9 if bem["ms"] > 0 else 0.0
    kinds = {k: v for k, v in prof.items() if k not in ("cg_iters", "cg_sweeps")}
    line = {"metric": "solves/s, one instance on a large cube", "value": 1e3 / statistics.mean(ms),
            "unit": "solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == lbm.LBM_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": f"large: one instance on a {args.n}^3-cell Kuhn cube, {N} nodes, {nb} surface "
                                   "nodes, random start on the sphere (seed 3), -3 T along z",
                       "n": args.n, "precision": "fp64" if prec == lbm.LBM_FP64 else "mixed",
                       "l2": f"BEM matrix {word * nb * nb / 1e9:.2f} GB > L2"},
            "mesh_setup_s": setup_s, "status": res["status"], "iterations": res["iterations"],
            "evaluations": res["evaluations"], "torque": res["torque"], "energy_J": res["energy"][4],
            "gpu_launches": launches, "clocks": clocks,
            "roofline": {"bound": "hbm", "kernel": "BEM products (forward row GEMV + transposed column GEMV)",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "bytes_per_launch": bem_bytes / max(bem["launches"], 1),
                         "avg_launch_ms": bem["ms"] / max(bem["launches"], 1)},
            "kernel_ms": {k: round(v["ms"], 2) for k, v in kinds.items()},
            "cg_sweeps": prof["cg_sweeps"]}
    print(json.dumps(line), flush=True)


def run_shell(args, ws, rank, local):
    """The bench's batch with the open boundary by space transformation (one
    JSON line; the default line carries the same leg)."""
    import torch
    import paper_1309_5796_gb300 as lbm
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = lbm.Context(local, stream=stream.cuda_stream)
    insts = batched_case(N_CELLS, BATCH, seed=rank_seed(rank))
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.launch_count()
    leg = shell_leg(ctx, local, insts, a=args.shell_a, s=args.shell_s,
                    precision="fp64" if args.precision == "fp64" else "mixed")
    launches = ctx.launch_count() - launches0
    clocks = sampler.stop()
    ctx.close()
    if rank != 0:
        return
    k = leg["shell_solve"]
    line = {"metric": "solves/s, the bench batch with the space-transformation boundary",
            "value": leg["solves_per_s"], "unit": "solves/s", "n_gpus": ws, "steps": 1, "warmup": 1,
            "ms_per_step": leg["ms_to_solution"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": leg["workload"], "n": N_CELLS, "batch": BATCH, "a": args.shell_a,
                       "s": args.shell_s, "l2": "work vectors 6 x grid x batch > L2"},
            "gpu_launches": launches, "clocks": clocks,
            "roofline": {"bound": "hbm", "kernel": k["kernel"], "achieved": k["GB_s"], "peak": None,
                         "unit": "GB/s", "frac": k["frac"], "traffic": k["traffic"],
                         "traffic_source": k["traffic_source"], "bytes_per_launch": k["bytes_per_launch"],
                         "avg_launch_ms": k["avg_launch_ms"], "peak_source": k["peak_source"]},
            "shell": leg}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    line["roofline"]["peak"] = float(peaks.get("hbm_gbs", 6800.0))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "served":
        run_served(args, ws, rank, local)
        return
    if args.workload == "large":
        run_large(args, ws, rank, local)
        return
    if args.workload == "shell":
        run_shell(args, ws, rank, local)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
