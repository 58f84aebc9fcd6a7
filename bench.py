#!/usr/bin/env python3
"""Benchmark of the octree multigrid solver on the 3D sphere workload.

Workload (seeded, synthetic; the paper's convergence test geometry): the unit
cube with 128^3 cells in 16^3-cell blocks (levels 16^3 .. 128^3 plus an 8^3
coarse level), sphere f = |x - (1/2,1/2,1/2)| - 0.2 with phi = 1 on it, phi = 0
on the walls, g = 0.  One step = one solve from phi = 0 to a relative residual
of 1e-8: the right-hand side set-up and the whole V-cycle path (smoothing,
residual, restriction, FAS right-hand side, coarse solve, prolongation) plus
the convergence tests.

Headline: V-cycle throughput of the mixed-precision solve (FP32 V-cycles in
FP64 defect correction) in million leaf unknowns x V-cycles per second; the
plain FP64 path is timed beside it.  Inputs are resident in HBM at the start
of the timed region; L2 (129 MB) is flushed by writing a 512 MiB buffer
before every timed step.  `e2e` repeats the measurement through the public
API with the right-hand side copied from pinned host memory and the solution
copied back inside the timed region.

Beside the headline, `batched_needle` reports the batched workload: the
adaptive 7-level needle-electrode tree (8^3 blocks, 30,195,712 leaf cells)
holding 32 Gaussian-charge right-hand sides, each step one batched solve of
all 32 to 1e-8 in one tree (mixed and FP64), with its own roofline, and
`batched_forest` the forest of 64 uneven problems (32^3 .. 256^3 cells,
ellipsoids) solved together, after the autotuner has picked the block tile
and sweep schedule on a sample forest, and `serving` the continuous-batching
request loop over seven resident sessions (p50/p99 latency and solves/s,
mixed and FP64), and `paper_table1` the seconds per FMG cycle on the
paper's Table 1 grid (512^3 sphere, 8^3 and 16^3 blocks), FP64, and
`sharp_shapes` the residual reduction per FMG cycle for the sharp
boundaries of Sec. 4.3.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own replica (replicas only: the method
has no cross-problem exchange); the value is the sum over ranks.
"""
import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gmg_inputs as I  # noqa: E402

METRIC = "V-cycle Munk/s"
UNIT = "Munk/s"
WORKLOAD = "sphere3d_128^3_16^3blocks_laplace_mixed_to_1e-8"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--skip-needle", action="store_true", help="leave out the batched needle workload")
    ap.add_argument("--skip-forest", action="store_true", help="leave out the batched uneven-tree workload")
    ap.add_argument("--skip-serving", action="store_true", help="leave out the serving-loop workload")
    ap.add_argument("--skip-table1", action="store_true", help="leave out the 512^3 FMG timing of the paper's Table 1")
    ap.add_argument("--skip-shapes", action="store_true", help="leave out the sharp-boundary FMG runs")
    ap.add_argument("--skip-tuned", action="store_true", help="leave out the autotuned headline solve")
    ap.add_argument("--skip-cpu-baseline", action="store_true",
                    help="leave out the oracle CPU baseline (profiling runs of the GPU legs)")
    ap.add_argument("--only", choices=["needle", "forest", "serving", "table1", "shapes"], default=None,
                    help="run one secondary workload alone (no headline line; for profiling)")
    ap.add_argument("--needle-rhs", type=int, default=32, help="right-hand sides of the batched needle workload")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _allreduce(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allreduce_max(x, world):
    """The largest x over the ranks (the job's time is its slowest replica's)."""
    import torch.distributed as dist
    return _allreduce(x, world, dist.ReduceOp.MAX if world > 1 else None)


def allreduce_sum(x, world):
    """The sum of x over the ranks (work done by all replicas)."""
    import torch.distributed as dist
    return _allreduce(x, world, dist.ReduceOp.SUM if world > 1 else None)


def replica_rate(units, ms, world):
    """Whole-job throughput of independent replicas, in millions per second:
    the units all ranks processed over the slowest rank's time (each rank
    passes its own units and milliseconds)."""
    return allreduce_sum(units, world) / (allreduce_max(ms, world) * 1e-3) / 1e6


def build_tree(G, p):
    t = G.Tree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"],
               max_coarse_cells=p.get("max_coarse_cells") or 0)
    t.set_walls(p["walls"], values=p["wall_values"], fn=p["wall_fn"])
    t.store_stencils(p["lsf"], p["phib"])
    t.bind()
    return t


def coop_split(t):
    """Highest level the cooperative coarse-cycle launch covers (levels with
    at most 160 blocks, the library's rule)."""
    return max(l for l in range(t.lmin, t.lmax + 1) if t.level_info(l)[0] <= 160)


def cluster_top(t):
    """Highest level of the cluster kernel at the bottom of the cycle (the
    library's rule: the single-block levels from the coarsest up, and the
    level of the roots' 2^D children when it holds exactly those)."""
    nroot = t.level_info(t.lmin)[0]
    l = t.lmin
    while l + 1 <= t.lmax and t.level_info(l + 1)[0] == nroot:
        l += 1
    if l + 1 <= coop_split(t) and t.level_info(l + 1)[0] == nroot * 2 ** t.dim:
        l += 1
    return l


# Bytes per cell of one level visit of the V-cycle (Sec. 2.2), S bytes a
# value: the down leg reads phi and b and writes phi (3S), plus the coarse
# level's restricted phi, b and old (3S/8); the up leg reads phi and b and
# writes phi (3S), plus the coarse correction's phi and old (2S/8).
LEVEL_VISIT_S = 3 + 3 / 8 + 3 + 2 / 8


def algorithmic_bytes(kind, prec, level, t, leaf_level, nrhs=1, cluster=False):
    """Minimum bytes one launch of a kernel must move (unique data), for
    nrhs right-hand-side slots (stencils are shared by the slots).  The
    coarse kernels count LEVEL_VISIT_S bytes a cell on every level they
    cover, plus the coarsest-level inverse once; with the cluster kernel at
    the bottom (cluster=True) the cooperative kernel runs twice per cycle
    (down and up leg) and each launch counts half of its levels' bytes."""
    S = 8 if prec == "fp64" else 4
    # BF16 storage (GMG_MIXED_BF16's finest level): phi 2 bytes, b and the
    # coarser level's fields 4 bytes
    Sp = 2 if prec == "bf16" else S
    Sc = 4 if prec == "bf16" else S
    D = t.dim
    if kind in ("coarse_solve", "coarse_cluster"):
        top = cluster_top(t) if cluster else t.lmin - 1
        lo, hi = (t.lmin, top) if kind == "coarse_cluster" else (top + 1, coop_split(t))
        tot = 0.0
        for l in range(lo, hi + 1):
            nb, n, _ = t.level_info(l)
            tot += nrhs * nb * n ** D * LEVEL_VISIT_S * S
        if kind == "coarse_solve" and cluster:
            return tot / 2
        nb0, n0, _ = t.level_info(t.lmin)
        return tot + nb0 * (n0 ** D) ** 2 * 8  # coarsest-level inverses, once
    nb, n, _ = t.level_info(level)
    cells = nb * n ** D * nrhs
    # the cut lists: each listed cell (stencil differs from the regular one)
    # brings its 7 coefficients and its 4-byte index, read once for all slots
    listed = int(t.cut_counts(level).sum())
    entry = 7 * S + 4
    if prec == "bf16":
        entry = 7 * 4 + 4
    if kind == "smooth":  # read the other colour's phi, read b and write phi of one colour; one colour's list
        return cells * (Sp + 0.5 * Sc) + listed * entry / 2
    if kind == "resid_restrict":  # read phi, b; write parent phi, b
        return cells * (Sp + Sc + 2 * Sc / 8) + listed * entry
    if kind == "prolong":  # read/write phi, read parent phi, old
        return cells * (2 * Sp + 2 * Sc / 8)
    if kind == "fas_rhs":  # read phi, b; write b, old
        return cells * 4 * S + listed * entry
    if kind == "resid_norm":  # read phi64, b64 (+ write r32 in the mixed path)
        return cells * (16 + 4) + listed * (7 * 8 + 4)
    if kind in ("level_leg_down", "level_leg_up"):  # one cooperative launch: a leg's sweeps and transfer
        nsw = t.level_sweeps(level)[0 if kind == "level_leg_down" else 1]
        sweeps = 2 * nsw * (cells * (Sp + 0.5 * Sc) + listed * entry / 2)
        if kind == "level_leg_down":
            return sweeps + cells * (Sp + Sc + 2 * Sc / 8) + listed * entry
        return sweeps + cells * (2 * Sp + 2 * Sc / 8)
    if kind == "accumulate":  # read e32, read/write phi64 on the leaf cells of all levels
        if prec == "bf16":  # the finest level's e as BF16 (all its blocks are leaves)
            nbl, nl, _ = t.level_info(t.lmax)
            return nrhs * (t.n_leaf_cells * 20 - nbl * nl ** D * 2)
        return t.n_leaf_cells * nrhs * 20
    return 0


# FP64 arithmetic of this GPU: 152 SMs x 2070 MHz x 2 FP64 FMAs (4 flops) a
# clock per SM = 1.259 TFLOP/s, the nominal 1.25 TFLOP/s (ncu: the FP64 pipe
# takes 16 cycles per warp instruction per SM, i.e. 2 thread operations a
# clock).
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12


def residual_flops(t, level, nrhs):
    """Algorithmic FP64 flops of one residual launch: per cell the sum of
    the 2D neighbours (2D - 1 adds), phi_sum - 2D phi (one FMA) and b - h^-2
    (...) (one FMA), an FMA counted as 2 flops: 9 in 3D, 7 in 2D."""
    nb, n, _ = t.level_info(level)
    D = t.dim
    return nb * n ** D * nrhs * ((2 * D - 1) + 4)


def source_hash():
    """Hash of the library's device code (the .cu, .cuh and .h files of csrc,
    which hold every kernel and its launches); the host-only set-up (.cpp)
    does not enter it."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2205_09411_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_kind, prec, level):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    want = "%s %s %d" % (kernel_kind, prec, level)
    src = source_hash()
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            parts = line.split()
            if len(parts) == 5 and " ".join(parts[:3]) == want and parts[4] == src:
                return float(parts[3])
    return None


def _oracle_vcycles(budget_s):
    """One oracle instance of the 128^3 workload doing FP64 V-cycles from
    phi = 0 until the time budget is used: (cell updates, seconds, cycles).
    Runs in a worker process of cpu_baseline's pool."""
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import gmg_inputs as In
    from _helpers import oracle_problem
    o = oracle_problem(In.problem("c2"))
    n = o.num_leaf_cells()
    k, t0 = 0, time.perf_counter()
    while True:
        o.vcycle(1)
        k += 1
        el = time.perf_counter() - t0
        if el > budget_s or k >= 12:
            break
    o.close()
    return n * k, el, k


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(p, budget_s=8.0):
    """The oracle as it stands (serial FP64 C): V-cycles of the same workload
    from phi = 0, (1) on one host core, and (2) one independent oracle
    instance per host core in a process pool (spawned, so that no worker
    inherits the CUDA context), whose summed cell updates over the slowest
    worker's time give the all-core throughput."""
    import multiprocessing as mp
    units, el, k = _oracle_vcycles(budget_s)
    serial = units / el / 1e6
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_vcycles, [budget_s] * cores)
    total = sum(r[0] for r in res) / max(r[1] for r in res) / 1e6
    return {"value": total, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": "one oracle instance per core (%d processes), each %d-%d FP64 V-cycles of the 128^3 "
                      "workload from phi=0 (about %.0f s each, serial C)" % (cores, min(r[2] for r in res),
                                                                            max(r[2] for r in res), budget_s),
            "serial": {"value": serial, "unit": UNIT, "cores": 1,
                       "sample": "%d FP64 oracle V-cycles of the 128^3 workload from phi=0 (%.1f s, one core)" % (k, el)}}


def run_reference(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _helpers import oracle_problem
    p = I.problem("c2")
    o = oracle_problem(p)
    n = o.num_leaf_cells()
    for _ in range(args.warmup):
        o.vcycle(1)
    o.set_rhs(np.zeros(n))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.vcycle(1)
    el = time.perf_counter() - t0
    v = n * args.steps / el / 1e6
    out = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "step": "one FP64 oracle V-cycle (bounded sample)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "%d serial FP64 oracle V-cycles of the 128^3 workload" % args.steps},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def roofline_of(prof, t, nrhs, peak, peak_kind):
    """Roofline of the kernel with the largest total time in a profiled
    pass: algorithmic bytes per launch / CUDA-event time per launch."""
    by_kind = {}
    for kind, prec, level, cnt, ms in prof:
        by_kind.setdefault((kind, prec), 0.0)
        by_kind[(kind, prec)] += ms
    prof_total = sum(by_kind.values())
    dom_kind, dom_prec = max(by_kind, key=by_kind.get)
    rows = [r for r in prof if r[0] == dom_kind and r[1] == dom_prec]
    lev = max(rows, key=lambda r: r[4])[2]
    row = [r for r in rows if r[2] == lev][0]
    per_launch_ms = row[4] / row[3]
    cluster = any(r[0] == "coarse_cluster" for r in prof)
    alg = algorithmic_bytes(dom_kind, dom_prec, lev, t, t.lmax, nrhs, cluster)
    achieved = alg / (per_launch_ms * 1e-3) / 1e9
    traffic = ncu_traffic(dom_kind, dom_prec, lev)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "%s_%s_level%d" % (dom_kind, dom_prec, lev),
            "per_launch_us": per_launch_ms * 1e3, "algorithmic_bytes": alg,
            "share_of_kernel_time": by_kind[(dom_kind, dom_prec)] / prof_total,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind}
    if dom_kind == "resid_norm" and dom_prec == "fp64":
        # bound by the FP64 pipe, not by HBM: flops against the FP64 peak
        fl = residual_flops(t, lev, nrhs)
        tf = fl / (per_launch_ms * 1e-3) / 1e12
        roof.update({"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": tf / FP64_PEAK_TFLOPS, "algorithmic_flops": fl,
                     "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak},
                     "peak_source": "derived: 152 SMs x 2070 MHz x 4 FP64 flop/clk/SM (the nominal 1.25 TFLOP/s); "
                                    "5 adds and 2 FMAs per cell can fill at most 9/14 of it"})
    return roof, by_kind


def finest_roofline(prof, t, nrhs, peak, peak_kind):
    """HBM roofline of the finest level's half-sweep in a profiled pass (its
    BF16 variant when the pass ran GMG_MIXED_BF16 on that level, else the
    FP32 one): algorithmic bytes per launch / CUDA-event time per launch."""
    rows = [r for r in prof if r[0] == "smooth" and r[2] == t.lmax and r[1] in ("bf16", "fp32")]
    if not rows:
        return None
    row = max(rows, key=lambda r: (r[1] == "bf16", r[4]))
    per_launch_ms = row[4] / row[3]
    alg = algorithmic_bytes("smooth", row[1], t.lmax, t, t.lmax, nrhs)
    achieved = alg / (per_launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "smooth_%s_level%d" % (row[1], t.lmax), "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "per_launch_us": per_launch_ms * 1e3,
            "algorithmic_bytes": alg, "peak_source": peak_kind}


def run_needle(G, args, world, flush, stream):
    """Batched needle workload: the adaptive 7-level needle tree (8^3
    blocks, 30,195,712 leaf cells) with 32 Gaussian-charge right-hand sides
    in one tree, each step one batched solve of all 32 to 1e-8, mixed and
    FP64.  Right-hand sides are generated on the device (seeded)."""
    import torch
    R = args.needle_rhs
    p = I.problem("c3", n_rhs=R)
    t0 = time.perf_counter()
    t = G.Tree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
               max_coarse_cells=p["max_coarse_cells"], w_min=p["w_min"], nrhs=R)
    t.set_walls(p["walls"], values=p["wall_values"], fn=p["wall_fn"])
    t.store_stencils(p["lsf"], p["phib"])
    t.bind()
    setup_s = time.perf_counter() - t0
    n = t.n_leaf_cells
    xc = torch.tensor(t.leaf_centers(), device="cuda")
    g = torch.empty((R, n), dtype=torch.float64, device="cuda")
    for r in range(R):
        g[r] = I.charge_density_torch(xc, p["charges"][r])
    del xc
    torch.cuda.synchronize()

    # schedule: the autotuner's pick of sweeps and FP32 cycles per step for
    # this tree (mixed path), kept for both precisions' timed runs
    from paper_2205_09411_gb300 import autotune as AT
    t1 = time.perf_counter()
    sched = AT.tune(t, lambda: t.set_rhs(g), G.MIXED, args.tol, reps=1,
                    axes=("fine_sweeps", "inner_cycles", "coarse_sweeps", "slots_per_cta"))
    tune_s = time.perf_counter() - t1

    def one(prec, profile=False):
        if profile:
            t.profile(True)
            t.profile_read()
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t.set_rhs(g)
        st = t.solve(prec, args.tol, 60)
        e1.record(stream)
        e1.synchronize()
        prof = None
        if profile:
            prof = t.profile_read()
            t.profile(False)
        return e0.elapsed_time(e1), st, t.last_launch_count() + 1, prof

    res = {}
    for name, prec in (("mixed", G.MIXED), ("mixed_bf16", G.MIXED_BF16), ("fp64", G.FP64)):
        one(prec)  # warm-up (graph capture)
        barrier(world)
        times, cyc, worst, launches = [], 0, 0.0, 0
        for _ in range(max(1, args.steps)):
            ms, st, nl, _ = one(prec)
            times.append(ms)
            cyc += sum(x["cycles"] for x in st["slots"])
            worst = max(worst, st["rel_l2"])
            launches += nl
        total = allreduce_max(sum(times), world)
        ts = sorted(times)
        vc = cyc * (sched.inner_cycles if prec != G.FP64 else 1)  # V-cycles (FP32 ones in the mixed path)
        res[name] = {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                     "solves_per_s": world * R * len(ts) / (total * 1e-3),
                     "munks": world * n * vc / (total * 1e-3) / 1e6,
                     "steps_per_solve": cyc / (R * len(ts)), "v_cycles_per_solve": vc / (R * len(ts)),
                     "worst_final_rel_residual": worst, "gpu_launches_per_batch": launches / len(ts)}
    _, _, _, prof = one(G.MIXED, profile=True)
    _, _, _, prof_bf = one(G.MIXED_BF16, profile=True)
    peak, peak_kind = peaks()
    roof, by_kind = roofline_of(prof, t, R, peak, peak_kind)
    roof_bf, _ = roofline_of(prof_bf, t, R, peak, peak_kind)
    res["mixed_bf16"]["roofline"] = roof_bf
    res["mixed_bf16"]["finest_level_kernels_us_per_launch"] = {
        "%s_%s_l%d" % (k, p_, lv): round(ms * 1e3 / cnt, 2) for k, p_, lv, cnt, ms in prof_bf if p_ == "bf16"}
    res["mixed_bf16"]["finest_level_roofline"] = finest_roofline(prof_bf, t, R, peak, peak_kind)
    out = {"workload": "needle3d_adaptive_7levels_8^3blocks_%drhs_gaussian_mixed_to_1e-8" % R, "unknowns": n,
           "rhs": R, "blocks": t.n_blocks, "levels": [t.lmin, t.lmax], "setup_s": setup_s,
           "latency_is": "one batched solve of all %d right-hand sides from phi = 0" % R,
           "mixed": res["mixed"], "mixed_bf16": res["mixed_bf16"], "fp64": res["fp64"], "roofline": roof,
           "autotuned": {"fine_sweeps": list(sched.fine_sweeps), "coarse_sweeps": list(sched.coarse_sweeps),
                         "inner_cycles": sched.inner_cycles, "slots_per_cta": sched.slots_per_cta,
                         "trials": len(sched.trials), "tuning_s": tune_s},
           "kernel_ms_by_kind": {"%s_%s" % k: v for k, v in sorted(by_kind.items(), key=lambda kv: -kv[1])},
           "kernel_us_per_launch": {"%s_%s_l%d" % (k, p_, lv): round(ms * 1e3 / cnt, 2)
                                    for k, p_, lv, cnt, ms in prof}}
    t.close()
    del g
    torch.cuda.empty_cache()
    return out


def host_tree(G, p, N=None, nrhs=1):
    """Set-up tree (walls, stencils), not bound."""
    N = N or p["N"]
    h1 = p["h1"] if N == p["N"] else 1.0 / N
    t = G.Tree(p["dim"], N, p["cb"], p["lo"], h1, p["max_level"], refine=p["refine"],
               max_coarse_cells=p.get("max_coarse_cells") or 0, w_min=p.get("w_min", 0.0), nrhs=nrhs)
    t.set_walls(p["walls"], values=p["wall_values"], fn=p["wall_fn"])
    t.store_stencils(p["lsf"], p["phib"])
    return t


def forest_of(G, ps, N, threads=16, times=None):
    """Forest of the problems with N^3 blocks; the trees' set-up calls run
    in parallel threads (they release the GIL; the boundary detection of
    the built-in level sets runs on the device).  times: a dict that
    receives the seconds of the trees' set-up and of the forest's creation
    and binding."""
    from concurrent.futures import ThreadPoolExecutor
    qs = [dict(p, max_level=int(round(np.log2(p["n"] / N))) + 1) for p in ps]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        trees = list(ex.map(lambda p: host_tree(G, p, N), qs))
    t1 = time.perf_counter()
    F = G.Forest(trees)
    F.bind()
    if times is not None:
        times["trees_s"] = t1 - t0
        times["forest_and_bind_s"] = time.perf_counter() - t1
        times["boundary_detection"] = "device" if all(t.setup_on_device() for t in trees) else "host"
    return F, trees, qs


def forest_rhs_device(F, trees, qs, N):
    import torch
    g = torch.empty(F.n_leaf_cells, dtype=torch.float64, device="cuda")
    for i, (t, q) in enumerate(zip(trees, qs)):
        off, n = F.tree_leaves(i)
        bix, _ = t.level_blocks(t.lmax)
        g[off:off + n] = I.box_noise_rhs_torch(bix, N, q["n"], q["noise_seed"])
    return g


def run_forest(G, args, world, flush, stream):
    """Batched uneven trees: 64 independent problems (n^3, n in {32, 64,
    128, 256}, ellipsoids, random Dirichlet values, box-filtered noise) in
    one forest, each step one solve of all 64 to 1e-8; block tile and sweep
    schedule picked first by the autotuner on a sample forest of 8 problems
    drawn from the same distribution."""
    import torch
    from paper_2205_09411_gb300 import autotune as AT
    t0 = time.perf_counter()
    sample = I.forest_problems(8, index=4)
    log_lines = []

    def build(N):
        F, trees, qs = forest_of(G, sample, N)
        F._rhs = forest_rhs_device(F, trees, qs, N)
        return F

    best = AT.tune_block_tile(build, lambda F: (lambda: F.set_rhs(F._rhs)), tiles=(8, 16), precision=G.MIXED,
                              tol=args.tol, reps=1, log=log_lines.append)
    tune_s = time.perf_counter() - t0
    N = best.block_n
    t0 = time.perf_counter()
    setup_parts = {}
    F, trees, qs = forest_of(G, I.forest_problems(64, index=3), N, times=setup_parts)
    AT.apply(F, best)
    t1 = time.perf_counter()
    g = forest_rhs_device(F, trees, qs, N)
    setup_parts["rhs_s"] = time.perf_counter() - t1
    setup_s = time.perf_counter() - t0
    n = F.n_leaf_cells
    sizes = [q["n"] for q in qs]
    del trees
    res = {}
    for name, prec in (("mixed", G.MIXED), ("mixed_bf16", G.MIXED_BF16), ("fp64", G.FP64)):
        F.set_rhs(g)
        F.solve(prec, args.tol, 80)  # warm-up (graph capture)
        barrier(world)
        times, munk_cyc, worst = [], 0, 0.0
        for _ in range(max(1, args.steps)):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            F.set_rhs(g)
            st = F.solve(prec, args.tol, 80)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            for i, u in enumerate(st["units"]):
                off, cnt = F.tree_leaves(i)
                munk_cyc += cnt * u["cycles"] * (best.inner_cycles if prec != G.FP64 else 1)
            worst = max(worst, st["rel_l2"])
        total = allreduce_max(sum(times), world)
        ts = sorted(times)
        res[name] = {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                     "solves_per_s": world * 64 * len(ts) / (total * 1e-3),
                     "munks": world * munk_cyc / (total * 1e-3) / 1e6,
                     "worst_final_rel_residual": worst}
    profs = {}
    for prec in (G.MIXED, G.MIXED_BF16):
        F.profile(True)
        F.profile_read()
        F.set_rhs(g)
        F.solve(prec, args.tol, 80)
        profs[prec] = F.profile_read()
        F.profile(False)
    prof = profs[G.MIXED]
    peak, peak_kind = peaks()
    roof, by_kind = roofline_of(prof, F, 1, peak, peak_kind)
    res["mixed_bf16"]["finest_level_roofline"] = finest_roofline(profs[G.MIXED_BF16], F, 1, peak, peak_kind)
    res["mixed_bf16"]["finest_level_roofline_fp32_state"] = finest_roofline(prof, F, 1, peak, peak_kind)
    out = {"workload": "forest_64_uniform_trees_32^3-256^3_ellipsoids_mixed_to_1e-8", "unknowns": n,
           "trees": 64, "tree_sizes": {str(k): sizes.count(k) for k in sorted(set(sizes))},
           "latency_is": "one solve of all 64 problems (each to its own 1e-8) from phi = 0",
           "autotuned": {"block_n": N, "fine_sweeps": list(best.fine_sweeps),
                         "coarse_sweeps": list(best.coarse_sweeps), "cta_threads": best.cta_threads,
                         "coop_max_blocks": best.coop_max_blocks, "fused": best.fused,
                         "inner_cycles": best.inner_cycles,
                         "tuning_s": tune_s, "trials": len(best.trials),
                         "sample": "8 problems of the same distribution (seed index 4), tiles 8 and 16"},
           "setup_s": setup_s, "setup_parts": setup_parts, "mixed": res["mixed"], "mixed_bf16": res["mixed_bf16"],
           "fp64": res["fp64"], "roofline": roof,
           "kernel_ms_by_kind": {"%s_%s" % k: v for k, v in sorted(by_kind.items(), key=lambda kv: -kv[1])}}
    F.close()
    del g
    torch.cuda.empty_cache()
    return out


def run_serving(G, args, world):
    """Serving loop: Poisson arrivals of Gaussian-charge right-hand sides for
    seven resident sessions (the 2D circle at 512^2, spheres at 64^3, 128^3
    and 256^3, the needle at 5, 6 and 7 levels), 8 slots each, HBM budget
    160 GB; continuous batching (serving.Server).  Sessions are loaded and
    their graphs captured by a warm-up request each, then the autotuner picks
    each session's sweep schedule; the timed run serves a fresh seeded
    stream, mixed and FP64, then the same stream at ten times the rate (the
    loop's capacity)."""
    import torch
    from paper_2205_09411_gb300.serving import Request, Server, Session, poisson_arrivals, summarize
    specs = {"circle2d_512": I.problem("c1", max_level=7),
             "sphere_64": I.problem("c2", max_level=3),
             "sphere_128": I.problem("c2"),
             "sphere_256": I.problem("c2", max_level=5),
             "needle_5lev": I.problem("c3", max_level=5, n_rhs=1),
             "needle_6lev": I.problem("c3", max_level=6, n_rhs=1),
             "needle_7lev": I.problem("c3", max_level=7, n_rhs=1)}
    t0 = time.perf_counter()
    sessions = [Session(name, make=lambda slots, p=p: host_tree(G, p, nrhs=slots)) for name, p in specs.items()]

    def on_load(s):
        s.ctx["xc"] = torch.tensor(s.tree.leaf_centers(), device="cuda")
        s.ctx["out"] = torch.empty((1, s.tree.n_leaf_cells), dtype=torch.float64, device="cuda")

    def result_to(s, slot):  # the solution gathered into a device buffer
        s.tree.solution_slots(slot, 1, out=s.ctx["out"], stream=s.stream)
        return None

    names = list(specs)
    n_req, rate = 160, 60.0
    charges = I.gaussian_charges(n_req + len(names), 5)
    pick = I.rng_for(6).integers(len(names), size=n_req)
    arrive = poisson_arrivals(rate, n_req, 7)

    def req(i, name, at):
        return Request(name, lambda s, c=charges[i]: I.charge_density_torch(s.ctx["xc"], c), at)

    from paper_2205_09411_gb300 import autotune as AT
    out = {"sessions": {}, "rate_per_s": rate, "requests": n_req, "slots_per_session": 8, "budget_gb": 160.0,
           "schedules_mixed": {}, "schedules_fp64": {}}
    for label, prec in (("mixed", G.MIXED), ("fp64", G.FP64)):
        srv = Server(sessions, budget_bytes=160e9, slots=8, precision=prec, tol=args.tol, on_load=on_load,
                     new_stream=lambda: torch.cuda.Stream(), result_to=result_to,
                     stream_context=lambda s: torch.cuda.stream(s.stream))
        srv.run([req(n_req + k, name, 0.0) for k, name in enumerate(names)])  # load + graph capture
        torch.cuda.synchronize()
        # each session's sweep schedule (and, mixed, FP32 cycles per step) by
        # the autotuner, on a sample right-hand side in all its slots
        t1 = time.perf_counter()
        for k, s_ in enumerate(sessions):
            g_ = I.charge_density_torch(s_.ctx["xc"], charges[n_req + k]).repeat(8, 1).contiguous()
            sched = AT.tune(s_.tree, lambda: s_.tree.set_rhs(g_), prec, args.tol, reps=1,
                            axes=("fine_sweeps", "coarse_sweeps", "inner_cycles", "slots_per_cta"))
            out["schedules_%s" % label][s_.name] = {"fine_sweeps": list(sched.fine_sweeps),
                                                     "coarse_sweeps": list(sched.coarse_sweeps),
                                                     "inner_cycles": sched.inner_cycles,
                                                     "slots_per_cta": sched.slots_per_cta}
        out["tuning_s_%s" % label] = time.perf_counter() - t1
        srv.run([req(n_req + k, name, 0.0) for k, name in enumerate(names)])  # graphs of the tuned schedules
        torch.cuda.synchronize()
        done = srv.run([req(i, names[int(pick[i])], float(arrive[i])) for i in range(n_req)])
        torch.cuda.synchronize()
        out[label] = summarize(done) | {"resident_gb": max(srv.peak_bytes, srv.resident_bytes()) / 1e9}
        # the same requests arriving ten times faster: the loop's capacity
        done = srv.run([req(i, names[int(pick[i])], float(arrive[i]) / 10) for i in range(n_req)])
        torch.cuda.synchronize()
        out[label + "_at_10x_rate"] = summarize(done)
    for s in sessions:
        if s.resident:
            out["sessions"][s.name] = {"leaf_cells": s.tree.n_leaf_cells, "workspace_gb": s.nbytes / 1e9}
            s.tree.close()
            s.tree = None
    out["setup_and_run_s"] = time.perf_counter() - t0
    torch.cuda.empty_cache()
    return out


PAPER_TABLE1_S_PER_FMG = {8: {4: 5.55, 8: 2.77, 16: 1.62, 32: 1.46}, 16: {4: 2.97, 8: 1.53, 16: 1.01, 32: 0.95},
                          32: {4: 2.36, 8: 1.31, 16: 0.87, 32: 0.84}}


def run_table1(G, args, world, stream):
    """The timing workload of the paper's Table 1: the Sec. 4.1 sphere
    geometry (domain [-1/2, 1/2]^3, sphere R = 1/4) on a uniform 512^3 grid
    (134,217,728 cells), seconds per FMG cycle in FP64, with 8^3 and 16^3
    blocks.  Boundary values here: phi = 1 on the sphere, 0 on the walls
    (the timing does not depend on them).  The paper's times (Fortran/OpenMP
    on an AMD EPYC 7H12, 4-32 cores) are quoted beside it as context."""
    import torch
    out = {"workload": "sphere3d_512^3_uniform_fmg_fp64", "cells": 512 ** 3, "blocks": {}}
    for N in (8, 16):
        ml = int(round(np.log2(512 / N))) + 1
        p = I.problem("sphere3d", N=N, h1=1.0 / N, max_level=ml, wall_fn=None, wall_values=(0.0,) * 6, phib=1.0)
        t0 = time.perf_counter()
        t = host_tree(G, p)
        t.bind()
        setup = time.perf_counter() - t0
        t.set_rhs(torch.zeros(t.n_leaf_cells, dtype=torch.float64, device="cuda"))
        t.fmg(1)  # warm-up and graph capture
        t.set_rhs(torch.zeros(t.n_leaf_cells, dtype=torch.float64, device="cuda"))
        r0, _ = t.residual()
        k = max(2, min(args.steps, 4))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        t.fmg(k)
        e1.record(stream)
        e1.synchronize()
        per = e0.elapsed_time(e1) / k * 1e-3
        r1, _ = t.residual()
        # time to a 1e-8 relative residual from phi = 0: V-cycle or FMG steps,
        # FP64 or mixed (FP32 cycles in FP64 defect correction)
        to_tol = {}
        for cyc, fmg in (("vcycle", 0), ("fmg", 1)):
            t.set_option("fmg_steps", fmg)
            for name, prec in (("fp64", G.FP64), ("mixed", G.MIXED)):
                zero = torch.zeros(t.n_leaf_cells, dtype=torch.float64, device="cuda")
                t.set_rhs(zero)
                t.solve(prec, args.tol, 60)  # graph capture
                t.set_rhs(zero)
                torch.cuda.synchronize()
                e0.record(stream)
                st = t.solve(prec, args.tol, 60)
                e1.record(stream)
                e1.synchronize()
                to_tol["%s_%s" % (name, cyc)] = {"ms": e0.elapsed_time(e1), "steps": st["cycles"],
                                                 "rel_residual": st["rel_l2"]}
        t.set_option("fmg_steps", 0)
        out["blocks"]["%d^3" % N] = {"s_per_fmg_cycle": per, "munk_fmg_per_s": 512 ** 3 / per / 1e6,
                                     "levels": [t.lmin, t.lmax], "fmg_cycles_timed": k,
                                     "rel_residual_after": r1, "reduction_per_cycle": (r0 / r1) ** (1.0 / k),
                                     "solve_to_tol": to_tol, "setup_s": setup,
                                     "paper_s_per_fmg_cycle_by_cores": PAPER_TABLE1_S_PER_FMG.get(N)}
        t.close()
        torch.cuda.empty_cache()
    out["paper_best_s_per_fmg_cycle"] = 0.84
    out["paper_hardware"] = "AMD EPYC 7H12, 32 cores, 32^3 blocks (Table 1)"
    return out


def run_shapes(G, args, world, stream):
    """Sharp boundaries of Sec. 4.3 (spheroid, rhombus, heart, astroid):
    residual reduction per FMG cycle from phi = 0 on uniform 1024^2 and
    2048^2 grids (8^2 coarse grid, w_min = 4e-3) and, revolved, on 256^3
    (8^3 coarse grid, w_min = 8e-3), FP64, with the time per FMG cycle.  The
    paper shows these reductions as a figure (no printed numbers); it notes
    that the astroid's is lowest and changes with the refinement level."""
    import torch
    out = {}
    for dim, ml, label in ((2, 8, "1024^2"), (2, 9, "2048^2"), (3, 6, "256^3")):
        for shape in I.SHAPES:
            p = I.sharp_problem(shape, dim, ml)
            t = host_tree(G, p)
            t.bind()
            t.set_rhs(torch.zeros(t.n_leaf_cells, dtype=torch.float64, device="cuda"))
            r = [t.residual()[0]]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            times = []
            for k in range(4):
                e0.record(stream)
                t.fmg(1)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                r.append(t.residual()[0])
            out["%s_%s" % (shape, label)] = {"reduction_per_fmg": [r[k] / r[k + 1] for k in range(4)],
                                             "rel_residual": r[-1], "ms_per_fmg_cycle": float(np.median(times[1:])),
                                             "cells": t.n_leaf_cells}
            t.close()
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import paper_2205_09411_gb300 as G
    world, rank, local = dist_setup(args.gpus)
    assert torch.cuda.is_available(), "bench needs a CUDA device"
    torch.cuda.set_device(local)
    G.build()
    if args.only:  # one secondary workload alone (profiling runs)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        leg = {"needle": lambda: run_needle(G, args, world, flush, stream),
               "forest": lambda: run_forest(G, args, world, flush, stream),
               "serving": lambda: run_serving(G, args, world),
               "table1": lambda: run_table1(G, args, world, stream),
               "shapes": lambda: run_shapes(G, args, world, stream)}[args.only]()
        if rank == 0:
            print(json.dumps({"only": args.only, args.only: leg}))
        return
    p = I.problem("c2")
    t_setup = time.perf_counter()
    t = build_tree(G, p)
    t_setup = time.perf_counter() - t_setup
    n = t.n_leaf_cells
    g = np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64)
    g_dev = torch.tensor(g, device="cuda")
    g_pin = torch.tensor(g).pin_memory()
    out_pin = torch.zeros(n, dtype=torch.float64).pin_memory()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def solve(prec):
        t.set_rhs(g_dev)
        st = t.solve(prec, args.tol, 60)
        return st, t.last_launch_count() + 1

    for _ in range(args.warmup):
        solve(G.MIXED)
        solve(G.FP64)
    torch.cuda.synchronize()

    def timed(prec, profile=False, e2e=False):
        times, cycles, launches = [], 0, 0
        if profile:
            t.profile(True)
            t.profile_read()
        barrier(world)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if e2e:
                t.set_rhs(g_pin)
                st = t.solve(prec, args.tol, 60)
                t.solution(out_pin)
                nl = t.last_launch_count() + 2
            else:
                st, nl = solve(prec)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            cycles += st["cycles"]
            launches += nl
        torch.cuda.synchronize()
        barrier(world)
        prof = t.profile_read() if profile else None
        if profile:
            t.profile(False)
        total = allreduce_max(sum(times), world)
        return dict(times=times, total_ms=total, cycles=cycles, launches=launches, prof=prof, rel=st["rel_l2"])

    clocks = Clocks(local)
    clocks.start()
    mixed = timed(G.MIXED)
    clk = clocks.stop()
    fp64 = timed(G.FP64)
    e2e = timed(G.MIXED, e2e=True)
    for _ in range(args.warmup):
        solve(G.MIXED_BF16)
    bf16 = timed(G.MIXED_BF16)
    bf16["prof"] = timed(G.MIXED_BF16, profile=True)["prof"]
    # kernel durations: the same steps again with CUDA events around every
    # kernel (each phase is queued behind a short delay kernel, so the events
    # time the kernels and not the host)
    mixed["prof"] = timed(G.MIXED, profile=True)["prof"]

    def munks(r):  # r["total_ms"] is already the maximum over the ranks
        return replica_rate(n * r["cycles"], r["total_ms"], world)

    def lat(r):
        ts = sorted(r["times"])
        return {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                "solves_per_s": world * len(ts) / (r["total_ms"] * 1e-3), "cycles_per_solve": r["cycles"] / len(ts)}

    # roofline of the dominant kernel (largest total time in the timed region)
    peak, peak_kind = peaks()
    roofline, by_kind = roofline_of(mixed["prof"], t, 1, peak, peak_kind)

    result = {
        "metric": METRIC, "value": munks(mixed), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mixed["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "unknowns": n, "block": "16^3", "levels": [t.lmin, t.lmax],
                   "cut_blocks_finest": t.num_cut_blocks(t.lmax), "tol": args.tol,
                   "l2": "flushed before every timed step (512 MiB write)", "parallelism": "replicas",
                   "setup_s": t_setup},
        "mixed": lat(mixed) | {"munks": munks(mixed), "final_rel_residual": mixed["rel"]},
        "fp64": lat(fp64) | {"munks": munks(fp64), "final_rel_residual": fp64["rel"]},
        "mixed_bf16": lat(bf16) | {"munks": munks(bf16), "final_rel_residual": bf16["rel"],
                                   "finest_level_roofline": finest_roofline(bf16["prof"], t, 1, peak, peak_kind),
                                   "finest_level_kernels_us_per_launch": {
                                       "%s_%s_l%d" % (k, p_, lv): round(ms * 1e3 / cnt, 2)
                                       for k, p_, lv, cnt, ms in bf16["prof"] if p_ == "bf16"}},
        "e2e": {"value": munks(e2e), "unit": UNIT, "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": mixed["launches"],
        "roofline": roofline,
        "kernel_ms_by_kind": {"%s_%s" % k: v for k, v in sorted(by_kind.items(), key=lambda kv: -kv[1])},
        "kernel_us_per_launch": {"%s_%s_l%d" % (k, p_, lv): round(ms * 1e3 / cnt, 2)
                                 for k, p_, lv, cnt, ms in mixed["prof"]},
        "clocks": clk,
    }
    if not args.skip_tuned:
        # the same solve with the autotuner's schedule for this tree (sweeps per
        # level group, FP32 cycles per step, CTA size, cooperative block limit);
        # the headline above keeps the paper's 2 + 2 sweeps on every level
        from paper_2205_09411_gb300 import autotune as AT
        t1 = time.perf_counter()
        sched = AT.tune(t, lambda: t.set_rhs(g_dev), G.MIXED, args.tol, reps=2)
        tune_s = time.perf_counter() - t1
        for _ in range(args.warmup):
            solve(G.MIXED)
        tuned = timed(G.MIXED)
        tv = tuned["cycles"] * sched.inner_cycles
        result["tuned"] = lat(tuned) | {
            "munks": world * n * tv / (tuned["total_ms"] * 1e-3) / 1e6, "final_rel_residual": tuned["rel"],
            "v_cycles_per_solve": tv / len(tuned["times"]), "schedule": {
                "fine_sweeps": list(sched.fine_sweeps), "coarse_sweeps": list(sched.coarse_sweeps),
                "inner_cycles": sched.inner_cycles, "cta_threads": sched.cta_threads,
                "coop_max_blocks": sched.coop_max_blocks, "fused": sched.fused}, "tuning_s": tune_s}
    t.close()
    if not args.skip_needle:
        result["batched_needle"] = run_needle(G, args, world, flush, stream)
    if not args.skip_forest:
        result["batched_forest"] = run_forest(G, args, world, flush, stream)
    if not args.skip_serving:
        result["serving"] = run_serving(G, args, world)
    if not args.skip_table1:
        result["paper_table1"] = run_table1(G, args, world, stream)
    if not args.skip_shapes:
        result["sharp_shapes"] = run_shapes(G, args, world, stream)
    if rank == 0 and world == 1 and not args.skip_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(p)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
