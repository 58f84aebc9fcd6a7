"""Autotuner of the solver's execution schedule.

It picks, by timing real solves on the GPU, the choices that change how
fast a solve reaches its tolerance but not what it converges to:

* the block tile (cells per block side: the tree is rebuilt for each),
* the sweep schedule: N_down / N_up red-black sweeps on the fine levels
  (those launched one kernel per phase) and on the coarse levels (those in
  the cooperative launch), which trades cost per V-cycle against cycles,
* the FP32 V-cycles per defect-correction step of the mixed path,
* with several right-hand-side slots, the slots of a block per CTA,
* the CTA size of the block kernels, the block-count limit of the
  cooperative coarse launch and the fused FP32 sweeps.

Every candidate solves the same right-hand sides to the same relative
residual; the score is the wall time of that solve (median of `reps`).
The search is greedy, one knob at a time, in the order above, starting
from the library's defaults.  Results can be cached in a JSON file keyed by
the workload's signature.
"""
from __future__ import annotations

import json
import os
import statistics
import time
from dataclasses import asdict, dataclass, field

from . import FP64, MIXED

__all__ = ["Schedule", "apply", "time_solve", "tune", "tune_block_tile", "signature"]


@dataclass
class Schedule:
    block_n: int = 0                   # 0: as built
    fine_sweeps: tuple = (2, 2)        # (N_down, N_up) on the fine levels
    coarse_sweeps: tuple = (2, 2)      # (N_down, N_up) on the cooperative levels
    cta_threads: int = 0               # 0: by block size
    coop_max_blocks: int = 160
    fused: bool = False
    inner_cycles: int = 1              # FP32 V-cycles per defect-correction step (mixed)
    slots_per_cta: int = 1             # slots of a block per CTA in the half-sweeps
    trials: list = field(default_factory=list, compare=False)

    def key(self):
        return (self.fine_sweeps, self.coarse_sweeps, self.cta_threads, self.coop_max_blocks, self.fused,
                self.inner_cycles, self.slots_per_cta)


def coop_levels(tree, coop_max_blocks):
    """Levels the cooperative launch covers under a block-count limit."""
    split = tree.lmin
    for l in range(tree.lmin, tree.lmax + 1):
        if tree.level_info(l)[0] <= coop_max_blocks:
            split = l
    return split


def apply(tree, s: Schedule):
    tree.set_option("cta_threads", s.cta_threads)
    tree.set_option("coop_max_blocks", s.coop_max_blocks)
    tree.set_option("fused_sweeps", 1 if s.fused else 0)
    tree.set_option("inner_cycles", s.inner_cycles)
    tree.set_option("slots_per_cta", s.slots_per_cta)
    split = coop_levels(tree, s.coop_max_blocks)
    for l in range(tree.lmin, tree.lmax + 1):
        nd, nu = s.coarse_sweeps if l <= split else s.fine_sweeps
        tree.set_level_sweeps(l, nd, nu)


def time_solve(tree, set_rhs, precision, tol, reps=2, max_cycles=80):
    """Median wall time (s) of set_rhs() + solve to tol, after one untimed run;
    None if a solve fails to converge."""
    import torch
    out = []
    for k in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        set_rhs()
        st = tree.solve(precision, tol, max_cycles, check=False)
        torch.cuda.synchronize()
        if st["rc"] != 0:
            return None, st
        if k:
            out.append(time.perf_counter() - t0)
    return statistics.median(out), st


def tune(tree, set_rhs, precision=MIXED, tol=1e-8, reps=2, log=None, axes=None, timer=None):
    """Greedy search over the runtime knobs of a bound tree (or forest)
    (`axes`: names to search, default all).  Returns the best Schedule
    (applied to the tree on return).  `timer(tree, set_rhs, precision, tol,
    reps)` -> (seconds or None, solve stats) scores a candidate (default:
    time_solve, real timed solves)."""
    timer = timer or time_solve
    best = Schedule()
    trials = []
    scored = {}  # schedule key -> seconds: a schedule is timed once

    def score(s):
        if s.key() in scored:
            return scored[s.key()]
        apply(tree, s)
        t, st = timer(tree, set_rhs, precision, tol, reps)
        trials.append(dict(asdict(s) | {"trials": None}, seconds=t, cycles=st.get("cycles")))
        if log:
            log("%-60s %s" % (s.key(), "diverged" if t is None else "%.4f s, %d cycles" % (t, st["cycles"])))
        scored[s.key()] = float("inf") if t is None else t
        return scored[s.key()]

    best_t = score(best)
    space = [
        ("cta_threads", [64, 128, 256]),
        ("fine_sweeps", [(1, 1), (2, 1), (1, 2), (2, 2), (3, 3)]),
        ("coarse_sweeps", [(1, 1), (2, 2), (4, 4)]),
        ("inner_cycles", [1, 2] if precision == MIXED else [1]),
        ("slots_per_cta", [1, 2, 4] if tree.nrhs > 1 else [1]),
        ("coop_max_blocks", [0, 64, 160, 640]),
        ("fused", [False, True]),
    ]
    for name, values in space:
        if axes is not None and name not in axes:
            continue
        for v in values:
            if getattr(best, name) == v:
                continue
            cand = Schedule(**(asdict(best) | {name: v, "trials": []}))
            t = score(cand)
            if t < best_t:
                best, best_t = cand, t
    best.trials = trials
    apply(tree, best)
    return best


def tune_block_tile(build, set_rhs_for, tiles=(8, 16), precision=MIXED, tol=1e-8, reps=2, log=None):
    """Block tile and schedule: build(n) returns a bound tree with n^3 (n^2)
    blocks, set_rhs_for(tree) a function that sets its right-hand sides.
    Each tile is tuned; the fastest (tile, schedule) wins."""
    best, best_t = None, float("inf")
    for n in tiles:
        tree = build(n)
        s = tune(tree, set_rhs_for(tree), precision, tol, reps, log)
        t = min(x["seconds"] for x in s.trials if x["seconds"] is not None)
        s.block_n = n
        if log:
            log("tile %d: best %.4f s" % (n, t))
        if t < best_t:
            best, best_t = s, t
        tree.close()
    return best


def signature(tree, precision, tol):
    """Cache key of a workload: shape of every level, slots, trees, precision."""
    levels = [tree.level_info(l)[:2] for l in range(tree.lmin, tree.lmax + 1)]
    return json.dumps(dict(levels=levels, nrhs=tree.nrhs, ntree=tree.ntree, prec=precision, tol=tol),
                      sort_keys=True)


def load_cached(path, key):
    if not path or not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    v = d.get(key)
    if v is None:
        return None
    v = dict(v)
    v.setdefault("inner_cycles", 1)
    v.setdefault("slots_per_cta", 1)
    v["fine_sweeps"] = tuple(v["fine_sweeps"])
    v["coarse_sweeps"] = tuple(v["coarse_sweeps"])
    v["trials"] = []
    return Schedule(**v)


def store_cached(path, key, s: Schedule):
    d = {}
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
    d[key] = asdict(s) | {"trials": []}
    with open(path, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)


__all__ += ["FP64", "MIXED", "load_cached", "store_cached", "coop_levels"]
