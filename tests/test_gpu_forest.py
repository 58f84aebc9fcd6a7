"""Forests: many independent trees (uneven sizes, their own level sets and
boundary values) in every launch of one V-cycle.

Each tree of a forest must behave exactly like the same tree solved alone:
its FP64 iterates match the oracle run on that tree (1e-12), and a forest
solve, FP64 or mixed, with one or several right-hand-side slots, gives
every (slot, tree) unit bit for bit the solution and cycle count of a solo
solve.
"""
import numpy as np
import pytest

import gmg_inputs as I
from _helpers import gpu_problem, oracle_problem, parity_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09411_gb300 as G
    G.build()


def problems():
    return I.forest_problems(5, index=7, sizes=(16, 32, 64))


def make_forest(ps, nrhs=1):
    import paper_2205_09411_gb300 as G
    trees = [gpu_problem(p, bind=False) for p in ps]
    F = G.Forest(trees, nrhs=nrhs)
    F.bind()
    return F, trees


def forest_rhs(F, ps, trees, scale=1.0):
    g = np.zeros(F.n_leaf_cells)
    for i, (p, t) in enumerate(zip(ps, trees)):
        off, n = F.tree_leaves(i)
        g[off:off + n] = scale * p["rhs"](t.leaf_centers())
    return g


def test_forest_iterates_match_oracle_per_tree():
    ps = problems()
    F, trees = make_forest(ps)
    F.set_rhs(forest_rhs(F, ps, trees))
    oracles = [oracle_problem(p) for p in ps]
    for k in range(3):
        F.vcycle(1)
        got = F.solution()
        for i, o in enumerate(oracles):
            o.vcycle(1)
            ref = o.solution()
            off, n = F.tree_leaves(i)
            err = np.abs(got[off:off + n] - ref).max() / np.abs(ref).max()
            assert err <= 1e-12, "tree %d cycle %d: %.3e" % (i, k + 1, err)
    rel, _ = F.residual()
    for i, o in enumerate(oracles):
        l2, _, bn = o.residual()
        assert abs(rel[i] - l2 / bn) <= 1e-6 * (l2 / bn) + 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_forest_solve_equals_solo_solves(prec):
    import paper_2205_09411_gb300 as G
    P = G.FP64 if prec == "fp64" else G.MIXED
    ps = problems()
    R = 2
    F, trees = make_forest(ps, nrhs=R)
    g = np.stack([forest_rhs(F, ps, trees), forest_rhs(F, ps, trees, -0.5)])
    F.set_rhs(g)
    st = F.solve(P, 1e-8, 60)
    phi = F.solution()
    for i, p in enumerate(ps):
        off, n = F.tree_leaves(i)
        for r in range(R):
            t = gpu_problem(p, rhs=False)
            t.set_rhs(g[r, off:off + n].copy())
            st1 = t.solve(P, 1e-8, 60)
            u = r * F.ntree + i
            assert st["units"][u]["cycles"] == st1["cycles"], (i, r)
            assert st["units"][u]["rel_l2"] == st1["rel_l2"], (i, r)
            assert np.array_equal(phi[r, off:off + n], t.solution()), "tree %d slot %d" % (i, r)


def test_forest_rejects_mismatched_trees():
    import paper_2205_09411_gb300 as G
    ps = problems()
    a = gpu_problem(ps[0], bind=False)
    q = dict(ps[1])
    q["walls"] = (1, 0, 0, 0, 0, 0)  # a Neumann wall: wall types differ
    b = gpu_problem(q, bind=False)
    with pytest.raises(G.GmgError):
        G.Forest([a, b])
    c = gpu_problem(ps[2])  # bound
    with pytest.raises(G.GmgError):
        G.Forest([a, c])


def test_sweep_schedule_default_is_unchanged_and_others_converge():
    """Setting every level's sweeps to the parameters' (2, 2) gives the same
    iterates bit for bit; a level-dependent schedule (1 + 1 on the fine
    levels, 4 + 4 on the coarse ones) still solves to 1e-8 by the oracle's
    own residual."""
    import paper_2205_09411_gb300 as G
    p = problems()[4]
    a = gpu_problem(p)
    b = gpu_problem(p)
    for l in range(b.lmin, b.lmax + 1):
        b.set_level_sweeps(l, 2, 2)
    a.vcycle(3)
    b.vcycle(3)
    assert np.array_equal(a.solution(), b.solution())
    for l in range(b.lmin, b.lmax + 1):
        b.set_level_sweeps(l, *((1, 1) if l == b.lmax else (4, 4)))
    assert b.level_sweeps(b.lmax) == (1, 1)
    b.set_rhs(np.asarray(p["rhs"](b.leaf_centers()), dtype=np.float64))
    st = b.solve(G.MIXED, 1e-8, 80)
    o = oracle_problem(p)
    o.set_solution(b.solution())
    l2, _, bn = o.residual()
    assert st["rel_l2"] <= 1e-8 and l2 / bn <= 1.05e-8


def test_autotuner_returns_a_converging_schedule():
    import paper_2205_09411_gb300 as G
    from paper_2205_09411_gb300 import autotune as AT
    ps = problems()[:3]
    F, trees = make_forest(ps)
    g = forest_rhs(F, ps, trees)
    s = AT.tune(F, lambda: F.set_rhs(g), G.MIXED, 1e-8, reps=1)
    assert len(s.trials) >= 10
    assert all(x["seconds"] is None or x["seconds"] > 0 for x in s.trials)
    F.set_rhs(g)
    st = F.solve(G.MIXED, 1e-8, 80)
    assert st["rel_l2"] <= 1e-8
    split = AT.coop_levels(F, s.coop_max_blocks)
    for l in range(F.lmin, F.lmax + 1):
        assert F.level_sweeps(l) == tuple(s.coarse_sweeps if l <= split else s.fine_sweeps)


def test_inner_cycles_converge_with_fewer_steps():
    """Two FP32 V-cycles per defect-correction step: the mixed solve still
    meets 1e-8 by the oracle's own residual, in no more steps than with one."""
    import paper_2205_09411_gb300 as G
    p = problems()[3]
    g = None
    steps = []
    for inner in (1, 2):
        t = gpu_problem(p, rhs=False)
        g = np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64)
        t.set_option("inner_cycles", inner)
        t.set_rhs(g)
        st = t.solve(G.MIXED, 1e-8, 80)
        steps.append(st["cycles"])
        o = oracle_problem(p)
        o.set_solution(t.solution())
        l2, _, bn = o.residual()
        assert st["rel_l2"] <= 1e-8 and l2 / bn <= 1.05e-8
    assert steps[1] <= steps[0]


def test_remesh_tree_solves_like_a_fresh_tree_and_transfer_helps():
    """A re-meshed tree (needle, one level deeper) gives bit for bit the
    V-cycle iterates of the same tree set up from scratch, and the previous
    solution transferred to it as the initial guess needs fewer cycles than
    phi = 0."""
    import paper_2205_09411_gb300 as G
    p4 = I.problem("c3", max_level=4, n_rhs=1)
    p5 = I.problem("c3", max_level=5, n_rhs=1)
    old = gpu_problem(p4)
    old.solve(G.FP64, 1e-10, 80)
    new = old.remesh(p5["refine"], 5)
    new.bind()
    ref = gpu_problem(p5)
    g = np.asarray(p5["rhs"](new.leaf_centers()), dtype=np.float64)
    for t in (new, ref):
        t.set_rhs(g)
        t.vcycle(3)
    assert np.array_equal(new.solution(), ref.solution())
    new.set_rhs(g)
    st0 = new.solve(G.FP64, 1e-8, 80)
    new.set_rhs(g)
    new.transfer_solution_from(old)
    st1 = new.solve(G.FP64, 1e-8, 80)
    assert st1["cycles"] < st0["cycles"], (st1, st0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fmg_steps_solve(prec):
    """Solve steps made of FMG cycles (FP64, or FP32 FMG inside the mixed
    defect correction) reach 1e-8 by the oracle's own residual, in fewer
    steps than V-cycle steps at most."""
    import paper_2205_09411_gb300 as G
    P = G.FP64 if prec == "fp64" else G.MIXED
    p = parity_cases()["adaptive3d"]
    steps = {}
    for fmg in (0, 1):
        t = gpu_problem(p)
        t.set_option("fmg_steps", fmg)
        st = t.solve(P, 1e-8, 80)
        steps[fmg] = st["cycles"]
        o = oracle_problem(p)
        o.set_solution(t.solution())
        l2, _, bn = o.residual()
        assert st["rel_l2"] <= 1e-8 and l2 / bn <= 1.05e-8
    assert steps[1] <= steps[0], steps


def test_forest_256_tree_at_the_tuned_schedule_matches_oracle():
    """The batched-trees workload's largest member: a 256^3 ellipsoid tree in
    a forest of 16^3-cell blocks run with 128-thread CTAs (the schedule the
    autotuner picks for that workload), beside a 32^3 and a 64^3 tree; FP64
    iterates of every tree against the oracle after each of 3 V-cycles."""
    ps = I.forest_problems(3, index=4, sizes=(256,), N=16)
    ps[1] = I.forest_problems(1, index=5, sizes=(32,), N=16)[0]
    ps[2] = I.forest_problems(1, index=6, sizes=(64,), N=16)[0]
    F, trees = make_forest(ps)
    F.set_option("cta_threads", 128)
    F.set_rhs(forest_rhs(F, ps, trees))
    oracles = [oracle_problem(p) for p in ps]
    for k in range(3):
        F.vcycle(1)
        got = F.solution()
        for i, o in enumerate(oracles):
            o.vcycle(1)
            ref = o.solution()
            off, n = F.tree_leaves(i)
            err = np.abs(got[off:off + n] - ref).max() / np.abs(ref).max()
            assert err <= 1e-12, "tree %d (n=%d) cycle %d: %.3e" % (i, ps[i]["n"], k + 1, err)
