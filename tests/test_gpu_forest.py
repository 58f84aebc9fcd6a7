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
from _helpers import gpu_problem, oracle_problem

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
