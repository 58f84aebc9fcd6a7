"""Right-hand-side slots: several right-hand sides of one tree in every launch.

Each slot must behave exactly like a tree of its own: its FP64 iterates match
the oracle run on that right-hand side alone (1e-12), and a batched solve,
or a serving-style sequence of gmg_iterate calls in which slots join, finish
and are reused at different times, gives every right-hand side bit for bit
the solution and cycle count of a solo solve.  The arithmetic of a slot
never mixes with another's, and a slot that has converged is frozen.
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


def slot_rhs(p, xc, R):
    """R right-hand sides: the problem's own, seeded noise of growing scale,
    and a zero one (the boundary terms alone)."""
    rng = I.rng_for(300 + p["index"])
    g = [np.asarray(p["rhs"](xc), dtype=np.float64)]
    for k in range(1, R - 1):
        g.append(rng.standard_normal(len(xc)) * (1.0 + 3.0 * k))
    g.append(np.zeros(len(xc)))
    return np.stack(g[:R])


@pytest.mark.parametrize("name", ["c1", "adaptive2d", "adaptive3d", "c2_32", "ragged3d"])
def test_slot_iterates_match_oracle(name):
    p = parity_cases()[name]
    R = 3
    t = gpu_problem(p, nrhs=R)
    g = slot_rhs(p, t.leaf_centers(), R)
    t.set_rhs(g)
    oracles = []
    for r in range(R):
        o = oracle_problem(p, rhs=False)
        o.set_rhs(g[r])
        oracles.append(o)
    for k in range(6):
        t.vcycle(1)
        got = t.solution()
        for r in range(R):
            oracles[r].vcycle(1)
            ref = oracles[r].solution()
            err = np.abs(got[r] - ref).max() / max(np.abs(ref).max(), 1e-300)
            assert err <= 1e-12, "slot %d cycle %d: %.3e" % (r, k + 1, err)
    rel, _ = t.residual()
    for r in range(R):
        l2, _, bn = oracles[r].residual()
        assert abs(rel[r] - l2 / bn) <= 1e-6 * (l2 / bn) + 1e-13


def solo(p, g, precision, tol, maxc=60):
    import paper_2205_09411_gb300 as G
    t = gpu_problem(p, rhs=False)
    t.set_rhs(g)
    st = t.solve(precision, tol, maxc)
    return t.solution().copy(), st


@pytest.mark.parametrize("name", ["c1", "adaptive3d", "c2_64"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_solve_equals_solo(name, prec):
    import paper_2205_09411_gb300 as G
    P = G.FP64 if prec == "fp64" else G.MIXED
    p = parity_cases()[name]
    R = 4
    t = gpu_problem(p, nrhs=R)
    g = slot_rhs(p, t.leaf_centers(), R)
    t.set_rhs(g)
    st = t.solve(P, 1e-8, 60)
    got = t.solution()
    for r in range(R):
        ref, st1 = solo(p, g[r], P, 1e-8)
        assert st["slots"][r]["cycles"] == st1["cycles"]
        assert st["slots"][r]["rel_l2"] == st1["rel_l2"]
        assert np.array_equal(got[r], ref), "slot %d differs from its solo solve" % r


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iterate_sequence_with_joins_and_reuse(prec):
    """A serving-style schedule: right-hand sides join free slots between
    steps, finished slots are read out and reused; each result equals the
    solo solve bit for bit."""
    import paper_2205_09411_gb300 as G
    P = G.FP64 if prec == "fp64" else G.MIXED
    p = parity_cases()["adaptive3d"]
    R, tol = 3, 1e-8
    t = gpu_problem(p, nrhs=R)
    xc = t.leaf_centers()
    rng = I.rng_for(400)
    jobs = [rng.standard_normal(len(xc)) * s for s in (1.0, 5.0, 0.2, 2.0, 1.0)]
    arrive = [0, 0, 2, 3, 3]  # step at which each job is submitted
    slot_job = [-1] * R
    cycles = {}
    results = {}
    queue = []
    step = 0
    active = np.zeros(R, dtype=np.int32)
    while len(results) < len(jobs):
        assert step < 400
        queue += [j for j in range(len(jobs)) if arrive[j] == step]
        new = np.zeros(R, dtype=np.int32)
        for r in range(R):
            if slot_job[r] < 0 and queue:
                j = queue.pop(0)
                slot_job[r] = j
                cycles[j] = 0
                t.set_rhs_slots(r, jobs[j])
                new[r] = 1
        if new.any():
            rel, _ = t.iterate(P, new, residual_only=True)
            for r in np.nonzero(new)[0]:
                active[r] = 1 if rel[r] > tol else 0
        if active.any():
            rel, _ = t.iterate(P, active)
            for r in np.nonzero(active)[0]:
                cycles[slot_job[r]] += 1
                if rel[r] <= tol:
                    active[r] = 0
        for r in range(R):
            if slot_job[r] >= 0 and not active[r]:
                results[slot_job[r]] = t.solution_slots(r, 1)[0].copy()
                slot_job[r] = -1
        step += 1
    for j, g in enumerate(jobs):
        ref, st1 = solo(p, g, P, tol)
        assert cycles[j] == st1["cycles"]
        assert np.array_equal(results[j], ref), "job %d differs from its solo solve" % j


def test_slot_bounds_rejected():
    import paper_2205_09411_gb300 as G
    p = parity_cases()["c1"]
    t = gpu_problem(p, nrhs=2)
    g = np.zeros(t.n_leaf_cells)
    with pytest.raises(G.GmgError):
        t.set_rhs_slots(2, g)
    with pytest.raises(G.GmgError):
        t.solution_slots(1, 2)
    t2 = gpu_problem(p, bind=False)
    t2.bind()
    with pytest.raises(G.GmgError):
        t2.set_num_rhs(4)  # after bind


def test_needle_gaussian_slots_match_oracle():
    """The batched needle workload at 4 levels: four Gaussian-charge
    right-hand sides in one tree; FP64 iterates per slot against the oracle,
    then a batched mixed solve whose every slot meets 1e-8 by the oracle's
    own residual."""
    import paper_2205_09411_gb300 as G
    p = parity_cases()["needle4"]
    R = 4
    t = gpu_problem(p, nrhs=R)
    xc = t.leaf_centers()
    g = np.stack([I.charge_density(xc, p["charges"][r]) for r in range(R)])
    t.set_rhs(g)
    oracles = []
    for r in range(R):
        o = oracle_problem(p, rhs=False)
        o.set_rhs(g[r])
        oracles.append(o)
    for k in range(4):
        t.vcycle(1)
        got = t.solution()
        for r in range(R):
            oracles[r].vcycle(1)
            ref = oracles[r].solution()
            err = np.abs(got[r] - ref).max() / np.abs(ref).max()
            assert err <= 1e-12, "slot %d cycle %d: %.3e" % (r, k + 1, err)
    t.set_rhs(g)
    st = t.solve(G.MIXED, 1e-8, 60)
    phi = t.solution()
    for r in range(R):
        assert st["slots"][r]["rel_l2"] <= 1e-8
        oracles[r].set_solution(phi[r])
        l2, _, bn = oracles[r].residual()
        assert l2 / bn <= 1.05e-8, (r, l2 / bn)


def test_many_waves_adaptive_slots_match_oracle():
    """A launch many CTA waves deep (the 5-level needle tree with 16 slots:
    about 16,000 CTAs per fine-level launch) still gives the oracle's
    iterates: no CTA reads coarse values that another CTA of the same launch
    rewrites (refinement-boundary ghosts during the restriction)."""
    import gmg_inputs as Imod
    p = Imod.problem("c3", max_level=5, n_rhs=2)
    R = 16
    t = gpu_problem(p, nrhs=R)
    xc = t.leaf_centers()
    g0 = I.charge_density(xc, p["charges"][0])
    g1 = I.charge_density(xc, p["charges"][1])
    g = np.stack([g0 if r % 2 == 0 else g1 for r in range(R)])
    t.set_rhs(g)
    refs = []
    for gr in (g0, g1):
        o = oracle_problem(p, rhs=False)
        o.set_rhs(gr)
        refs.append(o)
    for k in range(2):
        t.vcycle(1)
        got = t.solution()
        for i, o in enumerate(refs):
            o.vcycle(1)
            ref = o.solution()
            for r in range(i, R, 2):
                err = np.abs(got[r] - ref).max() / np.abs(ref).max()
                assert err <= 1e-12, "slot %d cycle %d: %.3e" % (r, k + 1, err)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_slot_groups_per_cta_give_identical_results(prec):
    """Half-sweeps that take 2 or 4 slots of a block per CTA (five slots, so
    one group is partial, and slots freeze at different cycles) give bit for
    bit the solutions and cycle counts of one slot per CTA."""
    import paper_2205_09411_gb300 as G
    P = G.FP64 if prec == "fp64" else G.MIXED
    p = parity_cases()["needle4"]
    R = 5
    out = []
    for spc in (1, 2, 4):
        t = gpu_problem(p, nrhs=R)
        t.set_option("slots_per_cta", spc)
        xc = t.leaf_centers()
        g = np.stack([I.charge_density(xc, p["charges"][r % 4]) * (1 + r) for r in range(R)])
        t.set_rhs(g)
        st = t.solve(P, 1e-8, 80)
        out.append((t.solution().copy(), [u["cycles"] for u in st["slots"]]))
    for sol, cyc in out[1:]:
        assert cyc == out[0][1]
        assert np.array_equal(sol, out[0][0])
