"""GMG_MIXED_BF16: the mixed path with the finest level's FP32 correction
state stored as BF16 (2 bytes a cell in that level's sweeps, restriction,
prolongation and accumulation; FP32 arithmetic, FP32 b).

The oracle is FP64 and has no BF16 iterates to compare with, so these tests
check what the mixed path promises: the solve stops at the requested 1e-8
relative residual, the oracle's own residual of the returned solution
confirms it, and the error against the oracle's converged solution per unit
of final residual stays within 4x of the FP64 path's (an iterate at a 1e-8
residual is not the converged solution; its error scales with the residual
it stopped at).  The kernel timing record shows that the BF16 kernels ran,
on the finest level only.  A tree whose finest level runs inside the coarse
cooperative kernel keeps FP32 state and gives GMG_MIXED's result bit for
bit.
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


def _bf16_levels(t, precision):
    """Levels whose kernels ran on BF16 storage in one solve step."""
    t.profile(True)
    t.profile_read()
    t.iterate(precision, np.ones(t.units, dtype=np.int32))
    rec = t.profile_read()
    t.profile(False)
    return sorted({lv for kind, prec, lv, n, ms in rec if prec == "bf16"}), rec


def _check_against_oracle(p, t, st, phi):
    """The oracle's residual of phi and its error per unit residual against
    the FP64 path's."""
    import paper_2205_09411_gb300 as G
    o = oracle_problem(p)
    o.set_solution(phi)
    l2, _, bn = o.residual()
    assert l2 / bn <= 1.05e-8, l2 / bn
    ko, _ = o.solve(1e-13, 80)
    assert ko >= 0
    ref = o.solution()
    scale = np.abs(ref).max()
    err_bf = np.abs(phi - ref).max() / scale
    t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
    st64 = t.solve(G.FP64, 1e-8, 60)
    err_64 = np.abs(t.solution() - ref).max() / scale
    ratio = max(1.0, st["rel_l2"] / st64["rel_l2"])
    assert err_bf <= 4 * err_64 * ratio + 1e-10, (err_bf, err_64, st["rel_l2"], st64["rel_l2"])


@pytest.mark.parametrize("name", ["c2_64", "adaptive3d", "ragged3d", "adaptive2d", "c1", "needle4"])
def test_bf16_solve_reaches_tolerance(name):
    """Per-level coarse phases (the finest level is then never inside the
    cooperative kernel), so every case runs its finest level on BF16."""
    import paper_2205_09411_gb300 as G
    p = parity_cases()[name]
    t = gpu_problem(p)
    t.set_option("coarse_coop", 0)
    lv, _ = _bf16_levels(t, G.MIXED_BF16)
    assert lv == [t.lmax], lv
    t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
    st = t.solve(G.MIXED_BF16, 1e-8, 80)
    assert st["rel_l2"] <= 1e-8
    _check_against_oracle(p, t, st, t.solution().copy())


def test_bf16_state_differs_from_fp32_state():
    """One BF16 step is not the FP32 step (the storage is really BF16), but
    reduces the residual by a comparable factor."""
    import paper_2205_09411_gb300 as G
    p = parity_cases()["c2_64"]
    rel = {}
    sol = {}
    for prec in (G.MIXED, G.MIXED_BF16):
        t = gpu_problem(p)
        t.set_option("coarse_coop", 0)
        r0, _ = t.iterate(prec, np.ones(1, dtype=np.int32), residual_only=True)
        r1, _ = t.iterate(prec, np.ones(1, dtype=np.int32))
        rel[prec] = r1[0] / r0[0]
        sol[prec] = t.solution().copy()
    assert not np.array_equal(sol[G.MIXED], sol[G.MIXED_BF16])
    assert rel[G.MIXED_BF16] < 0.2 and rel[G.MIXED_BF16] < 3 * rel[G.MIXED] + 1e-3, rel


def test_bf16_falls_back_to_fp32_when_the_finest_level_is_coarse():
    """The 2D configuration (64^2 in 8^2 blocks, 85 blocks in all) runs its
    whole cycle in the cooperative kernel: no BF16 level, and the solve
    equals GMG_MIXED's bit for bit."""
    import paper_2205_09411_gb300 as G
    p = parity_cases()["c1"]
    out = []
    for prec in (G.MIXED, G.MIXED_BF16):
        t = gpu_problem(p)
        lv, _ = _bf16_levels(t, prec)
        assert lv == []
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
        st = t.solve(prec, 1e-8, 60)
        out.append((st["cycles"], t.solution().copy()))
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])


def test_bf16_slots_and_slot_groups():
    """Four right-hand sides of the 4-level needle tree, half-sweeps with 1,
    2 and 4 slots per CTA: every slot reaches 1e-8 (checked by the oracle's
    residual for slot 3), and the grouping does not change any bit."""
    import paper_2205_09411_gb300 as G
    p = parity_cases()["needle4"]
    outs = []
    for spc in (1, 2, 4):
        t = gpu_problem(p, nrhs=4, rhs=False)
        xc = t.leaf_centers()
        g = np.stack([I.charge_density(xc, p["charges"][r]) for r in range(4)])
        t.set_option("coarse_coop", 0)
        t.set_option("slots_per_cta", spc)
        t.set_rhs(g)
        st = t.solve(G.MIXED_BF16, 1e-8, 80)
        assert st["rel_l2"] <= 1e-8  # the worst slot's
        outs.append(t.solution().copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    o = oracle_problem(p, rhs=False)
    o.set_rhs(g[3])
    o.set_solution(outs[0][3])
    l2, _, bn = o.residual()
    assert l2 / bn <= 1.05e-8


def test_bf16_full_size_sphere_configuration():
    """The 128^3 sphere configuration in the benchmark's launch
    configuration (captured graphs, cooperative and cluster coarse levels;
    the finest level, 512 blocks of 16^3, on BF16): 1e-8 by the oracle's own
    residual, in at most two steps more than GMG_MIXED."""
    import paper_2205_09411_gb300 as G
    p = I.problem("c2")
    t = gpu_problem(p)
    lv, _ = _bf16_levels(t, G.MIXED_BF16)
    assert lv == [t.lmax]
    cyc = {}
    for prec in (G.MIXED, G.MIXED_BF16):
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
        st = t.solve(prec, 1e-8, 60)
        assert st["rel_l2"] <= 1e-8
        cyc[prec] = st["cycles"]
    phi = t.solution().copy()
    assert cyc[G.MIXED_BF16] <= cyc[G.MIXED] + 2, cyc
    o = oracle_problem(p)
    o.set_solution(phi)
    l2, _, bn = o.residual()
    assert l2 / bn <= 1.05e-8


@pytest.mark.parametrize("name,option,value", [("c2_64", "fmg_steps", 1), ("adaptive3d", "inner_cycles", 2),
                                               ("needle4", "inner_cycles", 2), ("c2_64", "fused_sweeps", 1)])
def test_bf16_with_schedule_options(name, option, value):
    """BF16 state under the other schedule options: FMG steps (the finest
    level's BF16 kernels inside each FMG cycle), two FP32 cycles per step on
    adaptive trees (the covered cells' phi restricted from the BF16 level
    between them) and fused sweeps on the FP32 levels below: 1e-8 by the
    oracle's own residual, with the BF16 kernels on the finest level only."""
    import paper_2205_09411_gb300 as G
    p = parity_cases()[name]
    t = gpu_problem(p)
    t.set_option("coarse_coop", 0)
    t.set_option(option, value)
    lv, _ = _bf16_levels(t, G.MIXED_BF16)
    assert lv == [t.lmax], lv
    t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
    st = t.solve(G.MIXED_BF16, 1e-8, 80)
    assert st["rel_l2"] <= 1e-8
    o = oracle_problem(p)
    o.set_solution(t.solution())
    l2, _, bn = o.residual()
    assert l2 / bn <= 1.05e-8
