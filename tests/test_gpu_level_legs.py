"""A level's down and up legs as one cooperative launch each (grid barriers
between the phases, GMG_OPT_LEVEL_LEGS) against the per-phase launches: the
same block functions on the same inputs, so FP64 iterates, mixed solves and
BF16-state solves are equal bit for bit; the FP64 iterates also match the
oracle's."""
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


def _runs(p, coop, legs, prec, steps):
    t = gpu_problem(p)
    t.set_option("coarse_coop", coop)
    t.set_option("level_legs", legs)
    its = []
    if prec is None:
        for _ in range(steps):
            t.vcycle(1)
            its.append(t.solution().copy())
    else:
        st = t.solve(prec, 1e-30, steps, check=False)
        assert st["cycles"] == steps
        its.append(t.solution().copy())
    t.profile(True)
    t.profile_read()
    t.iterate(prec if prec is not None else 0, np.ones(t.units, dtype=np.int32))
    kinds = {k for k, _, _, _, _ in t.profile_read()}
    t.profile(False)
    t.close()
    return its, kinds


@pytest.mark.parametrize("name,coop", [("c2", 1), ("c2_64", 0)])
def test_level_legs_equal_per_phase_launches(name, coop):
    """On the 128^3 sphere only the FP32 level 4 qualifies (512 CTAs, four
    per SM; FP64 16^3 tiles allow two per SM, and under BF16 state level 4
    keeps its per-phase BF16 kernels).  With per-level coarse phases on the
    64^3 sphere, levels 2 and 3 (8 and 64 blocks) qualify in every
    precision (level 2 only under BF16 state)."""
    import paper_2205_09411_gb300 as G
    p = I.problem("c2") if name == "c2" else parity_cases()[name]
    for prec, steps in ((None, 3), (G.MIXED, 3), (G.MIXED_BF16, 3)):
        on, kinds_on = _runs(p, coop, 1, prec, steps)
        off, kinds_off = _runs(p, coop, 0, prec, steps)
        expect = name == "c2_64" or prec == G.MIXED
        assert ("level_leg_down" in kinds_on and "level_leg_up" in kinds_on) == expect, (prec, kinds_on)
        assert "level_leg_down" not in kinds_off
        for a, b in zip(on, off):
            assert np.array_equal(a, b)
    if name == "c2_64":  # FP64 legs (16^3 FP64 tiles, two CTAs per SM) against the oracle
        o = oracle_problem(p)
        on, _ = _runs(p, coop, 1, None, 4)
        for k in range(4):
            o.vcycle(1)
            ref = o.solution()
            assert np.abs(on[k] - ref).max() <= 1e-12 * np.abs(ref).max()
