"""Host logic of the schedule autotuner, with a fake tree and a
deterministic cost model in place of timed GPU solves: the greedy search
keeps the best value of each knob in turn, applies the winner (sweeps split
between the fine and the cooperative levels), skips a diverging candidate,
and its results round-trip through the cache."""
import pytest

from paper_2205_09411_gb300 import MIXED, FP64
from paper_2205_09411_gb300 import autotune as AT


class FakeTree:
    """Levels 0..4 with 1, 8, 64, 512, 4096 blocks; records what is applied."""

    def __init__(self, nrhs=1):
        self.lmin, self.lmax, self.nrhs, self.ntree = 0, 4, nrhs, 1
        self.options, self.sweeps = {}, {}

    def level_info(self, l):
        return (8 ** l, 16, 1.0 / (16 * 2 ** l))

    def set_option(self, name, value):
        self.options[name] = value

    def set_level_sweeps(self, l, nd, nu):
        self.sweeps[l] = (nd, nu)


def cost_model(tree, set_rhs, precision, tol, reps):
    """A made-up, deterministic cost: fastest at cta 128, fine sweeps (1, 2),
    coarse (2, 2), 2 inner cycles, 2 slots per CTA, coop limit 160, unfused;
    coarse sweeps (4, 4) diverge."""
    o, sw = tree.options, tree.sweeps
    if sw[0] == (4, 4):
        return None, {"rc": -4}
    t = 1.0
    t += {64: 0.3, 128: 0.0, 256: 0.1}.get(o["cta_threads"], 0.2)
    t += {(1, 2): 0.0, (2, 2): 0.05}.get(sw[4], 0.2)
    t += 0.0 if sw[0] == (2, 2) else 0.1
    t += 0.0 if o["inner_cycles"] == 2 else 0.05
    t += 0.0 if o["slots_per_cta"] == 2 else 0.02
    t += 0.0 if o["coop_max_blocks"] == 160 else 0.07
    t += 0.0 if not o["fused_sweeps"] else 0.01
    return t, {"rc": 0, "cycles": 6}


def test_greedy_search_finds_the_model_optimum():
    tree = FakeTree(nrhs=4)
    s = AT.tune(tree, lambda: None, MIXED, 1e-8, reps=1, timer=cost_model)
    assert (s.cta_threads, s.fine_sweeps, s.coarse_sweeps, s.inner_cycles, s.slots_per_cta, s.coop_max_blocks,
            s.fused) == (128, (1, 2), (2, 2), 2, 2, 160, False)
    # the winner is applied: levels with at most 160 blocks (0..2) take the
    # coarse sweeps, the others the fine ones
    assert tree.options["cta_threads"] == 128 and tree.options["inner_cycles"] == 2
    assert [tree.sweeps[l] for l in range(5)] == [(2, 2)] * 3 + [(1, 2)] * 2
    assert any(x["seconds"] is None for x in s.trials)  # the diverging candidate was scored, not chosen
    assert len(s.trials) == 1 + 3 + 4 + 2 + 1 + 2 + 3 + 1  # each distinct schedule timed once


def test_axes_limit_and_fp64_has_no_inner_cycles():
    tree = FakeTree()
    s = AT.tune(tree, lambda: None, FP64, 1e-8, reps=1, axes=("fine_sweeps", "inner_cycles"), timer=cost_model)
    assert s.fine_sweeps == (1, 2) and s.inner_cycles == 1 and s.cta_threads == 0
    assert len(s.trials) == 1 + 4


def test_coop_levels_and_cache_round_trip(tmp_path):
    tree = FakeTree()
    assert [AT.coop_levels(tree, m) for m in (0, 1, 8, 64, 5000)] == [0, 0, 1, 2, 4]
    s = AT.tune(tree, lambda: None, MIXED, 1e-8, reps=1, timer=cost_model)
    key = AT.signature(tree, MIXED, 1e-8)
    path = str(tmp_path / "sched.json")
    AT.store_cached(path, key, s)
    back = AT.load_cached(path, key)
    assert back.key() == s.key()
    assert AT.load_cached(path, AT.signature(FakeTree(nrhs=2), MIXED, 1e-8)) is None
