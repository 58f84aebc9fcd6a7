"""bench.py's measurement arithmetic on the CPU: the algorithmic bytes of
each kernel kind (the roofline's numerator) from a fake tree, and the
roofline of the dominant kernel from a fake kernel-time table."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class FakeTree:
    """Levels 0..2 of 16^3 blocks (1, 8, 64 blocks); 10 listed cells per
    block of level 2 (6 of colour 0, 4 of colour 1), none elsewhere."""
    lmin, lmax, n_leaf_cells, dim = 0, 2, 64 * 16 ** 3, 3

    def level_info(self, l):
        return (8 ** l, 16, 1.0 / (16 * 2 ** l))

    def num_cut_blocks(self, l):
        return 64 if l == 2 else 0

    def cut_counts(self, l):
        return np.tile([6, 4], (8 ** l, 1)) if l == 2 else np.zeros((8 ** l, 2), dtype=int)


def test_algorithmic_bytes_per_kind():
    t = FakeTree()
    cells = 64 * 4096
    listed = 640
    S = 4
    # a half-sweep needs the other colour's phi and its own colour's b, and
    # writes its own colour's phi: half a value each per cell
    assert bench.algorithmic_bytes("smooth", "fp32", 2, t, 2) == cells * 1.5 * S + listed * (7 * S + 4) / 2
    assert bench.algorithmic_bytes("smooth", "fp32", 2, t, 2, nrhs=3) == 3 * cells * 1.5 * S + listed * (7 * S + 4) / 2
    assert bench.algorithmic_bytes("resid_restrict", "fp32", 2, t, 2) == cells * 2.25 * S + listed * (7 * S + 4)
    assert bench.algorithmic_bytes("prolong", "fp32", 2, t, 2) == cells * 2.25 * S
    assert bench.algorithmic_bytes("fas_rhs", "fp32", 1, t, 2) == 8 * 4096 * 4 * S
    assert bench.algorithmic_bytes("resid_norm", "fp64", 2, t, 2) == cells * 20 + listed * 60
    assert bench.algorithmic_bytes("accumulate", "fp64", 2, t, 2, nrhs=2) == t.n_leaf_cells * 2 * 20


def test_bf16_state_bytes():
    """BF16 finest-level state: phi 2 bytes, b and the coarser level's fields
    4 bytes, FP32 cut-list coefficients."""
    t = FakeTree()
    cells = 64 * 4096
    listed = 640
    entry = 7 * 4 + 4
    assert bench.algorithmic_bytes("smooth", "bf16", 2, t, 2) == cells * (2 + 0.5 * 4) + listed * entry / 2
    assert bench.algorithmic_bytes("resid_restrict", "bf16", 2, t, 2) == cells * (2 + 4 + 1) + listed * entry
    assert bench.algorithmic_bytes("prolong", "bf16", 2, t, 2) == cells * (2 * 2 + 1)
    # phi64 += e: 20 bytes a leaf cell, 18 on the finest level (all leaves there)
    assert bench.algorithmic_bytes("accumulate", "bf16", 2, t, 2) == t.n_leaf_cells * 20 - cells * 2


def test_level_leg_bytes_are_the_phases_bytes():
    """A leg in one launch moves what its per-phase launches move: N sweeps of
    two half-sweeps, plus the residual and restriction (down) or the
    prolongation (up)."""
    class Swept(FakeTree):
        def level_sweeps(self, l):
            return (2, 3)
    t = Swept()
    ab = bench.algorithmic_bytes
    half = ab("smooth", "fp32", 2, t, 2)
    assert ab("level_leg_down", "fp32", 2, t, 2) == 4 * half + ab("resid_restrict", "fp32", 2, t, 2)
    assert ab("level_leg_up", "fp32", 2, t, 2) == 6 * half + ab("prolong", "fp32", 2, t, 2)


def test_coarse_cycle_bytes_follow_the_level_visit_model():
    """The coarse kernels count 3S + 3S/8 (down leg) + 3S + 2S/8 (up leg)
    bytes a cell on each level they cover, plus the coarsest-level inverse
    once; with the cluster kernel at the bottom it takes the levels up to
    the roots' children level and the cooperative kernel, launched for the
    down and the up leg, the levels above, half of them per launch."""
    t = FakeTree()
    S = 4
    split = bench.coop_split(t)
    assert split == 2  # every level has at most 160 blocks
    c0, c1, c2 = 4096, 8 * 4096, 64 * 4096
    v = (3 + 3 / 8 + 3 + 2 / 8) * S
    inv = c0 ** 2 * 8
    assert bench.algorithmic_bytes("coarse_solve", "fp32", -1, t, 2) == pytest.approx((c0 + c1 + c2) * v + inv)
    assert bench.cluster_top(t) == 1  # level 1 holds the root's 8 children
    assert bench.algorithmic_bytes("coarse_cluster", "fp32", -1, t, 2, cluster=True) == pytest.approx((c0 + c1) * v + inv)
    assert bench.algorithmic_bytes("coarse_solve", "fp32", -1, t, 2, cluster=True) == pytest.approx(c2 * v / 2)
    assert bench.algorithmic_bytes("coarse_solve", "fp64", -1, t, 2, nrhs=2) == pytest.approx(2 * (c0 + c1 + c2) * 2 * v + inv)


def test_roofline_of_picks_the_dominant_kernel():
    t = FakeTree()
    prof = [("smooth", "fp32", 2, 8, 0.080), ("resid_norm", "fp64", 2, 1, 0.050), ("prolong", "fp32", 2, 1, 0.01)]
    roof, by_kind = bench.roofline_of(prof, t, 1, 6784.2, "measured")
    assert roof["kernel"] == "smooth_fp32_level2" and roof["bound"] == "hbm"
    per_launch_s = 0.080 / 8 * 1e-3
    alg = bench.algorithmic_bytes("smooth", "fp32", 2, t, 2)
    assert roof["achieved"] == pytest.approx(alg / per_launch_s / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6784.2)
    assert roof["share_of_kernel_time"] == pytest.approx(0.080 / 0.140)


def test_fp64_residual_roofline_is_against_the_fp64_pipe():
    """When the FP64 residual dominates, its roofline counts its algorithmic
    FP64 flops (9 a cell in 3D: 5 adds, 2 FMAs) against the FP64 peak of
    152 SMs x 2070 MHz x 4 flops a clock, and keeps the HBM figures beside."""
    t = FakeTree()
    prof = [("smooth", "fp32", 2, 8, 0.020), ("resid_norm", "fp64", 2, 2, 0.100)]
    roof, _ = bench.roofline_of(prof, t, 3, 6784.2, "measured")
    assert roof["kernel"] == "resid_norm_fp64_level2" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    per_launch_s = 0.100 / 2 * 1e-3
    flops = 3 * 64 * 4096 * 9
    assert roof["algorithmic_flops"] == flops
    assert roof["achieved"] == pytest.approx(flops / per_launch_s / 1e12)
    assert roof["peak"] == pytest.approx(152 * 2.07e9 * 4 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    alg = bench.algorithmic_bytes("resid_norm", "fp64", 2, t, 2, nrhs=3)
    assert roof["hbm"]["achieved"] == pytest.approx(alg / per_launch_s / 1e9)
