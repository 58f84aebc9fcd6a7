"""GPU parity: the CUDA path against the FP64 oracle on the same seeded inputs.

FP64 path: after each of 12 V-cycles the leaf solution matches the oracle's
iterate to 1e-12 relative (max-norm, relative to max |phi|).  The two sides
share no code; their only differences are the rounding order of the same
formulas, which the multigrid contraction keeps near 1e-15.

Mixed path (FP32 V-cycles inside FP64 defect correction): reaches the same
1e-8 relative residual, checked independently by the oracle's own residual
of the returned solution, and its error against the oracle's converged FP64
solution is bounded per case.
"""
import numpy as np
import pytest

import gmg_inputs as I
from _helpers import gpu_problem, oracle_problem, parity_cases

pytestmark = pytest.mark.gpu

TOL_ITERATE = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09411_gb300 as G
    G.build()


CASES = sorted(parity_cases().keys())


@pytest.mark.parametrize("name", CASES)
def test_fp64_vcycle_iterates_match_oracle(name):
    p = parity_cases()[name]
    o = oracle_problem(p)
    t = gpu_problem(p)
    for k in range(12):
        o.vcycle(1)
        t.vcycle(1)
        ref = o.solution()
        got = t.solution()
        scale = max(np.abs(ref).max(), 1e-300)
        err = np.abs(got - ref).max() / scale
        assert err <= TOL_ITERATE, "cycle %d: relative max difference %.3e" % (k + 1, err)


@pytest.mark.parametrize("name", ["c1", "c2_64", "adaptive3d"])
def test_fp64_residual_norm_matches_oracle(name):
    p = parity_cases()[name]
    o = oracle_problem(p)
    t = gpu_problem(p)
    o.vcycle(3)
    t.vcycle(3)
    l2, linf, bn = o.residual()
    rel, mx = t.residual()
    assert abs(rel - l2 / bn) <= 1e-6 * (l2 / bn) + 1e-13
    assert abs(mx - linf) <= 1e-6 * linf + 1e-13 * bn


@pytest.mark.parametrize("name", ["c1", "c2_64", "ragged3d", "adaptive2d", "adaptive3d"])
def test_fp64_solve_matches_oracle(name):
    p = parity_cases()[name]
    o = oracle_problem(p)
    t = gpu_problem(p)
    ko, _ = o.solve(1e-10, 40)
    st = t.solve(0, 1e-10, 40)
    assert st["cycles"] == ko
    ref = o.solution()
    assert np.abs(t.solution() - ref).max() <= TOL_ITERATE * np.abs(ref).max()


@pytest.mark.parametrize("name", CASES)
def test_mixed_solve_reaches_tolerance(name):
    """The mixed path stops at the same 1e-8 relative residual as the FP64
    path; its error against the converged solution (an iterate at a 1e-8
    residual is not the converged solution) stays within 4x of the FP64
    path's error at the same tolerance."""
    p = parity_cases()[name]
    o = oracle_problem(p)
    t = gpu_problem(p)
    st = t.solve(1, 1e-8, 60)
    assert st["rel_l2"] <= 1e-8
    phi = t.solution()
    # independent check of the residual with the oracle's operator
    o.set_solution(phi)
    l2, _, bn = o.residual()
    assert l2 / bn <= 1.05e-8
    ko, _ = o.solve(1e-13, 60)
    assert ko >= 0
    ref = o.solution()
    scale = np.abs(ref).max()
    err_mixed = np.abs(phi - ref).max() / scale
    t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
    t.solve(0, 1e-8, 60)
    err_fp64 = np.abs(t.solution() - ref).max() / scale
    assert err_mixed <= 4 * err_fp64 + 1e-10, (err_mixed, err_fp64)


def test_full_size_sphere_configuration_matches_oracle():
    """128^3 sphere configuration at full size, in the launch configuration
    the benchmark times (graphs, cooperative and cluster coarse kernels):
    each of 12 FP64 V-cycles against the oracle, compared on every leaf
    cell."""
    p = I.problem("c2")
    o = oracle_problem(p)
    t = gpu_problem(p)
    for k in range(12):
        o.vcycle(1)
        t.vcycle(1)
        ref = o.solution()
        err = np.abs(t.solution() - ref).max() / np.abs(ref).max()
        assert err <= TOL_ITERATE, "cycle %d: %.3e" % (k + 1, err)


def test_full_size_needle_slot_matches_oracle():
    """The batched needle workload at full size (7 levels, 67,402 blocks,
    30.2 M leaf cells): one Gaussian-charge right-hand side in a 2-slot
    tree, 3 FP64 V-cycles against the oracle on every leaf cell."""
    p = I.problem("c3", n_rhs=2)
    t = gpu_problem(p, nrhs=2, rhs=False)
    xc = t.leaf_centers()
    g = np.stack([I.charge_density(xc, p["charges"][r]) for r in range(2)])
    t.set_rhs(g)
    o = oracle_problem(p, rhs=False)
    o.set_rhs(g[1])
    for k in range(3):
        o.vcycle(1)
        t.vcycle(1)
        ref = o.solution()
        err = np.abs(t.solution()[1] - ref).max() / np.abs(ref).max()
        assert err <= TOL_ITERATE, "cycle %d: %.3e" % (k + 1, err)


def test_zero_rhs_gives_zero_solution():
    p = dict(parity_cases()["no_boundary"])
    p["wall_values"] = (0,) * 6
    p["rhs"] = lambda xc: np.zeros(len(xc))
    t = gpu_problem(p)
    st = t.solve(0, 1e-8, 5)
    assert st["cycles"] == 0
    assert np.all(t.solution() == 0)


def test_device_arrays_round_trip():
    import torch
    p = parity_cases()["c1"]
    t = gpu_problem(p)
    g = torch.tensor(p["rhs"](t.leaf_centers()), dtype=torch.float64, device="cuda")
    t.set_rhs(g)
    t.vcycle(2)
    out = torch.zeros(t.n_leaf_cells, dtype=torch.float64, device="cuda")
    t.solution(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), t.solution())


@pytest.mark.parametrize("nrhs", [1, 3])
def test_pinned_host_arrays_round_trip(nrhs):
    """Pinned host arrays are read and written by the leaf scatter and gather
    kernels directly (no staging copy); pageable ones are staged.  Both give
    the device path's right-hand side and solution bit for bit, also for a
    range of slots."""
    import torch
    p = parity_cases()["needle4"]
    t = gpu_problem(p, nrhs=nrhs, rhs=False)
    n = t.n_leaf_cells
    rng = np.random.default_rng(7)
    g = rng.standard_normal((nrhs, n)) if nrhs > 1 else rng.standard_normal(n)
    outs = []
    for kind in ("device", "pinned", "pageable"):
        if kind == "device":
            gin = torch.tensor(g, device="cuda")
        elif kind == "pinned":
            gin = torch.tensor(g).pin_memory()
        else:
            gin = g.copy()
        t.set_rhs(gin)
        t.vcycle(2)
        if kind == "device":
            out = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        elif kind == "pinned":
            out = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
        else:
            out = np.zeros(g.shape)
        t.solution(out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy() if isinstance(out, torch.Tensor) else out)
        if nrhs > 1:  # one slot into a pinned buffer
            one = torch.zeros((1, n), dtype=torch.float64).pin_memory()
            t.solution_slots(nrhs - 1, 1, one)
            assert np.array_equal(one.numpy()[0], outs[-1][nrhs - 1])
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("name", ["c2_64", "adaptive3d", "ragged3d", "c1"])
@pytest.mark.parametrize("graphs,coop", [(0, 0), (1, 0), (0, 1)])
def test_execution_paths_give_the_oracle_iterates(name, graphs, coop):
    """The same V-cycle scheduled differently (captured graph or direct
    launches; coarse levels in one cooperative launch or one launch per
    phase) gives the oracle's iterates."""
    p = parity_cases()[name]
    o = oracle_problem(p)
    t = gpu_problem(p)
    t.set_option("graphs", graphs)
    t.set_option("coarse_coop", coop)
    for k in range(4):
        o.vcycle(1)
        t.vcycle(1)
    ref = o.solution()
    assert np.abs(t.solution() - ref).max() <= TOL_ITERATE * np.abs(ref).max()
    st = t.solve(1, 1e-8, 60)
    assert st["rel_l2"] <= 1e-8


@pytest.mark.parametrize("name", ["c2_64", "c2_32", "c1", "needle4", "adaptive3d", "no_boundary"])
def test_cluster_tail_gives_the_oracle_iterates(name):
    """The bottom of the V-cycle on a thread-block cluster (each CTA one
    part of the single-block levels and of the roots' children level, in
    shared memory, ghosts through distributed shared memory) gives the
    oracle's FP64 iterates after each of 6 V-cycles, FP64 and FMG, with
    clusters of 16 and of 8 CTAs in 3D (the same arithmetic: equal bit for
    bit); where the coarse solve of both paths sums a row the same way (at
    most 256 coarsest-level cells), the iterates and a mixed solve equal the
    single-CTA bottom's bit for bit."""
    p = parity_cases()[name]
    o = oracle_problem(p)
    out = []
    for mode, parts in ((2, 16), (2, 8), (0, 0)):
        t = gpu_problem(p)
        t.set_option("cluster_tail", mode)
        t.set_option("cluster_parts", parts)
        its = []
        for k in range(6):
            t.vcycle(1)
            its.append(t.solution().copy())
        t.fmg(1)
        its.append(t.solution().copy())
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
        st = t.solve(1, 1e-8, 60)
        assert st["rel_l2"] <= 1e-8
        its.append(t.solution().copy())
        out.append(its)
    for k in range(6):
        o.vcycle(1)
        ref = o.solution()
        assert np.abs(out[0][k] - ref).max() <= TOL_ITERATE * np.abs(ref).max(), k
    o.fmg(1)
    ref = o.solution()
    assert np.abs(out[0][6] - ref).max() <= TOL_ITERATE * np.abs(ref).max()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    q = gpu_problem(p, bind=False, rhs=False)
    if q.level_info(q.lmin)[1] ** p["dim"] <= 256:
        for a, b in zip(out[0], out[2]):
            assert np.array_equal(a, b)


def test_bounded_barrier_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: a grid barrier that can never
    complete ends its bounded wait with GMG_ERR_TIMEOUT; the device stays
    usable and the next solve is correct."""
    p = parity_cases()["c2_32"]
    t = gpu_problem(p)
    assert t.selftest_barrier_timeout(1 << 16) == -7
    o = oracle_problem(p)
    o.vcycle(3)
    t.vcycle(3)
    ref = o.solution()
    assert np.abs(t.solution() - ref).max() <= TOL_ITERATE * np.abs(ref).max()


@pytest.mark.parametrize("name", ["c2_64", "c2_32", "ragged3d", "c1", "adaptive3d"])
def test_fused_sweeps_equal_separate_half_sweeps(name):
    """The temporally blocked FP32 sweeps read exactly the inputs the
    separate half-sweeps read: three mixed defect-correction steps give the
    same solution either way."""
    p = parity_cases()[name]
    out = []
    for fused in (1, 0):
        t = gpu_problem(p)
        t.set_option("fused_sweeps", fused)
        st = t.solve(1, 1e-30, 3, check=False)
        assert st["cycles"] == 3
        out.append(t.solution())
    scale = np.abs(out[1]).max()
    assert np.abs(out[0] - out[1]).max() <= 1e-6 * scale


@pytest.mark.parametrize("name", ["c1", "needle4", "c2_64"])
def test_cta_sizes_give_identical_results(name):
    """The block kernels' CTA size (64, 128 or 256 threads) changes only
    which thread handles which cell: FP64 iterates and mixed solves are bit
    for bit the same."""
    p = parity_cases()[name]
    out = []
    for nt in (64, 128, 256):
        t = gpu_problem(p)
        t.set_option("cta_threads", nt)
        t.vcycle(3)
        a = t.solution().copy()
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
        st = t.solve(1, 1e-8, 60)
        out.append((a, t.solution().copy(), st["cycles"]))
    for a, b, c in out[1:]:
        assert np.array_equal(a, out[0][0]) and np.array_equal(b, out[0][1]) and c == out[0][2]


@pytest.mark.parametrize("name", ["c1", "needle4", "c2_64", "adaptive3d"])
def test_dependent_launch_gives_identical_results(name):
    """Programmatic dependent launch only lets a kernel be dispatched as its
    predecessor's CTAs exit; every kernel waits for its predecessor before
    reading a field.  FP64 iterates, FMG iterates and mixed solves are bit
    for bit the same with it on and off."""
    p = parity_cases()[name]
    out = []
    for pdl in (1, 0):
        t = gpu_problem(p)
        t.set_option("pdl", pdl)
        t.vcycle(3)
        a = t.solution().copy()
        t.fmg(1)
        f = t.solution().copy()
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
        st = t.solve(1, 1e-8, 60)
        out.append((a, f, t.solution().copy(), st["cycles"]))
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("name", ["c1", "c2_32", "adaptive2d", "adaptive3d", "needle4", "ragged3d"])
def test_fmg_iterates_match_oracle(name):
    """FMG cycles (Sec. 2.2) through the C ABI give the oracle's FMG iterates
    to 1e-12 after each of three cycles."""
    p = parity_cases()[name]
    o = oracle_problem(p)
    t = gpu_problem(p)
    for k in range(3):
        o.fmg(1)
        t.fmg(1)
        ref = o.solution()
        err = np.abs(t.solution() - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err <= TOL_ITERATE, "FMG cycle %d: relative max difference %.3e" % (k + 1, err)


def test_fmg_without_graphs_or_cooperative_launch():
    p = parity_cases()["adaptive3d"]
    o = oracle_problem(p)
    t = gpu_problem(p)
    t.set_option("graphs", 0)
    t.set_option("coarse_coop", 0)
    o.fmg(2)
    t.fmg(2)
    ref = o.solution()
    assert np.abs(t.solution() - ref).max() <= TOL_ITERATE * np.abs(ref).max()


@pytest.mark.parametrize("name", ["c1", "adaptive2d", "adaptive3d", "needle4", "ragged3d", "c2_32"])
def test_efield_matches_oracle(name):
    """E = -grad(phi) on cell faces (Sec. 4.4) from the same phi on both
    sides: the oracle's after four V-cycles, set on the GPU tree."""
    p = parity_cases()[name]
    o = oracle_problem(p)
    o.vcycle(4)
    phi = o.solution()
    t = gpu_problem(p)
    t.set_solution(phi)
    got = t.efield()
    ref = o.efield()
    scale = max(np.abs(ref).max(), 1e-300)
    assert np.abs(got - ref).max() <= 1e-12 * scale * 64


@pytest.mark.parametrize("shape", ["spheroid", "rhombus", "heart", "astroid"])
@pytest.mark.parametrize("dim", [2, 3])
def test_sharp_shapes_match_oracle(shape, dim):
    """Sec. 4.3's sharp boundaries with the unresolved-boundary search on:
    the set-up matches the oracle bit for bit (distances) and two FMG cycles
    match its iterates to 1e-12."""
    import gmg_inputs as Imod
    p = Imod.sharp_problem(shape, dim, 4 if dim == 2 else 3)
    o = oracle_problem(p)
    t = gpu_problem(p)
    for l in range(t.lmin, t.lmax + 1):
        assert np.array_equal(t.distances(l).reshape(-1), o.get_d(l).reshape(-1))
    o.fmg(2)
    t.fmg(2)
    ref = o.solution()
    assert np.abs(t.solution() - ref).max() <= TOL_ITERATE * np.abs(ref).max()


@pytest.mark.parametrize("name", ["c1", "adaptive3d"])
def test_solve_after_new_boundary_value(name):
    """A tree whose boundary value was changed after its set-up solves to
    the same solution, bit for bit, as a tree set up with that value."""
    p = parity_cases()[name]
    out = []
    for changed in (True, False):
        t = gpu_problem(dict(p, phib=0.7) if changed else dict(p, phib=1.9), bind=False)
        if changed:
            t.set_boundary_value(1.9)
        t.bind()
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
        st = t.solve(0, 1e-10, 40)
        out.append((t.solution().copy(), st["cycles"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


@pytest.mark.parametrize("name,prec", [("c1", 0), ("needle4", 1), ("adaptive3d", 0)])
def test_solve_history_equals_solve(name, prec):
    """The solve loop run step by step with its residual history gives
    gmg_solve's solution and cycle count bit for bit; the history starts at
    1 (phi = 0), ends at the returned residual and falls every step."""
    p = parity_cases()[name]
    t = gpu_problem(p)
    st = t.solve(prec, 1e-9, 60)
    ref = t.solution().copy()
    t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
    h = t.solve_history(prec, 1e-9, 60)
    assert np.array_equal(t.solution(), ref) and h["cycles"] == st["cycles"]
    hist = h["history"][:, 0]
    assert len(hist) == st["cycles"] + 1 and hist[0] == 1.0 and hist[-1] == h["rel_l2"] <= 1e-9
    assert np.all(np.diff(hist) < 0)


def _grid_case(name):
    """A parity case whose level set is a sphere sampled on a 41^D grid."""
    p = dict(parity_cases()[name])
    dim = p["dim"]
    m = 41
    lo = np.asarray(p["lo"][:dim]) - 0.05
    span = 1.1 / (m - 1)
    axes = [lo[d] + np.arange(m) * span for d in range(dim)]
    grid = np.meshgrid(*axes, indexing="ij")
    c = np.array([0.47, 0.52, 0.55])[:dim]
    values = np.sqrt(sum((grid[d] - c[d]) ** 2 for d in range(dim))) - 0.23
    return p, values, lo, span


@pytest.mark.parametrize("name", ["c1", "adaptive3d"])
def test_grid_level_set_iterates_match_oracle(name):
    """With a sampled level set (GMG_LSF_GRID / OT_LSF_GRID, set-ups equal bit
    for bit on the host) the FP64 V-cycle iterates through the C ABI equal
    the oracle's to 1e-12."""
    import oracle as O
    import paper_2205_09411_gb300 as G
    p, values, lo, span = _grid_case(name)
    dim = p["dim"]
    t = G.Tree(dim, p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
               max_coarse_cells=p.get("max_coarse_cells") or (64 if dim == 2 else 512), w_min=p.get("w_min", 0.0))
    t.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    t.store_stencils(("grid", (values, lo, span)), p["phib"])
    t.bind()
    g = np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64)
    t.set_rhs(g)
    o = O.OracleTree(dim, p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
                     max_coarse_cells=p.get("max_coarse_cells"))
    o.set_params(2, 2, 1e-8, 1.5, p.get("w_min", 0.0))
    o.set_lsf_grid(values, lo, span)
    o.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    o.store_stencils(p["phib"])
    o.set_rhs(g)
    for k in range(4):
        o.vcycle(1)
        t.vcycle(1)
        ref = o.solution()
        assert np.abs(t.solution() - ref).max() <= TOL_ITERATE * np.abs(ref).max()
