"""CPU tests of the CUDA library's host logic: the shared library loads and
exports every function of include/gmg.h, and its block tree, leaf order and
boundary set-up (mask, line-search distances, cut-block counts, the
kernels' per-colour cut lists) equal the oracle's bit for bit.  No device
call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

import gmg_inputs as I
from _helpers import gpu_problem, oracle_problem, parity_cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    import paper_2205_09411_gb300 as G
    G.build()
    return G


def header_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_ ]+\*?\s*\**(gmg_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function(G):
    lib = ctypes.CDLL(G.LIB_PATH)
    names = header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_precision_constants_match_the_header(G):
    """The binding's precision codes are the header's GMG_FP64, GMG_MIXED and
    GMG_MIXED_BF16."""
    txt = open(os.path.join(ROOT, "include", "gmg.h")).read()
    defs = dict((k, int(v)) for k, v in re.findall(r"^#define (GMG_(?:FP64|MIXED|MIXED_BF16)) (\d+)", txt, flags=re.M))
    assert defs == {"GMG_FP64": G.FP64, "GMG_MIXED": G.MIXED, "GMG_MIXED_BF16": G.MIXED_BF16}


def test_library_fails_loudly_without_binary(G, tmp_path, monkeypatch):
    import paper_2205_09411_gb300 as mod
    monkeypatch.setattr(mod, "_lib", None)
    monkeypatch.setattr(mod, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        mod.load()


@pytest.mark.parametrize("name", sorted(parity_cases().keys()))
def test_tree_and_setup_equal_oracle(G, name):
    p = parity_cases()[name]
    o = oracle_problem(p, rhs=False)
    t = gpu_problem(p, bind=False)
    assert (t.lmin, t.lmax) == o.levels()
    assert t.n_leaf_cells == o.num_leaf_cells()
    for lev in range(t.lmin, t.lmax + 1):
        bg, hg = t.level_blocks(lev)
        bo, ho = o.level_blocks(lev)
        assert np.array_equal(bg, bo) and np.array_equal(hg, ho)
        assert t.level_n(lev) == o.level_n(lev) and t.level_h(lev) == o.level_h(lev)
        assert np.array_equal(t.mask(lev), o.get_mask(lev))
        dg, do = t.distances(lev), o.get_d(lev)
        assert np.array_equal(dg, do), np.abs(dg - do).max()
        assert t.num_cut_blocks(lev) == o.num_cut_blocks(lev)
        # the kernels' cut lists hold, per block and colour, exactly the
        # cells with some line-search distance below 1 (counted here from
        # the oracle's distances)
        n, D = t.level_n(lev), p["dim"]
        c = np.arange(n ** D)
        colour = (c % n + (c // n) % n + (c // (n * n) if D == 3 else 0)) % 2
        flagged = (do < 1.0).any(axis=2)
        expect = np.stack([(flagged & (colour == 0)).sum(1), (flagged & (colour == 1)).sum(1)], axis=1)
        assert np.array_equal(t.cut_counts(lev), expect)
    assert np.array_equal(t.leaf_centers(), o.leaf_centers())


def test_unresolved_search_equals_oracle(G):
    p = dict(dim=3, N=8, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1 / 8, max_level=2, refine=None,
             lsf=("capsule", (0.5, 0.5, 0.6, 0.5, 0.5, 1.0, 0.02)), walls=(1, 1, 1, 1, 0, 1),
             wall_values=(0,) * 6, wall_fn=None, phib=1.0, rhs=None, index=0)
    o = oracle_problem(p, w_min=0.008, rhs=False)
    t = gpu_problem(p, w_min=0.008, bind=False)
    n_virtual = 0
    for lev in range(t.lmin, t.lmax + 1):
        dg, do = t.distances(lev), o.get_d(lev)
        assert np.array_equal(dg, do)
        n_virtual += int((dg < 1).sum())
    assert n_virtual > 0


def test_invalid_arguments_are_rejected(G):
    with pytest.raises(G.GmgError):
        G.Tree(3, 7, max_level=2)       # odd block size
    with pytest.raises(G.GmgError):
        G.Tree(4, 8, max_level=2)       # dimension
    with pytest.raises(G.GmgError):
        G.Tree(3, 8, max_level=0)
    t = G.Tree(2, 8, max_level=2)
    with pytest.raises(G.GmgError):
        t.workspace_bytes()             # before store_stencils
    with pytest.raises(G.GmgError):
        t.cut_counts(1)                 # before store_stencils
    t.set_walls([0] * 4, values=[0.0] * 4)
    few = np.zeros((1, 5))              # one sample along x: not a grid
    with pytest.raises(G.GmgError):
        t.store_stencils(("grid", (few, [0.0, 0.0], 0.25)), 1.0)
    t.store_stencils(("sphere", (0.5, 0.5, 0.0, 0.25)), 1.0)
    with pytest.raises(G.GmgError):
        t.boundary_terms(t.lmax + 1)    # no such level


def test_forest_rejects_unlike_trees_and_new_boundary_values(G):
    """Trees of a forest share block size and sweeps; a forest's boundary
    value is set tree by tree before merging."""
    import gmg_inputs as I
    ps = I.forest_problems(2, index=3, sizes=(16, 32))
    a = gpu_problem(ps[0], bind=False)
    b = gpu_problem(dict(ps[1], N=16), bind=False)
    with pytest.raises(G.GmgError, match="block size"):
        G.Forest([a, b])
    b = gpu_problem(ps[1], bind=False)
    F = G.Forest([a, b])
    with pytest.raises(G.GmgError, match="single tree"):
        F.set_boundary_value(2.0)


def test_needle_tree_size():
    """The batched needle workload's tree: 7 levels of 8^3 blocks refined
    toward the needle axis hold 30,195,712 leaf cells after 2:1 balance
    (about 3e7, 512^3 effective near the needle)."""
    import gmg_inputs as I
    import paper_2205_09411_gb300 as G
    p = I.problem("c3", n_rhs=1)
    t = G.Tree(3, 8, (1, 1, 1), (0, 0, 0), 1 / 8, 7, refine=p["refine"], max_coarse_cells=64)
    assert t.n_leaf_cells == 30195712
    assert (t.lmin, t.lmax) == (0, 7)
    assert t.level_info(7)[2] == 1 / 512


def test_forest_structure():
    """A forest holds every block of its trees level by level, tree by tree,
    with tree-major leaves; its leaf centres are the trees' own."""
    import gmg_inputs as I
    import paper_2205_09411_gb300 as G
    from _helpers import gpu_problem
    ps = I.forest_problems(4, index=7, sizes=(16, 32, 64))
    trees = [gpu_problem(p, bind=False) for p in ps]
    F = G.Forest(trees)
    assert F.ntree == 4 and F.units == 4
    assert F.n_blocks == sum(t.n_blocks for t in trees)
    assert F.n_leaf_cells == sum(t.n_leaf_cells for t in trees)
    assert F.lmin == trees[0].lmin and F.lmax == max(t.lmax for t in trees)
    for l in range(F.lmin, F.lmax + 1):
        assert F.level_info(l)[0] == sum(t.level_info(l)[0] for t in trees if l <= t.lmax)
        # the forest's cut lists are its trees', level by level, tree by tree
        want = np.concatenate([t.cut_counts(l) for t in trees if l <= t.lmax])
        assert np.array_equal(F.cut_counts(l), want)
    xc = F.leaf_centers()
    off = 0
    for i, t in enumerate(trees):
        o, n = F.tree_leaves(i)
        assert (o, n) == (off, t.n_leaf_cells)
        assert np.array_equal(xc[o:o + n], t.leaf_centers())
        off += n
        assert F.num_cut_blocks(t.lmax) >= t.num_cut_blocks(t.lmax)


def test_box_noise_generators_agree():
    """The batched uneven-tree right-hand side: the leaf-order generator on
    torch (used at full size) equals the point-sampled numpy one, and the
    3^3 mean with zero padding is what it says (checked at a corner and an
    interior cell)."""
    import gmg_inputs as I
    import paper_2205_09411_gb300 as G
    n, N, seed = 16, 8, 1234
    t = G.Tree(3, N, (1, 1, 1), (0, 0, 0), 1 / 8, 2)
    bix, _ = t.level_blocks(t.lmax)
    a = I.box_noise_rhs(t.leaf_centers(), n, seed)
    b = I.box_noise_rhs_torch(bix, N, n, seed, device="cpu").numpy()
    assert np.allclose(a, b, rtol=0, atol=1e-15)
    w = np.random.Generator(np.random.PCG64(seed)).standard_normal((n, n, n))
    g = I.box_noise_grid(n, seed)
    assert abs(g[0, 0, 0] - w[:2, :2, :2].sum() / 27) < 1e-15
    assert abs(g[5, 6, 7] - w[4:7, 5:8, 6:9].sum() / 27) < 1e-15


def test_remesh_setup_equals_full_setup():
    """Re-meshing (Sec. 4.5): the needle tree refined one level deeper.
    Blocks that already existed reuse their set-up; the result equals a
    set-up from scratch of the new tree (distances and masks on every level,
    cut blocks), and only the new blocks were set up."""
    import gmg_inputs as I
    import paper_2205_09411_gb300 as G
    from _helpers import gpu_problem
    p4 = I.problem("c3", max_level=4, n_rhs=1)
    p5 = I.problem("c3", max_level=5, n_rhs=1)
    old = gpu_problem(p4, bind=False)
    new = old.remesh(p5["refine"], 5)
    ref = gpu_problem(p5, bind=False)
    assert (new.lmin, new.lmax, new.n_blocks) == (ref.lmin, ref.lmax, ref.n_blocks)
    for l in range(ref.lmin, ref.lmax + 1):
        assert np.array_equal(new.distances(l), ref.distances(l))
        assert np.array_equal(new.mask(l), ref.mask(l))
        assert new.num_cut_blocks(l) == ref.num_cut_blocks(l)
    computed, reused = new.setup_counts()
    assert reused > 0 and computed + reused == new.n_blocks
    assert computed <= new.n_blocks - old.n_blocks + 8  # new blocks only (a few may be removed ones)
    assert ref.setup_counts() == (ref.n_blocks, 0)


@pytest.mark.parametrize("name", ["c1", "adaptive3d", "needle4"])
def test_set_boundary_value_equals_full_setup(G, name):
    """A new boundary value on the stored boundary (no new line searches)
    gives the boundary terms, distances and cut lists of a full set-up with
    that value, bit for bit: a constant, and a function of x."""
    p = parity_cases()[name]
    for new in (2.5, lambda x: 1.0 + x[0] - 0.5 * x[1] + x[0] * x[1]):
        a = gpu_problem(dict(p, phib=0.3 if callable(p["phib"]) else p["phib"]), bind=False)
        a.set_boundary_value(new)
        b = gpu_problem(dict(p, phib=new), bind=False)
        for lev in range(a.lmin, a.lmax + 1):
            assert np.array_equal(a.boundary_terms(lev), b.boundary_terms(lev))
            assert np.array_equal(a.distances(lev), b.distances(lev))
            assert np.array_equal(a.cut_counts(lev), b.cut_counts(lev))


def test_set_boundary_value_needs_stored_stencils(G):
    p = parity_cases()["c1"]
    t = G.Tree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"])
    with pytest.raises(G.GmgError):
        t.set_boundary_value(1.0)


def _multilinear(values, origin, spacing, x):
    """Reference interpolation of gridded samples (numpy, independent of the
    library's): clamp to the sampled box, weights from the cell position."""
    dim = values.ndim
    i0, w = [], []
    for d in range(dim):
        n = values.shape[d]
        t = min(max((x[d] - origin[d]) / spacing, 0.0), n - 1.0)
        i = min(int(np.floor(t)), n - 2)
        i0.append(i)
        w.append(t - i)
    s = 0.0
    for corner in range(1 << dim):
        wt, idx = 1.0, []
        for d in range(dim):
            bit = (corner >> d) & 1
            wt *= w[d] if bit else 1.0 - w[d]
            idx.append(i0[d] + bit)
        s += wt * values[tuple(idx)]
    return s


def _grid_tree(G, p, lsf):
    t = G.Tree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
               max_coarse_cells=p.get("max_coarse_cells") or (64 if p["dim"] == 2 else 512),
               w_min=p.get("w_min", 0.0))
    t.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    t.store_stencils(lsf, p["phib"])
    return t


@pytest.mark.parametrize("dim", [2, 3])
def test_grid_level_set_reproduces_a_plane(G, dim):
    """Multilinear interpolation is exact on linear data: a plane sampled on
    a coarse grid gives the line-search distances of the plane itself (to
    the search tolerance)."""
    p = dict(parity_cases()["c1" if dim == 2 else "c2_32"])
    nrm = np.array([0.6, -0.48, 0.64][:dim])
    c = -0.2

    def plane(x):
        return float(np.dot(nrm, np.asarray(x)[:dim]) + c)
    m = 9
    axes = [np.linspace(0.0, 1.0, m)] * dim
    grid = np.meshgrid(*axes, indexing="ij")
    values = sum(nrm[d] * grid[d] for d in range(dim)) + c
    a = _grid_tree(G, p, ("grid", (values, [0.0] * dim, 1.0 / (m - 1))))
    b = _grid_tree(G, p, plane)
    for lev in range(a.lmin, a.lmax + 1):
        da, db = a.distances(lev), b.distances(lev)
        assert np.abs(da - db).max() <= 2e-8
        assert a.num_cut_blocks(lev) == b.num_cut_blocks(lev)


@pytest.mark.parametrize("name", ["c1", "adaptive3d", "needle4"])
def test_grid_level_set_setup_equals_oracle_grid(G, name):
    """The library's and the oracle's set-ups with the same sampled level set
    (each interpolating it in its own code) agree bit for bit: masks,
    distances, cut-block counts and the kernels' cut lists."""
    import oracle as O
    p = parity_cases()[name]
    dim = p["dim"]
    m = 41
    lo = np.asarray(p["lo"][:dim]) - 0.05
    span = 1.1 / (m - 1)
    axes = [lo[d] + np.arange(m) * span for d in range(dim)]
    grid = np.meshgrid(*axes, indexing="ij")
    c = np.array([0.47, 0.52, 0.55])[:dim]
    values = np.sqrt(sum((grid[d] - c[d]) ** 2 for d in range(dim))) - 0.23
    t = _grid_tree(G, p, ("grid", (values, lo, span)))
    o = O.OracleTree(dim, p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
                     max_coarse_cells=p.get("max_coarse_cells"))
    o.set_params(2, 2, 1e-8, 1.5, p.get("w_min", 0.0))
    o.set_lsf_grid(values, lo, span)
    o.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    o.store_stencils(p["phib"])
    assert (t.lmin, t.lmax) == o.levels()
    for lev in range(t.lmin, t.lmax + 1):
        assert np.array_equal(t.mask(lev), o.get_mask(lev))
        assert np.array_equal(t.distances(lev), o.get_d(lev))
        assert t.num_cut_blocks(lev) == o.num_cut_blocks(lev)


@pytest.mark.parametrize("name", ["c1", "adaptive3d"])
def test_grid_level_set_equals_oracle(G, name):
    """A sphere sampled on a grid: the library's set-up with the grid level
    set equals the oracle's with an independent numpy interpolation of the
    same samples (distances to the search tolerance, masks exactly)."""
    import oracle as O
    p = parity_cases()[name]
    dim = p["dim"]
    centre, radius = np.asarray(p["lsf"][1][:dim]), p["lsf"][1][3] if len(p["lsf"][1]) > 3 else 0.25
    m = 65
    lo = np.asarray(p["lo"][:dim])
    span = 1.0 / (m - 1) * 1.2
    axes = [lo[d] - 0.1 + np.arange(m) * span for d in range(dim)]
    grid = np.meshgrid(*axes, indexing="ij")
    values = np.sqrt(sum((grid[d] - centre[d]) ** 2 for d in range(dim))) - radius
    origin = [axes[d][0] for d in range(dim)]
    t = _grid_tree(G, p, ("grid", (values, origin, span)))
    o = O.OracleTree(dim, p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
                     max_coarse_cells=p.get("max_coarse_cells"))
    o.set_params(2, 2, 1e-8, 1.5, p.get("w_min", 0.0))
    o.set_lsf(O.LSF_CALLBACK, (), fn=lambda x: _multilinear(values, origin, span, x))
    o.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    o.store_stencils(p["phib"])
    for lev in range(t.lmin, t.lmax + 1):
        assert np.array_equal(t.mask(lev), o.get_mask(lev))
        assert np.abs(t.distances(lev) - o.get_d(lev)).max() <= 2e-8


def test_remesh_with_grid_level_set(G):
    """Re-meshing keeps the level set it was set up with, including a
    sampled one (the caller's samples stay alive): a refined tree re-meshed
    from a grid-level-set tree equals a fresh set-up of the refined tree,
    boundary terms and cut lists included."""
    from _helpers import refine_near
    p = dict(parity_cases()["c1"])
    m = 33
    ax = np.linspace(-0.05, 1.05, m)
    X, Y = np.meshgrid(ax, ax, indexing="ij")
    values = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2) - 0.25
    lsf = ("grid", (values, [ax[0], ax[0]], ax[1] - ax[0]))
    old = _grid_tree(G, p, lsf)
    rule = refine_near((0.75, 0.5), 0.12, p["N"], p["h1"], 2)
    new = old.remesh(rule, p["max_level"] + 1)
    fresh = dict(p, refine=rule, max_level=p["max_level"] + 1)
    ref = _grid_tree(G, fresh, lsf)
    assert (new.lmin, new.lmax, new.n_blocks) == (ref.lmin, ref.lmax, ref.n_blocks)
    for lev in range(ref.lmin, ref.lmax + 1):
        assert np.array_equal(new.distances(lev), ref.distances(lev))
        assert np.array_equal(new.boundary_terms(lev), ref.boundary_terms(lev))
        assert np.array_equal(new.cut_counts(lev), ref.cut_counts(lev))
    assert new.setup_counts()[1] > 0 and new.lmax == old.lmax + 1


def test_callback_errors_are_raised(G):
    """An exception inside a Python callback (refinement rule, level set,
    boundary value) is raised to the caller once the library call returns,
    instead of being swallowed by ctypes."""
    p = parity_cases()["c1"]

    def bad_rule(level, bix):
        raise ValueError("rule")
    with pytest.raises(RuntimeError, match="rule"):
        G.Tree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=bad_rule)
    t = G.Tree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"])
    t.set_walls(p["walls"], fn=p["wall_fn"])

    def bad_lsf(x):
        raise ValueError("lsf")
    with pytest.raises(RuntimeError, match="lsf"):
        t.store_stencils(bad_lsf, 1.0)
