"""gmg_residual_noalloc: the residual norm for callers that cannot allocate
device memory (it keeps its per-block partial sums in a static device array
of the library instead of the tree's workspace).  Checked through the C ABI
against gmg_residual on two calls in a row, and its size limit.  This file
is collected last so that a failure here stops a run only after every other
test has run."""
import ctypes as C

import numpy as np
import pytest

from _helpers import gpu_problem, parity_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09411_gb300 as G
    G.build()
    L = G.load()
    L.gmg_residual_noalloc.restype = C.c_int
    L.gmg_residual_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    return L


def _noalloc(L, t):
    import torch
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = L.gmg_residual_noalloc(t.h, C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0, L.gmg_last_error().decode()
    stream.synchronize()
    return out.cpu().numpy()


def _cases():
    import gmg_inputs as I
    c = parity_cases()
    # a 2D tree of 32^2-cell blocks (the kernels' specialised side in 2D)
    c["c1_n32"] = dict(c["c1"], N=32, h1=1 / 32, max_level=2)
    return c


@pytest.mark.parametrize("name", ["c2_64", "adaptive3d", "c1", "c1_n32"])
def test_noalloc_residual_matches_workspace_residual(lib, name):
    t = gpu_problem(_cases()[name])
    t.vcycle(2)
    for _ in range(2):  # two calls in a row
        got = _noalloc(lib, t)
        rel, linf = t.residual()
        np.testing.assert_allclose(got, [rel, linf], rtol=1e-12, atol=0)
    t.vcycle(1)
    got = _noalloc(lib, t)
    rel, linf = t.residual()
    np.testing.assert_allclose(got, [rel, linf], rtol=1e-12, atol=0)


def test_noalloc_rejects_trees_beyond_the_scratch(lib):
    import paper_2205_09411_gb300 as G
    t = G.Tree(2, 4, (160, 160, 1), (0, 0, 0), 1.0 / 640, 2)  # 25600 + 102400 + sub-levels > 131072 blocks
    assert t.n_blocks > 131072
    import torch
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = lib.gmg_residual_noalloc(t.h, C.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert b"131072" in lib.gmg_last_error()


def test_noalloc_residual_is_slot_0_of_a_multi_slot_tree(lib):
    """With several right-hand-side slots the call evaluates slot 0, as
    gmg_residual's unit 0, and leaves the tree's unit mask alone: a solve
    of the other slots afterwards is unchanged."""
    import gmg_inputs as I
    p = parity_cases()["needle4"]
    R = 4
    t = gpu_problem(p, nrhs=R, rhs=False)
    xc = t.leaf_centers()
    g = np.stack([I.charge_density(xc, p["charges"][r]) for r in range(R)])
    t.set_rhs(g)
    t.vcycle(2)
    for _ in range(2):
        got = _noalloc(lib, t)
        rel, linf = t.residual()
        np.testing.assert_allclose(got, [rel[0], linf[0]], rtol=1e-12, atol=0)


def test_noalloc_residual_of_a_forest_is_one_norm_over_its_trees(lib):
    """On a forest, slot 0 of all trees together: sqrt(sum_i ||r_i||^2 /
    sum_i ||b_i||^2) and the largest |r|, rebuilt on the host from the
    oracle's residual of each tree's solution."""
    import gmg_inputs as I
    import oracle as O  # noqa: F401
    import paper_2205_09411_gb300 as G
    from _helpers import oracle_problem
    ps = I.forest_problems(3, index=7, sizes=(16, 32))
    trees = [gpu_problem(p, bind=False) for p in ps]
    F = G.Forest(trees)
    F.bind()
    g = np.zeros(F.n_leaf_cells)
    for i, (p, tr) in enumerate(zip(ps, trees)):
        off, n = F.tree_leaves(i)
        g[off:off + n] = p["rhs"](tr.leaf_centers())
    F.set_rhs(g)
    F.vcycle(2)
    phi = F.solution()
    r2 = b2 = linf = 0.0
    for i, p in enumerate(ps):
        o = oracle_problem(p)
        off, n = F.tree_leaves(i)
        o.set_solution(phi[off:off + n])
        l2, li, bn = o.residual()
        r2, b2, linf = r2 + l2 * l2, b2 + bn * bn, max(linf, li)
    for _ in range(2):
        got = _noalloc(lib, F)
        np.testing.assert_allclose(got, [np.sqrt(r2 / b2), linf], rtol=1e-6, atol=0)
