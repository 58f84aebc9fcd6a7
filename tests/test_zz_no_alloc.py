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


@pytest.mark.parametrize("name", ["c2_64", "adaptive3d", "c1"])
def test_noalloc_residual_matches_workspace_residual(lib, name):
    t = gpu_problem(parity_cases()[name])
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
