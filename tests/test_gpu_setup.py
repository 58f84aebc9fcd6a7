"""Boundary detection on the device (Sec. 3.2, Sec. 3.6.1, Sec. 3.6.3) for
the built-in level sets: the mask, the line-search distances, the
unresolved-root search and everything built from them (stencils, cut lists,
boundary terms) equal the host set-up's bit for bit, hence the oracle's
(the host set-up equals the oracle's bit for bit in the host tests).  Also
times both paths on the batched-trees workload."""
import time

import numpy as np
import pytest

import gmg_inputs as I
from _helpers import parity_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09411_gb300 as G
    G.build()


def set_up(p, device):
    import paper_2205_09411_gb300 as G
    t = G.Tree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
               max_coarse_cells=p.get("max_coarse_cells") or (64 if p["dim"] == 2 else 512),
               w_min=p.get("w_min", 0.0))
    t.set_option("device_setup", device)
    t.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    kind, params = p["lsf"]
    t.store_stencils(None if kind == "none" else (kind, params), p["phib"])
    return t


def cases():
    c = parity_cases()
    out = {k: c[k] for k in ("c1", "c2_64", "ragged3d", "adaptive2d", "adaptive3d", "needle4")}
    out["needle6"] = I.problem("c3", max_level=6, n_rhs=1)  # unresolved-root search on coarse levels
    for i, q in enumerate(I.forest_problems(3, index=9, sizes=(32, 64), N=16)):
        out["ellipsoid%d" % i] = q
    return out


@pytest.mark.parametrize("name", list(cases()))
def test_device_set_up_equals_host_set_up(name):
    p = cases()[name]
    h = set_up(p, 0)
    d = set_up(p, 1)
    assert not h.setup_on_device() and d.setup_on_device()
    for l in range(h.lmin, h.lmax + 1):
        assert np.array_equal(h.mask(l), d.mask(l)), l
        assert h.num_cut_blocks(l) == d.num_cut_blocks(l), l
        assert np.array_equal(h.distances(l), d.distances(l)), l
        assert np.array_equal(h.cut_counts(l), d.cut_counts(l)), l
        assert np.array_equal(h.boundary_terms(l), d.boundary_terms(l)), l
    # and the solve on top of it
    for t in (h, d):
        t.bind()
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
        t.vcycle(2)
    assert np.array_equal(h.solution(), d.solution())


def test_device_set_up_of_the_batched_trees_is_fast():
    """The 64 ellipsoid trees of the batched workload (16^3 blocks): the
    device path against the host path (all host threads)."""
    ps = I.forest_problems(64, index=3, sizes=(32, 64, 128, 256), N=16)
    times = {}
    for dev in (1, 0):
        t0 = time.perf_counter()
        trees = [set_up(q, dev) for q in ps]
        times[dev] = time.perf_counter() - t0
        assert all(t.setup_on_device() == bool(dev) for t in trees)
        del trees
    print("set-up of 64 trees: device %.2f s, host %.2f s" % (times[1], times[0]))
    assert times[1] < times[0]
