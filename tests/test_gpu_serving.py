"""The serving loop on the GPU: three sessions (the 2D circle, a 32^3
sphere and the 4-level needle) under an HBM budget that holds only two at
once, requests arriving as a Poisson stream while others are mid-solve.
Every request's result equals, bit for bit and with the same cycle count,
the solve of its right-hand side alone on a fresh tree (so it is the same
alone and in the mix), for FP64 and mixed precision."""
import numpy as np
import pytest

import gmg_inputs as I
from _helpers import gpu_problem, parity_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09411_gb300 as G
    G.build()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_serving_results_equal_solo_solves(prec):
    import torch
    import paper_2205_09411_gb300 as G
    from paper_2205_09411_gb300.serving import Request, Server, Session, poisson_arrivals
    P = G.FP64 if prec == "fp64" else G.MIXED
    cases = {k: parity_cases()[k] for k in ("c1", "c2_32", "needle4")}
    sizes = {}
    sessions = []
    for name, p in cases.items():
        t = gpu_problem(p, bind=False, nrhs=3)
        sizes[name] = (t.n_leaf_cells, t.workspace_bytes())
        t.close()
        sessions.append(Session(name, make=lambda slots, p=p: gpu_problem(p, bind=False, nrhs=slots)))
    budget = sorted(b for _, b in sizes.values())[-1] + sorted(b for _, b in sizes.values())[-2]
    rng = I.rng_for(500)
    arrive = poisson_arrivals(400.0, 14, 501)
    names = list(cases)
    reqs = []
    for i in range(14):
        name = names[int(rng.integers(3))]
        reqs.append(Request(name, rng.standard_normal(sizes[name][0]) * (1 + i), float(arrive[i])))
    srv = Server(sessions, budget_bytes=budget, slots=3, precision=P, tol=1e-8,
                 new_stream=lambda: torch.cuda.Stream())
    done = srv.run(reqs)
    srv.close()
    assert len(done) == 14
    assert srv.peak_bytes <= budget
    assert any(e[0] == "evict" for e in srv.log) or len({r.session for r in done}) < 3
    for r in done:
        t = gpu_problem(cases[r.session], rhs=False)
        t.set_rhs(r.rhs)
        st = t.solve(P, 1e-8, 80)
        assert r.cycles == st["cycles"], r.id
        assert np.array_equal(r.result, t.solution()), "request %d differs from its solo solve" % r.id
        t.close()
