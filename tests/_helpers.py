"""Shared test helpers: read the paper's printed values and build oracle problems."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_values():
    out = {}
    with open(os.path.join(GOLDEN, "paper_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


def oracle_problem(p, n_down=2, n_up=2, eps_tol=1e-8, mask_factor=1.5, w_min=0.0, rhs=True):
    import oracle as O
    kinds = {"none": O.LSF_NONE, "sphere": O.LSF_SPHERE, "capsule": O.LSF_CAPSULE,
             "ellipsoid": O.LSF_ELLIPSOID}
    t = O.OracleTree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"])
    t.set_params(n_down, n_up, eps_tol, mask_factor, w_min)
    kind, params = p["lsf"]
    t.set_lsf(kinds[kind], params)
    t.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    t.store_stencils(p["phib"])
    if rhs:
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
    return t
