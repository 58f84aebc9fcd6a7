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


def oracle_problem(p, n_down=2, n_up=2, eps_tol=1e-8, mask_factor=1.5, w_min=None, rhs=True):
    import oracle as O
    if w_min is None:
        w_min = p.get("w_min", 0.0)
    kinds = {"none": O.LSF_NONE, "sphere": O.LSF_SPHERE, "capsule": O.LSF_CAPSULE,
             "ellipsoid": O.LSF_ELLIPSOID, "shape": O.LSF_SHAPE}
    t = O.OracleTree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
                     max_coarse_cells=p.get("max_coarse_cells"))
    t.set_params(n_down, n_up, eps_tol, mask_factor, w_min)
    kind, params = p["lsf"]
    t.set_lsf(kinds[kind], params)
    t.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    t.store_stencils(p["phib"])
    if rhs:
        t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
    return t


def gpu_problem(p, n_down=2, n_up=2, eps_tol=1e-8, mask_factor=1.5, w_min=None, bind=True, rhs=True, nrhs=1):
    """The same problem as oracle_problem, built through the CUDA library's C ABI
    (with nrhs right-hand-side slots; rhs=True fills only a single slot)."""
    import paper_2205_09411_gb300 as G
    if w_min is None:
        w_min = p.get("w_min", 0.0)
    t = G.Tree(p["dim"], p["N"], p["cb"], p["lo"], p["h1"], p["max_level"], refine=p["refine"],
               max_coarse_cells=p.get("max_coarse_cells") or (64 if p["dim"] == 2 else 512),
               n_down=n_down, n_up=n_up, eps_tol=eps_tol, mask_factor=mask_factor, w_min=w_min, nrhs=nrhs)
    t.set_walls(p["walls"], values=p.get("wall_values"), fn=p.get("wall_fn"))
    kind, params = p["lsf"]
    t.store_stencils(None if kind == "none" else (kind, params), p["phib"])
    if bind:
        t.bind()
        if rhs and nrhs == 1:
            t.set_rhs(np.asarray(p["rhs"](t.leaf_centers()), dtype=np.float64))
    return t


def refine_near(point, radius, N, h1, dim):
    """Refinement rule for tests: refine blocks within `radius` of `point`."""
    point = np.asarray(point, dtype=np.float64)

    def f(level, bix):
        bs = N * h1 / 2 ** (level - 1)
        lo = np.array(bix[:dim], dtype=np.float64) * bs
        q = np.clip(point, lo, lo + bs)
        return bool(np.linalg.norm(q - point) < radius)
    return f


def parity_cases():
    """Problems on which the CUDA path is compared with the oracle: the 2D
    configuration, small and full 3D sphere configurations, ragged root
    grids, mixed walls, adaptive trees and degenerate geometries."""
    import gmg_inputs as I
    rng_rhs = lambda seed: (lambda xc: I.rng_for(seed).standard_normal(len(xc)))
    cases = {
        "c1": I.problem("c1"),
        "c2_32": I.problem("c2", N=8, h1=1 / 8, max_level=3),
        "c2_64": I.problem("c2", N=16, h1=1 / 16, max_level=3),
        "ragged3d": dict(dim=3, N=8, cb=(3, 2, 1), lo=(0.0, 0.0, 0.0), h1=1 / 8, max_level=2, refine=None,
                         lsf=("sphere", (0.9, 0.55, 0.27, 0.33)), walls=(0, 1, 1, 0, 0, 1),
                         wall_values=(0.3, 0.0, 0.0, -0.6, 0.2, 0.0), wall_fn=None, phib=1.7,
                         rhs=rng_rhs(21), index=21),
        "adaptive2d": dict(dim=2, N=8, cb=(2, 2, 1), lo=(0.0, 0.0, 0.0), h1=1 / 16, max_level=4,
                           refine=refine_near([0.61, 0.4], 0.12, 8, 1 / 16, 2),
                           lsf=("sphere", (0.55, 0.45, 0.0, 0.2)), walls=(0, 1, 0, 0),
                           wall_values=(0.3, 0.0, -0.5, 0.8), wall_fn=None, phib=1.3, rhs=rng_rhs(22), index=22),
        "adaptive3d": dict(dim=3, N=8, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1 / 8, max_level=4,
                           refine=refine_near([0.4, 0.55, 0.5], 0.15, 8, 1 / 8, 3),
                           lsf=("sphere", (0.45, 0.5, 0.52, 0.18)), walls=(0, 0, 1, 0, 0, 0),
                           wall_values=(0.0, 1.0, 0.0, 0.5, 0.0, 0.0), wall_fn=None, phib=1.0,
                           rhs=rng_rhs(23), index=23),
        "no_boundary": dict(dim=3, N=8, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1 / 8, max_level=3, refine=None,
                            lsf=("none", ()), walls=(0, 0, 0, 0, 0, 0), wall_values=(0, 0, 0, 0, 0, 1.0),
                            wall_fn=None, phib=0.0, rhs=rng_rhs(24), index=24),
        "object_outside": dict(dim=2, N=8, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1 / 8, max_level=3, refine=None,
                               lsf=("sphere", (3.0, 3.0, 0.0, 0.5)), walls=(0, 0, 1, 1), wall_values=(1, -1, 0, 0),
                               wall_fn=None, phib=0.0, rhs=rng_rhs(25), index=25),
        "needle4": I.problem("c3", max_level=4, n_rhs=4),
        "single_level": dict(dim=2, N=8, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1 / 8, max_level=1, refine=None,
                             lsf=("sphere", (0.5, 0.5, 0.0, 0.3)), walls=(0, 0, 0, 0), wall_values=(0, 0, 0, 0),
                             wall_fn=None, phib=1.0, rhs=rng_rhs(26), index=26),
    }
    return cases
