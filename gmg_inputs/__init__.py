"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds only problem definitions: domains, block sizes, level-set
parameters, boundary values and right-hand sides.  It contains none of the
multigrid arithmetic, and it is the only code that both the CUDA library's
callers and the oracle use.  Every workload is synthetic (the paper uses
analytic test problems, not datasets):

* ``c1``  2D, [0,1]^2, 64^2 cells in 8^2 blocks (levels 8^2 .. 64^2); circle
  |x-(1/2,1/2)| - 1/4; manufactured u = sin(pi x) sin(pi y) + x^2 supplies
  g = Laplacian(u) everywhere, the circle's Dirichlet data and the walls'.
* ``c2``  3D, [0,1]^3, 128^3 cells in 16^3 blocks (coarse levels 8^3 and
  4^3 inside the root block); sphere |x-c| - 0.2; Laplace (g = 0) with
  phi = 1 on the sphere and 0 on the walls.
* ``sphere2d`` / ``sphere3d``  the convergence test of Sec. 4.1: a domain of
  unit size centred at the origin, f = |x| - R with R = 1/4, walls given by
  the analytic solutions log(|x|/R) (2D) and 1 - R/|x| (3D), phi_b = 0.

The base seed is 2205094110 + the configuration index (numpy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2205094110

WALL_DIRICHLET, WALL_NEUMANN = 0, 1


def rng_for(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


# ---------------------------------------------------------------------------
# manufactured solution of the 2D configuration
def c1_u(x):
    x = np.asarray(x, dtype=np.float64)
    return math.sin(math.pi * x[0]) * math.sin(math.pi * x[1]) + x[0] * x[0]


def c1_u_vec(xc):
    return np.sin(np.pi * xc[:, 0]) * np.sin(np.pi * xc[:, 1]) + xc[:, 0] ** 2


def c1_g_vec(xc):
    """Laplacian of c1_u, evaluated at the given points (n x 2)."""
    return -2.0 * np.pi ** 2 * np.sin(np.pi * xc[:, 0]) * np.sin(np.pi * xc[:, 1]) + 2.0


# analytic solutions of the sphere test (Sec. 4.1), phi_b = 0, a = 1
def sphere_solution(x, dim, R=0.25):
    x = np.asarray(x, dtype=np.float64)
    r = float(np.sqrt(np.sum(x[:dim] ** 2)))
    return math.log(r / R) if dim == 2 else 1.0 - R / r


def sphere_solution_vec(xc, dim, R=0.25):
    r = np.sqrt(np.sum(xc[:, :dim] ** 2, axis=1))
    return np.log(r / R) if dim == 2 else 1.0 - R / r


def problem(name: str, **over) -> dict:
    """Problem definition: geometry, boundary data and right-hand side.

    Keys: dim, N (cells per block side), cb (root blocks per side), lo, h1
    (cell size on level 1), max_level, refine (None = uniform), lsf (kind,
    params), walls (types), wall_values or wall_fn, phib (value or callable),
    rhs (callable centres -> g), n_vcycles, tol, and optionally
    max_coarse_cells (size of the coarsest level, default 64 in 2D and 512
    in 3D).
    """
    if name == "c1":
        p = dict(dim=2, N=8, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1.0 / 8, max_level=4, refine=None,
                 lsf=("sphere", (0.5, 0.5, 0.0, 0.25)), walls=(WALL_DIRICHLET,) * 4, wall_values=None,
                 wall_fn=c1_u, phib=c1_u, rhs=c1_g_vec, n_vcycles=12, tol=1e-8, index=0)
    elif name == "c2":
        p = dict(dim=3, N=16, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1.0 / 16, max_level=4, refine=None,
                 lsf=("sphere", (0.5, 0.5, 0.5, 0.2)), walls=(WALL_DIRICHLET,) * 6,
                 wall_values=(0.0,) * 6, wall_fn=None, phib=1.0,
                 rhs=lambda xc: np.zeros(len(xc)), n_vcycles=12, tol=1e-8, index=1, max_coarse_cells=64)
    elif name in ("sphere2d", "sphere3d"):
        dim = 2 if name == "sphere2d" else 3
        p = dict(dim=dim, N=8, cb=(1, 1, 1), lo=(-0.5, -0.5, -0.5 if dim == 3 else 0.0), h1=1.0 / 8,
                 max_level=3, refine=None, lsf=("sphere", (0.0, 0.0, 0.0, 0.25)),
                 walls=(WALL_DIRICHLET,) * (2 * dim), wall_values=None,
                 wall_fn=lambda x, _d=dim: sphere_solution(x, _d), phib=0.0,
                 rhs=lambda xc: np.zeros(len(xc)), n_vcycles=12, tol=1e-10, index=10 + dim)
    else:
        raise KeyError(name)
    p.update(over)
    return p


def scaled(p: dict, max_level: int) -> dict:
    """Same problem on a uniform tree refined to max_level."""
    q = dict(p)
    q["max_level"] = max_level
    return q


def random_rhs(n: int, index: int) -> np.ndarray:
    """Seeded N(0,1) right-hand side values for n cells."""
    return rng_for(index).standard_normal(n)
