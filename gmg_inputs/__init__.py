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
* ``c3``  3D adaptive needle electrode: [0,1]^3, 8^3-cell blocks, levels 1..7
  (finest cell 1/512); capsule level set around the segment x = y = 1/2,
  z in [0.6, 1] with radius 0.02 (hemispherical tip at z = 0.58), phi = 1 on
  the needle, phi = 0 on the bottom wall, zero flux on the other walls.
  Refinement rule of Sec. 4.1's refined test with r the distance to the
  needle axis: refine while dx > dx_min max(1, r / R_ref), r measured from
  the block; R_ref = NEEDLE_RREF gives about 3.0e7 leaf cells after 2:1
  balance.  Right-hand sides: sums of 1..20 Gaussian charge clouds
  (``gaussian_charges``).  The needle (diameter 0.04) is thinner than the
  cells of levels 0..3, so the unresolved-boundary search of Sec. 3.6.3 is
  on with w_min = 0.008 (the paper's 3D value); without it the V-cycle
  diverges on this geometry.
* ``forest_problems``  batched uneven trees: independent 3D problems on the
  unit cube with n^3 cells, n drawn from {32, 64, 128, 256}, 8^3-cell blocks;
  each a seeded ellipsoid level set (semi-axes U[0.1, 0.3], random
  rotation, centre U[0.35, 0.65]^3) with phi_b ~ U[0,1] on it and
  Dirichlet walls with values U[0,1] per wall; right-hand side white noise
  N(0,1) averaged over 3^3 cells (zero outside the domain).
* ``sharp_problem``  the sharp shapes of Sec. 4.3 (spheroid, rhombus, heart,
  astroid) on the unit square, or revolved about the z axis in 3D.
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


# needle electrode: axis segment a -> b (along z), radius
NEEDLE_A = (0.5, 0.5, 0.6)
NEEDLE_B = (0.5, 0.5, 1.0)
NEEDLE_RADIUS = 0.02
NEEDLE_RREF = 0.13  # refinement scale: 30,195,712 leaf cells at 7 levels after 2:1 balance


def needle_refine(r_ref, N=8, h1=1.0 / 8, max_level=7):
    """refine(level, bix): dx_level > dx_min * max(1, r / r_ref), with r the
    distance from the block to the needle's axis segment."""
    dx_min = h1 / 2 ** (max_level - 1)

    def f(level, bix):
        dx = h1 / 2 ** (level - 1)
        bs = N * dx
        lo = [bix[d] * bs for d in range(3)]
        ex = max(lo[0] - NEEDLE_A[0], NEEDLE_A[0] - (lo[0] + bs), 0.0)
        ey = max(lo[1] - NEEDLE_A[1], NEEDLE_A[1] - (lo[1] + bs), 0.0)
        ez = max(lo[2] - NEEDLE_B[2], NEEDLE_A[2] - (lo[2] + bs), 0.0)
        r = math.sqrt(ex * ex + ey * ey + ez * ez)
        return dx > dx_min * max(1.0, r / r_ref)
    return f


def gaussian_charges(n_rhs: int, index: int):
    """Seeded charge clouds of the batched needle workload: per right-hand
    side K ~ U{1..20} Gaussians with centres U[0,1]^3, widths U[0.01, 0.05]
    and amplitudes N(0, 1e3^2) rounded to FP32.  Returns a list of
    (centres K x 3, widths K, amplitudes K) per right-hand side."""
    rng = rng_for(index)
    out = []
    for _ in range(n_rhs):
        k = int(rng.integers(1, 21))
        c = rng.uniform(0.0, 1.0, size=(k, 3))
        w = rng.uniform(0.01, 0.05, size=k)
        a = rng.normal(0.0, 1e3, size=k).astype(np.float32).astype(np.float64)
        out.append((c, w, a))
    return out


def charge_density(xc, charges):
    """g(x) = sum_k a_k exp(-|x - c_k|^2 / (2 w_k^2)) at the points xc (n x 3,
    or n x 2 with the centres' first two coordinates)."""
    c, w, a = charges
    g = np.zeros(len(xc))
    for k in range(len(a)):
        d2 = np.sum((xc - c[k][:xc.shape[1]]) ** 2, axis=1)
        g += a[k] * np.exp(-d2 / (2.0 * w[k] ** 2))
    return g


def charge_density_torch(xc, charges):
    """The same sum on a torch tensor of points (any device)."""
    import torch
    c, w, a = charges
    g = torch.zeros(xc.shape[0], dtype=torch.float64, device=xc.device)
    for k in range(len(a)):
        ck = torch.tensor(c[k][:xc.shape[1]], dtype=torch.float64, device=xc.device)
        d2 = ((xc - ck) ** 2).sum(dim=1)
        g += float(a[k]) * torch.exp(-d2 / (2.0 * float(w[k]) ** 2))
    return g


def random_rotation(rng) -> np.ndarray:
    """A rotation matrix (det +1) from the QR factors of a Gaussian matrix."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def forest_problems(n_trees: int, index: int = 3, sizes=(32, 64, 128, 256), N: int = 8) -> list:
    """Seeded problems of the batched uneven-tree workload (one dict per
    tree, keys as problem()); 'n' is the tree's cells per side and
    'noise_seed' the seed of its right-hand side (box_noise_rhs)."""
    rng = rng_for(index)
    out = []
    for i in range(n_trees):
        n = int(rng.choice(sizes))
        semi = rng.uniform(0.1, 0.3, size=3)
        q = random_rotation(rng)
        c = rng.uniform(0.35, 0.65, size=3)
        phib = float(rng.uniform(0.0, 1.0))
        walls = tuple(float(v) for v in rng.uniform(0.0, 1.0, size=6))
        ml = int(round(math.log2(n / N))) + 1
        seed = 10_000 + 97 * index + i
        out.append(dict(dim=3, N=N, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1.0 / N, max_level=ml, refine=None,
                        lsf=("ellipsoid", tuple(c) + tuple(q.reshape(-1)) + tuple(semi)),
                        walls=(WALL_DIRICHLET,) * 6, wall_values=walls, wall_fn=None, phib=phib,
                        rhs=lambda xc, _n=n, _s=seed: box_noise_rhs(xc, _n, _s), n=n, noise_seed=seed,
                        n_vcycles=12, tol=1e-8, index=100 + i, max_coarse_cells=64))
    return out


def box_noise_rhs(xc, n: int, seed: int) -> np.ndarray:
    """White noise N(0,1) on the n^3 grid of the unit cube, averaged over the
    3^3 cells around each cell (cells outside the domain count as zero),
    sampled at the cell centres xc (any order)."""
    g = box_noise_grid(n, seed)
    ix = np.floor(np.asarray(xc) * n).astype(np.int64)
    return g[ix[:, 2], ix[:, 1], ix[:, 0]]


def box_noise_grid(n: int, seed: int) -> np.ndarray:
    """The filtered noise of box_noise_rhs on the whole n^3 grid, [z, y, x]."""
    w = np.random.Generator(np.random.PCG64(seed)).standard_normal((n, n, n))
    p = np.pad(w, 1)
    acc = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                acc += p[dz:dz + n, dy:dy + n, dx:dx + n]
    return acc / 27.0


def box_noise_rhs_torch(bix, N: int, n: int, seed: int, device="cuda"):
    """box_noise_rhs of a uniform tree in leaf order, built on a torch device
    from the leaf blocks' coordinates bix (k x 3, leaf order) and the block
    side N: the same noise (numpy PCG64), the 3^3 mean taken by avg_pool3d
    with zero padding."""
    import torch
    w = np.random.Generator(np.random.PCG64(seed)).standard_normal((n, n, n))
    g = torch.nn.functional.avg_pool3d(torch.tensor(w, device=device)[None, None], 3, stride=1, padding=1,
                                       count_include_pad=True)[0, 0]
    b = torch.tensor(np.asarray(bix, dtype=np.int64), device=device)
    c = torch.arange(N ** 3, device=device)
    x, y, z = c % N, (c // N) % N, c // (N * N)
    gx = (b[:, 0:1] * N + x[None, :]).reshape(-1)
    gy = (b[:, 1:2] * N + y[None, :]).reshape(-1)
    gz = (b[:, 2:3] * N + z[None, :]).reshape(-1)
    return g[gz, gy, gx]


SHAPES = {"spheroid": 0, "rhombus": 1, "heart": 2, "astroid": 3}


def sharp_problem(shape: str, dim: int = 2, max_level: int = 8) -> dict:
    """The sharp-boundary tests of Sec. 4.3: the unit square (cube) with
    8^2 (8^3) root cells, uniform refinement to max_level, phi = 1 on the
    shape and 0 on the walls, g = 0, w_min = 4e-3 in 2D and 8e-3 in 3D; in
    3D the shape is revolved about the z axis (reading SH)."""
    return dict(dim=dim, N=8, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1.0 / 8, max_level=max_level, refine=None,
                lsf=("shape", (float(SHAPES[shape]), 1.0 if dim == 3 else 0.0)), walls=(WALL_DIRICHLET,) * (2 * dim),
                wall_values=(0.0,) * 6, wall_fn=None, phib=1.0, rhs=lambda xc: np.zeros(len(xc)),
                n_vcycles=12, tol=1e-8, index=60 + SHAPES[shape], max_coarse_cells=64 if dim == 2 else 512,
                w_min=4e-3 if dim == 2 else 8e-3)


def problem(name: str, **over) -> dict:
    """Problem definition: geometry, boundary data and right-hand side.

    Keys: dim, N (cells per block side), cb (root blocks per side), lo, h1
    (cell size on level 1), max_level, refine (None = uniform), lsf (kind,
    params), walls (types), wall_values or wall_fn, phib (value or callable),
    rhs (callable centres -> g), n_vcycles, tol, and optionally
    max_coarse_cells (size of the coarsest level, default 64 in 2D and 512
    in 3D) and w_min (unresolved-boundary threshold of Sec. 3.6.3, default
    0 = off).
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
    elif name == "c3":
        ml = over.pop("max_level", 7)
        rref = over.pop("r_ref", NEEDLE_RREF)
        charges = gaussian_charges(over.pop("n_rhs", 32), 2)
        p = dict(dim=3, N=8, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=1.0 / 8, max_level=ml,
                 refine=needle_refine(rref, max_level=ml),
                 lsf=("capsule", NEEDLE_A + NEEDLE_B + (NEEDLE_RADIUS,)),
                 walls=(WALL_NEUMANN, WALL_NEUMANN, WALL_NEUMANN, WALL_NEUMANN, WALL_DIRICHLET, WALL_NEUMANN),
                 wall_values=(0.0,) * 6, wall_fn=None, phib=1.0, charges=charges,
                 rhs=lambda xc, _c=charges: charge_density(xc, _c[0]), n_vcycles=12, tol=1e-8, index=2,
                 max_coarse_cells=64, w_min=0.008)
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
