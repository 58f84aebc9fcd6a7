"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
solutions, exactness of the discretisation on polynomials, invariants, a
textbook matrix, a library solver, brute force on tiny inputs, and the
values the paper prints (tests/golden/paper_values.txt).  A plausible slip in
the oracle (a dropped term, a wrong sign or index, swapped d+/d-) fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest

import gmg_inputs as I
import oracle as O
from _helpers import oracle_problem, paper_values

EPS = 1e-8


# ---------------------------------------------------------------- helpers
def lex_perm(xc, h, lo):
    """Permutation taking canonical leaf order to x-fastest lexicographic order."""
    g = np.rint((xc - lo[:xc.shape[1]]) / h - 0.5).astype(np.int64)
    ext = g.max(0) + 1
    key = g[:, 0].copy()
    mul = ext[0]
    for d in range(1, xc.shape[1]):
        key += g[:, d] * mul
        mul *= ext[d]
    return np.argsort(key), g, ext


def wall_adjacent(g, ext):
    m = np.zeros(len(g), dtype=bool)
    for d in range(g.shape[1]):
        m |= (g[:, d] == 0) | (g[:, d] == ext[d] - 1)
    return m


def sphere_roots(a, k, s, h, c, R):
    """Smallest t in [0,1] with |a + t s h e_k - c| = R, or None (closed form)."""
    ak = a - c
    q = float(np.dot(ak, ak) - R * R)
    beta = s * ak[k]
    disc = beta * beta - q
    if disc < 0:
        return None
    sq = math.sqrt(disc)
    ts = sorted([(-beta - sq) / h, (-beta + sq) / h])
    for t in ts:
        if 0.0 <= t <= 1.0:
            return t, sq
    return None


def mk(dim, N, cb, h1, max_level, refine=None, lo=None, max_coarse_cells=None):
    lo = lo if lo is not None else (0.0, 0.0, 0.0)
    return O.OracleTree(dim, N, cb, lo, h1, max_level, refine=refine, max_coarse_cells=max_coarse_cells)


# ------------------------------------------------------------ coarse solver
def test_lu_solve_matches_library_solver():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((60, 60)) + 8 * np.eye(60)
    A[3, :] *= 1e-3  # forces pivoting
    b = rng.standard_normal(60)
    x = O.lu_solve(A, b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)


# -------------------------------------------------------------- line search
def test_line_search_bracketed_root_is_linear_root():
    d = O.line_search(lambda x: x[0] - 0.3, 2, [0, 0], [1, 0])
    assert abs(d - 0.3) <= 2 * EPS


def test_line_search_two_roots_keeps_the_nearer():
    f = lambda x: (x[0] - 0.2) * (x[0] - 0.7)
    assert abs(O.line_search(f, 2, [0, 0], [1, 0]) - 0.2) <= 2 * EPS
    assert abs(O.line_search(f, 2, [1, 0], [0, 0]) - 0.3) <= 2 * EPS


def test_line_search_narrow_pair_of_roots():
    f = lambda x: (x[0] - 0.5) ** 2 - 1e-4  # roots 0.49 and 0.51
    assert abs(O.line_search(f, 2, [0, 0], [1, 0]) - 0.49) <= 2 * EPS


def test_line_search_no_root_gives_one():
    assert O.line_search(lambda x: (x[0] - 0.5) ** 2 + 0.01, 2, [0, 0], [1, 0]) == 1.0
    assert O.line_search(lambda x: 1.0 + x[0], 3, [0, 0, 0], [0, 0, 1]) == 1.0


def test_line_search_root_at_start_is_clamped():
    d = O.line_search(lambda x: x[1], 2, [0.3, 0.0], [0.3, 1.0])
    assert EPS <= d <= 2 * EPS


@pytest.mark.parametrize("dim", [2, 3])
def test_distances_and_mask_match_sphere_intersections(dim):
    c = np.array([0.51, 0.47, 0.505])[:dim]
    R = 0.23
    t = mk(dim, 8, (1, 1, 1), 1 / 8, 3 if dim == 2 else 2)
    t.set_lsf(O.LSF_SPHERE, tuple(np.r_[c, np.zeros(3 - dim)]) + (R,))
    t.set_walls([0] * (2 * dim), values=[0.0] * (2 * dim))
    t.store_stencils(1.0)
    lmin, lmax = t.levels()
    checked = 0
    for lev in range(lmin, lmax + 1):
        d = t.get_d(lev).reshape(-1, 2 * dim)
        mask = t.get_mask(lev).ravel()
        xc = t.level_centers(lev)
        h = t.level_h(lev)
        for i, a in enumerate(xc):
            for k in range(dim):
                for s, side in ((-1, 0), (1, 1)):
                    nb = a[k] + s * h
                    if nb < 0 or nb > 1:
                        assert d[i, 2 * k + side] == 1.0
                        continue
                    root = sphere_roots(a, k, s, h, c, R)
                    if root is None:
                        assert d[i, 2 * k + side] == 1.0
                    else:
                        tt, chord = root
                        assert mask[i] == 1, "cell with a root within one cell is not masked"
                        if chord * h > 1e-6:
                            assert abs(d[i, 2 * k + side] - max(tt, EPS)) <= 2 * EPS
                            checked += 1
    assert checked > 50


@pytest.mark.parametrize("dim", [2, 3])
def test_grid_level_set_interpolates(dim):
    """The sampled level set (OT_LSF_GRID) is the multilinear interpolant of
    its samples: it returns the samples at the sample points, any linear
    function exactly (to rounding) everywhere in the box, and outside the
    box the value at the nearest point of the box."""
    rng = np.random.default_rng(5)
    m = [5, 6, 7][:dim]
    origin = np.array([-0.2, 0.1, 0.3])[:dim]
    h = 0.25
    axes = [origin[d] + h * np.arange(m[d]) for d in range(dim)]
    grid = np.meshgrid(*axes, indexing="ij")
    vals = rng.standard_normal(m)
    lsf = O.make_grid_lsf(vals, origin, h)
    for idx in [(0,) * dim, tuple(x - 1 for x in m), tuple(x // 2 for x in m)]:
        x = np.array([axes[d][idx[d]] for d in range(dim)])
        assert O.lsf_eval(lsf, dim, x) == vals[idx]
    a, c = rng.standard_normal(dim), 0.37
    lin = O.make_grid_lsf(sum(a[d] * grid[d] for d in range(dim)) + c, origin, h)
    hi = origin + h * (np.array(m) - 1)
    for x in rng.uniform(origin, hi, size=(50, dim)):
        assert abs(O.lsf_eval(lin, dim, x) - (a @ x + c)) <= 1e-14
    for x in rng.uniform(origin - 1.0, hi + 1.0, size=(50, dim)):
        assert O.lsf_eval(lin, dim, x) == O.lsf_eval(lin, dim, np.clip(x, origin, hi))


@pytest.mark.parametrize("dim", [2, 3])
def test_distances_from_both_sides_add_to_one(dim):
    """Invariant of the line search (Sec. 3.2): where the boundary crosses
    the segment between two neighbouring cell centres once (f changes sign),
    the relative distances searched from either end add up to 1 (to twice
    the search tolerance)."""
    c = np.array([0.52, 0.46, 0.49])[:dim]
    R = 0.27
    t = mk(dim, 8, (1, 1, 1), 1 / 8, 3 if dim == 2 else 2)
    t.set_lsf(O.LSF_SPHERE, tuple(np.r_[c, np.zeros(3 - dim)]) + (R,))
    t.set_walls([0] * (2 * dim), values=[0.0] * (2 * dim))
    t.store_stencils(1.0)
    lmin, lmax = t.levels()
    pairs = 0
    for lev in range(lmin, lmax + 1):
        d = t.get_d(lev).reshape(-1, 2 * dim)
        xc = t.level_centers(lev)
        h = t.level_h(lev)
        where = {tuple(np.round(a / h * 2).astype(int)): i for i, a in enumerate(xc)}
        f = np.linalg.norm(xc - c, axis=1) - R
        for i, a in enumerate(xc):
            for k in range(dim):
                b = a.copy()
                b[k] += h
                j = where.get(tuple(np.round(b / h * 2).astype(int)))
                if j is None or np.sign(f[i]) == np.sign(f[j]):
                    continue
                assert abs(d[i, 2 * k + 1] + d[j, 2 * k] - 1.0) <= 2 * EPS
                pairs += 1
    assert pairs > 50


# ------------------------------------------------------------ discretisation
@pytest.mark.parametrize("dim", [2, 3])
def test_cut_cell_operator_is_exact_for_quadratics(dim):
    """Eq. (lpl-1d-lsf) is the non-uniform three-point second derivative, so
    with phi_b = u(x0) it reproduces the Laplacian of any quadratic u."""
    cx = np.array([0.3, 1.0, -2.0, 0.5])
    if dim == 2:
        u = lambda x: 0.3 + x[0] - 2 * x[1] + 1.5 * x[0] ** 2 - x[1] ** 2 + 0.7 * x[0] * x[1]
        lap = 2 * 1.5 - 2 * 1.0
    else:
        u = lambda x: (0.3 + x[0] - 2 * x[1] + 0.5 * x[2] + 1.5 * x[0] ** 2 - x[1] ** 2 + 0.8 * x[2] ** 2
                       + 0.7 * x[0] * x[1] - 0.4 * x[1] * x[2] + 0.2 * x[0] * x[2])
        lap = 2 * 1.5 - 2 * 1.0 + 2 * 0.8
    del cx
    t = mk(dim, 8, (1, 1, 1), 1 / 8, 3 if dim == 2 else 2)
    t.set_lsf(O.LSF_SPHERE, (0.51, 0.48, 0.5, 0.27))
    t.set_walls([0] * (2 * dim), fn=u)
    t.store_stencils(u)
    xc = t.leaf_centers()
    uu = np.array([u(np.r_[x, np.zeros(3 - dim)]) for x in xc])
    Au = t.apply_composite(uu, with_bterm=True)
    lmin, lmax = t.levels()
    h = t.level_h(lmax)
    d = t.get_d(lmax).reshape(-1, 2 * dim)
    _, g, ext = lex_perm(xc, h, np.zeros(3))
    inner = ~wall_adjacent(g, ext)
    ncut = int((d.min(1) < 1).sum())
    assert ncut > 20
    # rounding bound: eps * |u| * sum of |stencil coefficients|, c <= 2/(d h^2)
    bound = 200 * np.finfo(float).eps * np.abs(uu).max() * np.sum(4.0 / (d * h * h), axis=1)
    err = np.abs(Au - lap)
    assert np.all(err[inner] <= bound[inner] + 1e-9), err[inner].max()


def _textbook_1d(n, lo_type, hi_type):
    T = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    T[0, 0] += -1.0 if lo_type == 0 else 1.0
    T[-1, -1] += -1.0 if hi_type == 0 else 1.0
    return T


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_operator_equals_textbook_laplacian(dim):
    """Without an irregular boundary the operator is the 5/7-point Laplacian
    (Eq. (lpl-1d) per dimension) with ghost -phi_i (Dirichlet) or +phi_i
    (Neumann), assembled here from Kronecker products."""
    types = [0, 1, 1, 0, 0, 1][:2 * dim]
    cb = (2, 1, 1)
    t = mk(dim, 4, cb, 1 / 8, 2)
    t.set_lsf(O.LSF_NONE)
    vals = [0.7, 0.0, 0.0, -1.2, 0.4, 0.0][:2 * dim]
    t.set_walls(types, values=vals)
    t.store_stencils(0.0)
    A, b = t.composite_matrix()
    xc = t.leaf_centers()
    h = t.level_h(t.levels()[1])
    perm, g, ext = lex_perm(xc, h, np.zeros(3))
    Ap = A[np.ix_(perm, perm)]
    Ts = [_textbook_1d(ext[k], types[2 * k], types[2 * k + 1]) for k in range(dim)]
    L = np.zeros_like(Ap)
    for k in range(dim):
        M = np.ones((1, 1))
        for j in range(dim - 1, -1, -1):
            M = np.kron(M, Ts[k] if j == k else np.eye(ext[j]))
        L += M
    L /= h * h
    np.testing.assert_allclose(Ap, L, rtol=1e-13, atol=1e-9)
    # Dirichlet wall values enter the rhs as -2 phi_w / h^2 (ghost 2 phi_w - phi_i)
    t.set_rhs(np.zeros(len(xc)))
    _, _, _, r = t.residual(want_field=True)
    expect = np.zeros(len(xc))
    for k in range(dim):
        for side in (0, 1):
            if types[2 * k + side] == 0:
                on = g[:, k] == (0 if side == 0 else ext[k] - 1)
                expect[on] -= 2 * vals[2 * k + side] / (h * h)
    np.testing.assert_allclose(r, expect, rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_operator_is_regular_where_no_distance_is_below_one(dim):
    """Eq. (lpl-1d-lsf) with d_- = d_+ = 1 is Eq. (lpl-1d): on a uniform
    tree cut by a sphere, every cell whose 2D distances are all 1 and which
    has no wall neighbour has the textbook row (-2D on the diagonal, 1 to
    each neighbour, over h^2), whether or not its block is cut."""
    c = np.array([0.5, 0.5, 0.5])[:dim]
    t = mk(dim, 4, (1, 1, 1), 1 / 4, 3 if dim == 2 else 2)
    t.set_lsf(O.LSF_SPHERE, tuple(np.r_[c, np.zeros(3 - dim)]) + (0.3,))
    t.set_walls([0] * (2 * dim), values=[0.0] * (2 * dim))
    t.store_stencils(1.0)
    lmin, lmax = t.levels()
    A, _ = t.composite_matrix()
    xc = t.leaf_centers()
    h = t.level_h(lmax)
    d = t.get_d(lmax).reshape(-1, 2 * dim)
    xl = t.level_centers(lmax)
    dist_of = {tuple(np.round(a / h * 2).astype(int)): d[i] for i, a in enumerate(xl)}
    where = {tuple(np.round(a / h * 2).astype(int)): i for i, a in enumerate(xc)}
    regular = cut_rows = 0
    for i, a in enumerate(xc):
        key = tuple(np.round(a / h * 2).astype(int))
        if np.any(dist_of[key] < 1.0) or np.any(a < h) or np.any(a > 1 - h):
            continue
        row = np.zeros(A.shape[1])
        row[i] = -2 * dim / (h * h)
        for k in range(dim):
            for s in (-1, 1):
                b = a.copy()
                b[k] += s * h
                row[where[tuple(np.round(b / h * 2).astype(int))]] = 1 / (h * h)
        assert np.array_equal(A[i], row)
        regular += 1
        cut_rows += 1 if np.linalg.norm(a - c) < 0.3 + 2 * h and np.linalg.norm(a - c) > 0.3 - 2 * h else 0
    assert regular > 20 and cut_rows > 0


def _refine_near(point, radius, N, h1, dim):
    point = np.asarray(point)

    def f(level, bix):
        bs = N * h1 / 2 ** (level - 1)
        lo = np.array(bix[:dim]) * bs
        q = np.clip(point, lo, lo + bs)
        return np.linalg.norm(q - point) < radius
    return f


@pytest.mark.parametrize("dim", [2, 3])
def test_composite_operator_annihilates_linear_functions(dim):
    """Reading G is exact for linear phi, restriction keeps linear phi: the
    composite operator gives 0 on linear phi away from the walls, also at
    refinement boundaries."""
    N, h1 = 4, 1 / 8
    t = mk(dim, N, (2, 2, 2), h1, 4, refine=_refine_near([0.3, 0.62, 0.45][:dim], 0.1, N, h1, dim))
    t.set_lsf(O.LSF_NONE)
    t.set_walls([1] * (2 * dim), values=[0.0] * (2 * dim))
    t.store_stencils(0.0)
    lev = t.leaf_levels()
    assert len(np.unique(lev)) >= 3
    xc = t.leaf_centers()
    coef = np.array([1.3, -0.7, 0.9])[:dim]
    u = 0.4 + xc @ coef
    Au = t.apply_composite(u, with_bterm=False)
    hs = np.array([t.level_h(int(l)) for l in lev])
    # wall ghosts (and coarse wall ghosts used by the tangential slopes of
    # reading G, two coarse cells = four fine cells deep) are not linear-exact
    near_wall = np.zeros(len(xc), dtype=bool)
    for d in range(dim):
        near_wall |= (xc[:, d] < 4 * hs) | (xc[:, d] > 1 - 4 * hs)
    assert (~near_wall).sum() > 100
    assert np.abs(Au[~near_wall]).max() <= 1e-9 / hs.min() ** 2


@pytest.mark.parametrize("dim,sub", [(2, False), (3, False), (3, True)])
def test_restriction_and_prolongation_exact_on_linear(dim, sub):
    if sub:
        t = mk(dim, 8, (1, 1, 1), 1 / 8, 1, max_coarse_cells=64)
        fine_l = 1
    else:
        t = mk(dim, 4, (2, 2, 2), 1 / 8, 3)
        fine_l = 3
    t.set_lsf(O.LSF_NONE)
    t.set_walls([0] * (2 * dim), values=[0.0] * (2 * dim))
    t.store_stencils(0.0)
    assert t.levels()[0] <= fine_l - 1
    coef = np.array([0.6, -1.1, 0.35])[:dim]
    lin = lambda xc: 0.2 + xc @ coef
    xf, xcrs = t.level_centers(fine_l), t.level_centers(fine_l - 1)
    np.testing.assert_allclose(t.restrict_test(fine_l, lin(xf)), lin(xcrs), rtol=0, atol=1e-14)
    fine = t.prolong_test(fine_l, lin(xcrs))
    hf = t.level_h(fine_l)
    ext = np.rint(1.0 / hf * np.ones(dim) * np.array([2, 2, 2][:dim] if not sub else 1)).astype(int)
    _, g, ext = lex_perm(xf, hf, np.zeros(3))
    inner = ~wall_adjacent(g, ext)
    np.testing.assert_allclose(fine[inner], lin(xf)[inner], rtol=0, atol=1e-13)
    # at a Dirichlet wall the reflected coarse ghost makes the prolongation
    # of a function vanishing on the wall exact: check one wall-adjacent value
    assert np.any(~inner)


def test_gsrb_half_sweep_solves_its_colour():
    """A red half-sweep solves every red equation given the black values
    (Sec. 2.2): the red residual vanishes away from walls, black is kept."""
    p = I.problem("c1")
    t = oracle_problem(p)
    lmin, lmax = t.levels()
    rng = np.random.default_rng(3)
    n = len(t.level_centers(lmax))
    phi0 = rng.standard_normal(n)
    t.set_level(lmax, phi0, 0)
    t.set_level(lmax, rng.standard_normal(n), 1)
    t.halfsweep(lmax, 0)
    phi1 = t.get_level(lmax, 0)
    r = t.level_residual(lmax)
    xc = t.level_centers(lmax)
    h = t.level_h(lmax)
    _, g, ext = lex_perm(xc, h, np.zeros(3))
    red = (g.sum(1) % 2) == 0
    inner = ~wall_adjacent(g, ext)
    assert np.abs(r[red & inner]).max() <= 1e-7  # |A| ~ 1e4..1e10, values O(1)
    assert np.array_equal(phi1[~red], phi0[~red])
    assert not np.allclose(phi1[red], phi0[red])


# ----------------------------------------------------------- multigrid
def _dense_case(kind):
    rng = np.random.default_rng(11)
    if kind == "uniform2d":
        t = mk(2, 4, (1, 1), 1 / 4, 3)
        t.set_lsf(O.LSF_SPHERE, (0.52, 0.47, 0.0, 0.3))
        t.set_walls([0, 0, 1, 0], values=[0.2, -0.4, 0.0, 1.0])
    elif kind == "adaptive2d":
        t = mk(2, 4, (2, 2), 1 / 8, 3, refine=_refine_near([0.61, 0.4], 0.1, 4, 1 / 8, 2))
        t.set_lsf(O.LSF_SPHERE, (0.55, 0.45, 0.0, 0.2))
        t.set_walls([0, 1, 0, 0], values=[0.3, 0.0, -0.5, 0.8])
    else:
        t = mk(3, 4, (1, 1, 1), 1 / 4, 2)
        t.set_lsf(O.LSF_SPHERE, (0.5, 0.52, 0.48, 0.3))
        t.set_walls([0, 0, 0, 1, 0, 0], values=[0.1, 0.2, 0.3, 0.0, 0.5, 0.6])
    t.store_stencils(1.3)
    t.set_rhs(rng.standard_normal(t.num_leaf_cells()))
    return t


@pytest.mark.parametrize("kind", ["uniform2d", "adaptive2d", "uniform3d"])
def test_multigrid_converges_to_dense_solution(kind):
    """Brute force: the FAS V-cycle's fixed point is the solution of the
    assembled composite linear system (numpy's dense solver)."""
    t = _dense_case(kind)
    if kind == "adaptive2d":
        assert len(np.unique(t.leaf_levels())) >= 2
    A, b = t.composite_matrix()
    assert A.shape[0] <= 1024
    x = np.linalg.solve(A, b)
    k, hist = t.solve(1e-14, 60)
    assert k > 0, hist
    phi = t.solution()
    assert np.abs(phi - x).max() <= 1e-10 * np.abs(x).max()
    # the exact solution is a fixed point of one V-cycle
    t.set_solution(x)
    t.vcycle(1)
    assert np.abs(t.solution() - x).max() <= 1e-11 * np.abs(x).max()


def _solve_error(p, ml, tol=1e-11):
    q = I.scaled(p, ml)
    t = oracle_problem(q)
    k, _ = t.solve(tol, 40)
    assert k > 0
    xc = t.leaf_centers()
    return t, xc


def test_manufactured_solution_converges_second_order():
    """Configuration c1: L-inf and L2 errors against u fall like dx^2."""
    p = I.problem("c1")
    errs = []
    for ml in (4, 5, 6, 7):  # 64^2 .. 512^2
        t, xc = _solve_error(p, ml)
        e = t.solution() - I.c1_u_vec(xc)
        errs.append((np.abs(e).max(), np.sqrt(np.mean(e * e))))
        t.close()
    errs = np.array(errs)
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 2.8) and np.all(ratios < 6.0), ratios
    assert np.exp(np.mean(np.log(ratios))) > 3.3


@pytest.mark.parametrize("dim", [2, 3])
def test_sphere_closed_form_second_order(dim):
    """Sec. 4.1: with f = |x| - R, R = 1/4, the analytic log(r/R) (2D) and
    1 - R/r (3D) solutions; the error falls like dx^2 (Fig. sphere-convergence b)."""
    p = I.problem("sphere2d" if dim == 2 else "sphere3d")
    levels = (3, 4, 5, 6) if dim == 2 else (2, 3, 4)
    errs = []
    for ml in levels:
        t, xc = _solve_error(p, ml)
        outside = np.sqrt(np.sum(xc ** 2, 1)) > 0.25
        e = (t.solution() - I.sphere_solution_vec(xc, dim))[outside]
        errs.append((np.abs(e).max(), np.sqrt(np.mean(e * e))))
        t.close()
    errs = np.array(errs)
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 2.5), ratios
    assert np.exp(np.mean(np.log(ratios[-1]))) > 3.0, ratios


def _sphere3d_max_error(ml):
    t, xc = _solve_error(I.problem("sphere3d"), ml)
    outside = np.sqrt(np.sum(xc ** 2, 1)) > 0.25
    e = np.abs(t.solution() - I.sphere_solution_vec(xc, 3))[outside].max()
    t.close()
    return e


def test_sphere3d_error_against_the_printed_value():
    """Sec. 4.1 prints a maximum error of 0.11e-3 on the 256^3 grid
    (l_max = 6) once FMG has converged.  Measured here at 64^3 and 128^3
    (3.56e-5): the error falls by 4 per halving of dx (second order), and
    the 256^3 error this order predicts, e128^2 / e64, lies below the
    printed value: with the paper's stencils and second-order walls the
    scheme is at least as accurate as the paper's.  (Measured at 256^3 it is
    8.96e-6, about 12 times below the printed value; the test below, run
    with GMG_SLOW_TESTS=1, measures it.)"""
    pv = paper_values()["sphere3d_lmax6_maxerr_fmg2"]
    e64, e128 = _sphere3d_max_error(4), _sphere3d_max_error(5)
    assert 3.5 < e64 / e128 < 4.5, (e64, e128)
    assert e128 * e128 / e64 < pv, (e64, e128)


@pytest.mark.skipif(os.environ.get("GMG_SLOW_TESTS") != "1", reason="256^3 oracle solve (about 2.5 min); GMG_SLOW_TESTS=1 runs it")
def test_sphere3d_error_at_the_printed_resolution():
    """The same problem at the printed resolution (256^3): the oracle's
    maximum error is second order from 128^3 and below the printed 0.11e-3."""
    pv = paper_values()["sphere3d_lmax6_maxerr_fmg2"]
    e128, e256 = _sphere3d_max_error(5), _sphere3d_max_error(6)
    assert 3.5 < e128 / e256 < 4.5, (e128, e256)
    assert e256 < pv, e256


def test_converged_solution_is_symmetric():
    """A sphere centred in the cube: the converged solution is invariant
    under axis reflections and permutations."""
    t = mk(3, 8, (1, 1, 1), 1 / 8, 3)
    t.set_lsf(O.LSF_SPHERE, (0.5, 0.5, 0.5, 0.2))
    t.set_walls([0] * 6, values=[0.0] * 6)
    t.store_stencils(1.0)
    t.set_rhs(np.zeros(t.num_leaf_cells()))
    k, _ = t.solve(1e-13, 40)
    assert k > 0
    xc = t.leaf_centers()
    perm, g, ext = lex_perm(xc, t.level_h(3), np.zeros(3))
    phi = np.empty(len(xc))
    phi[perm] = t.solution()[perm]
    grid = np.zeros(tuple(ext[::-1]))
    grid[g[:, 2], g[:, 1], g[:, 0]] = t.solution()
    for arr in (grid[::-1], grid[:, ::-1], grid[:, :, ::-1], grid.transpose(1, 0, 2), grid.transpose(2, 1, 0)):
        assert np.abs(arr - grid).max() <= 1e-10


def test_vcycle_reduction_is_in_multigrid_range():
    """parity unpinned (the paper prints per-FMG factors only): a sanity
    range for the per-V-cycle residual reduction on the two workloads."""
    for name in ("c1",):
        t = oracle_problem(I.problem(name))
        r0 = t.residual()[0]
        t.vcycle(2)
        r2 = t.residual()[0]
        t.vcycle(1)
        r3 = t.residual()[0]
        assert r3 / r2 < 0.15 and r2 / r0 < 0.05


# ----------------------------------------------------------------- mesh
def test_tree_is_balanced_and_tiles_the_domain():
    dim, N, h1, ml = 3, 4, 1 / 8, 5
    cb = (2, 1, 1)
    t = mk(dim, N, cb, h1, ml, refine=_refine_near([0.33, 0.41, 0.2], 0.02, N, h1, dim))
    lmin, lmax = t.levels()
    fine = np.full((cb[2] << (lmax - 1), cb[1] << (lmax - 1), cb[0] << (lmax - 1)), -1, dtype=int)
    nleaf = 0
    for lev in range(1, lmax + 1):
        bix, hc = t.level_blocks(lev)
        s = 1 << (lmax - lev)
        for b, has in zip(bix, hc):
            if has:
                continue
            sl = fine[b[2] * s:(b[2] + 1) * s, b[1] * s:(b[1] + 1) * s, b[0] * s:(b[0] + 1) * s]
            assert np.all(sl == -1), "overlapping leaves"
            sl[...] = lev
            nleaf += 1
    assert np.all(fine >= 1), "leaves do not cover the domain"
    assert len(np.unique(fine)) >= 4
    # 2:1 balance across faces, edges and corners
    for ax in range(3):
        for sh in (1, -1):
            nb = np.roll(fine, sh, axis=ax)
            valid = np.ones_like(fine, dtype=bool)
            idx = [slice(None)] * 3
            idx[ax] = 0 if sh == 1 else -1
            valid[tuple(idx)] = False
            assert np.all(np.abs(fine - nb)[valid] <= 1)
    pad = np.pad(fine, 1, mode="edge")
    Z, Y, X = fine.shape
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nb = pad[1 + dz:1 + dz + Z, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X]
                assert np.abs(fine - nb).max() <= 1
    assert t.num_leaf_cells() == sum(
        int(((fine == lev).sum() / (1 << (3 * (lmax - lev))))) * N ** 3 for lev in range(1, lmax + 1))


def test_unresolved_root_correction_places_virtual_boundary():
    """Sec. 3.6.3: a sphere much smaller than the coarse cells is found by
    gradient descent; the virtual boundary sits on the axis toward the
    sphere at the normalised distance (|a - c| - R) / dx."""
    c, R, w = np.array([0.53, 0.47, 0.51]), 0.02, 0.004
    t = mk(3, 8, (1, 1, 1), 1 / 8, 1)
    t.set_params(2, 2, 1e-8, 1.5, w)
    t.set_lsf(O.LSF_SPHERE, tuple(c) + (R,))
    t.set_walls([0] * 6, values=[0.0] * 6)
    t.store_stencils(1.0)
    d = t.get_d(1).reshape(-1, 6)
    xc = t.level_centers(1)
    h = t.level_h(1)
    mask = t.get_mask(1).ravel()
    n_checked = 0
    for i, a in enumerate(xc):
        if not mask[i]:
            continue
        roots = [sphere_roots(a, k, s, h, c, R) for k in range(3) for s in (-1, 1)]
        if any(r is not None for r in roots):
            continue
        dist = np.linalg.norm(a - c) - R
        reach = math.floor(h / w) * w
        if dist > reach - 1e-3:
            if dist > reach + 1e-3:
                assert np.all(d[i] == 1.0)
            continue
        ax = int(np.argmax(np.abs(c - a)))
        side = 1 if c[ax] - a[ax] > 0 else 0
        nb = a[ax] + (h if side else -h)
        if not (0 < nb < 1):
            continue
        assert abs(d[i, 2 * ax + side] - dist / h) < 1e-4, (d[i], dist / h)
        others = np.delete(d[i], 2 * ax + side)
        assert np.all(others == 1.0)
        n_checked += 1
    assert n_checked >= 1


@pytest.mark.parametrize("dim", [2, 3])
def test_fmg_reduction_per_cycle_in_the_printed_range(dim):
    """Sec. 4.1 prints a residual reduction of about 40-80 (2D) and 30-40
    (3D) per FMG iteration on the sphere test.  From phi = 0, FMG cycles 2-4
    reduce the residual by factors within half to twice that range, and FMG
    cycles converge to the same discrete solution as V-cycles (a broken FMG
    - no coarse right-hand side, no prolongation, no V-cycle on the way up -
    fails one of these)."""
    p = I.problem("sphere2d" if dim == 2 else "sphere3d")
    q = I.scaled(p, 5 if dim == 2 else 4)
    lo, hi = (40, 80) if dim == 2 else (30, 40)
    t = oracle_problem(q)
    res = []
    for k in range(4):
        t.fmg(1)
        l2, _, bn = t.residual()
        res.append(l2 / bn)
    factors = np.array(res[:-1]) / np.array(res[1:])
    assert np.all(factors > lo / 2) and np.all(factors < hi * 2), factors
    t.fmg(4)
    ref, _ = _solve_error(p, q["max_level"], tol=1e-13)
    a, b = t.solution(), ref.solution()
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
    t.close()
    ref.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_efield_exact_for_linear_phi(dim):
    """Sec. 4.4: the face gradients use the boundary distance next to the
    object.  For phi = a.x + c with phi_b and Dirichlet wall values taken
    from the same linear function, every face value - regular, across the
    object's boundary, at refinement boundaries (reading G) and at the walls
    - is exactly -a; cells inside the object get 0.  (The refinement region
    stays away from the walls: a refinement ghost whose tangential slope
    reaches a Dirichlet wall uses the operator's homogeneous reflection.)"""
    from _helpers import refine_near
    N, h1 = 8, 1 / 16
    c, R = (0.47, 0.52, 0.5)[:dim], 0.13
    a = np.array([0.7, -1.3, 0.4][:dim])
    lin = lambda x: float(np.dot(a, np.asarray(x)[:dim]) + 0.25)
    p = dict(dim=dim, N=N, cb=(2, 2, 2 if dim == 3 else 1), lo=(0.0, 0.0, 0.0), h1=h1, max_level=3,
             refine=refine_near([0.5, 0.5, 0.5][:dim], 0.16, N, h1, dim),
             lsf=("sphere", tuple(c) + (0.0,) * (3 - dim) + (R,)), walls=(0,) * (2 * dim), wall_values=None,
             wall_fn=lin, phib=lin, rhs=lambda xc: np.zeros(len(xc)), index=40)
    t = oracle_problem(p, rhs=False)
    levels = set(t.leaf_levels())
    assert len(levels) > 1  # refinement boundaries present
    xc = t.leaf_centers()
    t.set_solution(xc @ a + 0.25)
    E = t.efield()
    inside = np.sqrt(np.sum((xc - np.array(c)) ** 2, 1)) < R
    assert inside.any() and (~inside).any()
    assert np.abs(E[inside]).max() == 0.0
    err = np.abs(E[~inside] + a).max()
    assert err < 1e-9, err


@pytest.mark.parametrize("shape", ["spheroid", "rhombus", "heart", "astroid"])
def test_sharp_shape_distances_match_closed_form_roots(shape):
    """Sec. 4.3 shapes on a 64^2 grid: every line-search distance across the
    boundary equals the root solved by hand from the shape's equation -
    along x for the spheroid (|p| = sqrt((1 - q^2)/8)), the rhombus
    (|p| = (1.5 - |q|)/8) and the astroid (|p| = (0.8 (0.8 - |q|^(2/3)/1.5))^(3/2)),
    along y for the heart (q = |p|^(2/3) +- sqrt(1 - p^2)) - to 2 eps_tol."""
    q = I.sharp_problem(shape, 2, 4)
    q["w_min"] = 0.0
    t = oracle_problem(q, rhs=False)
    l = t.levels()[1]
    h = 1 / 64
    d = t.get_d(l).reshape(-1, 4)
    # leaf order of a uniform tree: blocks in Morton order, cells x fastest
    xc = t.leaf_centers()
    checked = 0
    for c in range(len(xc)):
        x, y = xc[c]
        P, Q = 4 * (x - 0.5), 4 * (y - 0.5)
        if shape == "heart":
            if abs(P) >= 1:
                continue
            roots = [abs(P) ** (2 / 3) + s * np.sqrt(1 - P * P) for s in (1, -1)]
            for k, step in ((3, 1), (2, -1)):  # +y and -y neighbours
                ts = [(0.5 + r / 4 - y) / (step * h) for r in roots]
                ts = [v for v in ts if 0 < v < 1]
                if ts and d[c, k] < 1:  # two roots in one segment: the nearer one
                    assert abs(d[c, k] - min(ts)) < 2e-8, (c, k, d[c, k], ts)
                    checked += 1
            continue
        if shape == "spheroid":
            if abs(Q) >= 1:
                continue
            pr = np.sqrt((1 - Q * Q) / 8)
        elif shape == "rhombus":
            if abs(Q) >= 1.5:
                continue
            pr = (1.5 - abs(Q)) / 8
        else:
            v = 0.8 * (0.8 - abs(Q) ** (2 / 3) / 1.5)
            if v <= 0:
                continue
            pr = v ** 1.5
        for k, step in ((1, 1), (0, -1)):  # +x and -x neighbours
            ts = [(xr - x) / (step * h) for xr in (0.5 + pr / 4, 0.5 - pr / 4)]
            ts = [v for v in ts if 0 < v < 1]
            if ts and d[c, k] < 1:  # two roots in one segment: the nearer one
                assert abs(d[c, k] - min(ts)) < 2e-8, (c, k, d[c, k], ts)
                checked += 1
    assert checked >= 8, checked
    t.close()


# ------------------------------------------- capsule and ellipsoid level sets
def _quad_interval(p0, p1, p2):
    """t-interval where p2 t^2 + p1 t + p0 <= 0 (p2 > 0), or None."""
    disc = p1 * p1 - 4 * p2 * p0
    if disc < 0:
        return None
    sq = math.sqrt(disc)
    return ((-p1 - sq) / (2 * p2), (-p1 + sq) / (2 * p2))


def _ball_interval(a, w, c, r):
    """t-interval of the line a + t w inside the ball |x - c| <= r."""
    u = a - c
    return _quad_interval(u @ u - r * r, 2 * (u @ w), w @ w)


def _capsule_interval(a, w, A, B, r):
    """t-interval of the line a + t w inside the capsule of radius r around
    the segment A-B (A-B along z here): the union of the two end balls and
    the finite cylinder, written out from their equations.  The capsule is
    convex, so the union is one interval."""
    parts = [_ball_interval(a, w, A, r), _ball_interval(a, w, B, r)]
    up, wp = (a - A)[:2], w[:2]
    if wp @ wp > 0:
        cyl = _quad_interval(up @ up - r * r, 2 * (up @ wp), wp @ wp)
        if cyl is not None and A[2] <= a[2] <= B[2]:  # z stays a[2] on an x or y ray
            parts.append(cyl)
    elif up @ up <= r * r:  # a z ray inside the radius: the cylinder's z range
        t0, t1 = (A[2] - a[2]) / w[2], (B[2] - a[2]) / w[2]
        parts.append((min(t0, t1), max(t0, t1)))
    parts = [q for q in parts if q is not None]
    if not parts:
        return None
    return min(q[0] for q in parts), max(q[1] for q in parts)


def _ellipsoid_interval(a, w, c, Q, S):
    """t-interval of the line a + t w inside |S^-1 Q^T (x - c)| <= 1: the
    roots of a quadratic in t, solved here."""
    u = (Q.T @ (a - c)) / S
    v = (Q.T @ w) / S
    return _quad_interval(u @ u - 1.0, 2 * (u @ v), v @ v)


def _check_distances_against_intervals(t, interval, min_checked):
    """Every line-search distance of every level equals the nearest entry or
    exit point of the body along the segment to the neighbour centre (the
    body is convex: at most two roots per segment, the nearer one kept,
    Sec. 3.2), and every cell with such a root is masked (Sec. 3.6.1)."""
    lmin, lmax = t.levels()
    checked = 0
    for lev in range(lmin, lmax + 1):
        d = t.get_d(lev).reshape(-1, 6)
        mask = t.get_mask(lev).ravel()
        xc = t.level_centers(lev)
        h = t.level_h(lev)
        for i, a in enumerate(xc):
            for k in range(3):
                for s, side in ((-1, 0), (1, 1)):
                    if not 0 <= a[k] + s * h <= 1:
                        assert d[i, 2 * k + side] == 1.0
                        continue
                    w = np.zeros(3)
                    w[k] = s * h
                    iv = interval(a, w)
                    roots = [] if iv is None else [x for x in iv if 0.0 <= x <= 1.0]
                    if not roots:
                        assert d[i, 2 * k + side] == 1.0, (lev, i, k, s)
                        continue
                    assert mask[i] == 1, "cell with a root within one cell is not masked"
                    # skip near-tangent chords, where the two roots are closer
                    # than the search resolves (Sec. 3.2)
                    if iv[1] - iv[0] > 1e-4:
                        assert abs(d[i, 2 * k + side] - max(min(roots), EPS)) <= 2 * EPS, (lev, i, k, s, roots)
                        checked += 1
    assert checked >= min_checked, checked


def test_capsule_distances_match_hand_solved_intersections():
    """The needle level set (capsule: distance to a segment minus the
    radius, reading N): distances along x, y and z on a 32^3 tree equal the
    entry points into the cylinder wall, either hemispherical cap, or past
    the segment's ends, solved from the shapes' equations."""
    A, B, r = np.array([0.47, 0.52, 0.43]), np.array([0.47, 0.52, 0.81]), 0.11
    t = mk(3, 8, (1, 1, 1), 1 / 8, 3)
    t.set_lsf(O.LSF_CAPSULE, tuple(A) + tuple(B) + (r,))
    t.set_walls([0] * 6, values=[0.0] * 6)
    t.store_stencils(1.0)
    _check_distances_against_intervals(t, lambda a, w: _capsule_interval(a, w, A, B, r), 400)
    # rays through the caps only: z rays inside the radius, and x rays
    # below the segment's lower end
    xc, h = t.level_centers(3), t.level_h(3)
    d = t.get_d(3).reshape(-1, 6)
    caps = 0
    for i, a in enumerate(xc):
        if np.hypot(*(a - A)[:2]) < r and abs(a[2] - A[2]) < 2 * h and d[i, 4] < 1:
            caps += 1
        if A[2] - r < a[2] < A[2] and d[i, 0] < 1:
            caps += 1
    assert caps >= 20, caps
    t.close()


@pytest.mark.parametrize("rotated", [False, True])
def test_ellipsoid_distances_match_hand_solved_intersections(rotated):
    """The ellipsoid level set of the batched-trees workload,
    a_min (|S^-1 Q^T (x - c)| - 1): distances on a 32^3 tree equal the roots
    of the ray-quadric equation solved here, for axis-aligned semi-axes and
    for a rotation Q (a transposed Q or swapped semi-axes fail this)."""
    c = np.array([0.48, 0.53, 0.51])
    S = np.array([0.31, 0.17, 0.23])
    if rotated:
        Q, _ = np.linalg.qr(np.random.default_rng(11).standard_normal((3, 3)))
    else:
        Q = np.eye(3)
    t = mk(3, 8, (1, 1, 1), 1 / 8, 3)
    t.set_lsf(O.LSF_ELLIPSOID, tuple(c) + tuple(Q.ravel()) + tuple(S))
    t.set_walls([0] * 6, values=[0.0] * 6)
    t.store_stencils(1.0)
    _check_distances_against_intervals(t, lambda a, w: _ellipsoid_interval(a, w, c, Q, S), 400)
    t.close()
