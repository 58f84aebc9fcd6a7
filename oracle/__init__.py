"""Serial FP64 oracle for the octree geometric-multigrid Poisson solver with
level-set Dirichlet boundaries (arXiv 2205.09411).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously correct
CPU implementation written from the paper (``gmg_oracle.c``, serial C in
FP64) against which the CUDA library is checked.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product package never does, and the oracle imports nothing from the
product package.

The C library is compiled on first use (``build()``) with
``gcc -O2 -ffp-contract=off`` so that no multiply-add contraction changes the
IEEE results of the level-set and line-search arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmg_oracle.c")
_HDR = os.path.join(_HERE, "gmg_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgmg_oracle.so")
_lib = None
_lock = threading.Lock()

LSF_NONE, LSF_SPHERE, LSF_CAPSULE, LSF_ELLIPSOID, LSF_CALLBACK, LSF_SHAPE, LSF_GRID = 0, 1, 2, 3, 4, 5, 6
WALL_DIRICHLET, WALL_NEUMANN = 0, 1

FN = C.CFUNCTYPE(C.c_double, C.POINTER(C.c_double), C.c_void_p)
REFINE_FN = C.CFUNCTYPE(C.c_int, C.c_int, C.POINTER(C.c_int), C.c_void_p)


class LSF(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 16), ("fn", FN), ("user", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH) or
             os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
            vp = C.c_void_p
            sig = {
                "ot_create": (vp, [C.c_int, C.c_int, ip, dp, C.c_double, C.c_int, REFINE_FN, vp, C.c_int]),
                "ot_destroy": (None, [vp]),
                "ot_levels": (None, [vp, ip, ip]),
                "ot_level_nblocks": (C.c_int, [vp, C.c_int]),
                "ot_level_n": (C.c_int, [vp, C.c_int]),
                "ot_level_h": (C.c_double, [vp, C.c_int]),
                "ot_level_blocks": (None, [vp, C.c_int, ip, ip]),
                "ot_num_leaf_cells": (C.c_int64, [vp]),
                "ot_leaf_centers": (None, [vp, dp]),
                "ot_leaf_levels": (None, [vp, ip]),
                "ot_set_params": (None, [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]),
                "ot_set_walls": (None, [vp, ip, dp, FN, vp]),
                "ot_set_lsf": (None, [vp, C.POINTER(LSF)]),
                "ot_store_stencils": (C.c_int, [vp, FN, vp, C.c_double]),
                "ot_num_cut_blocks": (C.c_int, [vp, C.c_int]),
                "ot_set_rhs": (None, [vp, dp]),
                "ot_set_solution": (None, [vp, dp]),
                "ot_get_solution": (None, [vp, dp]),
                "ot_get_level": (None, [vp, C.c_int, C.c_int, dp]),
                "ot_vcycle": (None, [vp, C.c_int]),
                "ot_fmg": (None, [vp, C.c_int]),
                "ot_efield": (None, [vp, dp]),
                "ot_residual": (C.c_double, [vp, dp, dp, dp]),
                "ot_solve": (C.c_int, [vp, C.c_double, C.c_int, dp]),
                "ot_line_search": (C.c_double, [FN, vp, C.c_int, dp, dp, C.c_double]),
                "ot_lsf_eval": (C.c_double, [C.POINTER(LSF), C.c_int, dp]),
                "ot_get_d": (None, [vp, C.c_int, dp]),
                "ot_get_mask": (None, [vp, C.c_int, ip]),
                "ot_apply_composite": (None, [vp, dp, dp, C.c_int]),
                "ot_composite_matrix": (C.c_int, [vp, dp, dp]),
                "ot_prolong_test": (None, [vp, C.c_int, dp, dp]),
                "ot_restrict_test": (None, [vp, C.c_int, dp, dp]),
                "ot_lu_solve": (C.c_int, [C.c_int, dp, dp, dp]),
                "ot_halfsweep": (None, [vp, C.c_int, C.c_int]),
                "ot_level_residual": (None, [vp, C.c_int, dp]),
                "ot_set_level": (None, [vp, C.c_int, C.c_int, dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _as_fn(f):
    """Wrap a Python callable f(x: ndarray[3]) -> float as a C callback."""
    if f is None:
        return FN()

    def cb(xp, _u):
        return float(f(np.ctypeslib.as_array(xp, shape=(3,)).copy()))

    return FN(cb)


def make_lsf(kind, params=(), fn=None):
    s = LSF()
    s.kind = kind
    for i, v in enumerate(params):
        s.p[i] = float(v)
    s.fn = _as_fn(fn) if fn is not None else FN()
    s._keep = s.fn
    return s


def make_grid_lsf(values, origin, spacing):
    """LSF_GRID from samples values[i, j(, k)] at origin + (i, j, k) * spacing
    (the samples are kept alive with the struct)."""
    values = np.asarray(values, dtype=np.float64)
    samples = np.ascontiguousarray(values.transpose())  # x fastest
    s = LSF()
    s.kind = LSF_GRID
    for d in range(values.ndim):
        s.p[d] = float(values.shape[d])
        s.p[3 + d] = float(origin[d])
        s.p[6 + d] = float(spacing)
    s.fn = FN()
    s.user = samples.ctypes.data
    s._keep = samples
    return s


def lsf_eval(lsf: LSF, dim: int, x) -> float:
    xx = np.zeros(3)
    xx[:len(x)] = x
    return lib().ot_lsf_eval(C.byref(lsf), dim, _dp(xx))


def line_search(f, dim, a, b, eps_tol=1e-8) -> float:
    """Relative distance from a toward b to the first root (Sec. 3.2)."""
    aa, bb = np.zeros(3), np.zeros(3)
    aa[:len(a)] = a
    bb[:len(b)] = b
    cb = _as_fn(f)
    return lib().ot_line_search(cb, None, dim, _dp(aa), _dp(bb), eps_tol)


def lu_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    rc = lib().ot_lu_solve(len(b), _dp(A), _dp(b), _dp(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return x


class OracleTree:
    """One problem: tree + geometry + right-hand side (all FP64, serial)."""

    def __init__(self, dim, N, cb=(1, 1, 1), lo=(0.0, 0.0, 0.0), h1=None, max_level=1, refine=None,
                 max_coarse_cells=None):
        L = lib()
        self.dim, self.N = dim, N
        cb = np.array(list(cb) + [1] * (3 - len(cb)), dtype=np.int32)[:3]
        lo = np.array(list(lo) + [0.0] * (3 - len(lo)), dtype=np.float64)[:3]
        if h1 is None:
            h1 = 1.0 / (cb[0] * N)
        if max_coarse_cells is None:
            max_coarse_cells = 64 if dim == 2 else 512
        if refine is None:
            self._refine = REFINE_FN()
        else:
            def rcb(level, bix, _u):
                return 1 if refine(level, (bix[0], bix[1], bix[2])) else 0
            self._refine = REFINE_FN(rcb)
        self._cb, self._lo = cb, lo
        self.h = L.ot_create(dim, N, _ip(cb), _dp(lo), float(h1), max_level, self._refine, None,
                             max_coarse_cells)
        if not self.h:
            raise ValueError("invalid tree parameters")
        self._keep = []

    def close(self):
        if self.h:
            lib().ot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- structure -------------------------------------------------------
    def levels(self):
        a, b = C.c_int(), C.c_int()
        lib().ot_levels(self.h, C.byref(a), C.byref(b))
        return a.value, b.value

    def level_blocks(self, level):
        nb = lib().ot_level_nblocks(self.h, level)
        bix = np.zeros((nb, 3), dtype=np.int32)
        hc = np.zeros(nb, dtype=np.int32)
        if nb:
            lib().ot_level_blocks(self.h, level, _ip(bix), _ip(hc))
        return bix, hc

    def level_n(self, level):
        return lib().ot_level_n(self.h, level)

    def level_h(self, level):
        return lib().ot_level_h(self.h, level)

    def num_leaf_cells(self):
        return int(lib().ot_num_leaf_cells(self.h))

    def leaf_centers(self):
        n = self.num_leaf_cells()
        x = np.zeros((n, self.dim))
        lib().ot_leaf_centers(self.h, _dp(x))
        return x

    def leaf_levels(self):
        n = self.num_leaf_cells()
        v = np.zeros(n, dtype=np.int32)
        lib().ot_leaf_levels(self.h, _ip(v))
        return v

    # --- set-up ----------------------------------------------------------
    def set_params(self, n_down=2, n_up=2, eps_tol=1e-8, mask_factor=1.5, w_min=0.0):
        lib().ot_set_params(self.h, n_down, n_up, eps_tol, mask_factor, w_min)

    def set_walls(self, types, values=None, fn=None):
        t = np.zeros(6, dtype=np.int32)
        t[:len(types)] = types
        v = np.zeros(6)
        if values is not None:
            v[:len(values)] = values
        cb = _as_fn(fn)
        self._keep.append(cb)
        lib().ot_set_walls(self.h, _ip(t), _dp(v), cb, None)

    def set_lsf(self, kind, params=(), fn=None):
        s = make_lsf(kind, params, fn)
        self._keep.append(s)
        lib().ot_set_lsf(self.h, C.byref(s))

    def set_lsf_grid(self, values, origin, spacing):
        """Level set sampled at origin + (i, j[, k]) * spacing: values[i, j(, k)]."""
        s = make_grid_lsf(values, origin, spacing)
        self._keep.append(s)
        lib().ot_set_lsf(self.h, C.byref(s))

    def store_stencils(self, phib=0.0):
        if callable(phib):
            cb = _as_fn(phib)
            self._keep.append(cb)
            return lib().ot_store_stencils(self.h, cb, None, 0.0)
        return lib().ot_store_stencils(self.h, FN(), None, float(phib))

    def num_cut_blocks(self, level):
        return lib().ot_num_cut_blocks(self.h, level)

    def get_d(self, level):
        nb, n = lib().ot_level_nblocks(self.h, level), self.level_n(level)
        out = np.zeros(nb * n ** self.dim * 2 * self.dim)
        lib().ot_get_d(self.h, level, _dp(out))
        return out.reshape(nb, n ** self.dim, 2 * self.dim)

    def get_mask(self, level):
        nb, n = lib().ot_level_nblocks(self.h, level), self.level_n(level)
        out = np.zeros(nb * n ** self.dim, dtype=np.int32)
        lib().ot_get_mask(self.h, level, _ip(out))
        return out.reshape(nb, n ** self.dim)

    # --- solve -----------------------------------------------------------
    def set_rhs(self, g):
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert g.shape == (self.num_leaf_cells(),)
        lib().ot_set_rhs(self.h, _dp(g))

    def set_solution(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        lib().ot_set_solution(self.h, _dp(phi))

    def solution(self):
        out = np.zeros(self.num_leaf_cells())
        lib().ot_get_solution(self.h, _dp(out))
        return out

    def get_level(self, level, which=0):
        nb, n = lib().ot_level_nblocks(self.h, level), self.level_n(level)
        out = np.zeros(nb * n ** self.dim)
        lib().ot_get_level(self.h, level, which, _dp(out))
        return out

    def vcycle(self, n=1):
        lib().ot_vcycle(self.h, n)

    def fmg(self, n=1):
        lib().ot_fmg(self.h, n)

    def efield(self):
        out = np.zeros((self.num_leaf_cells(), self.dim))
        lib().ot_efield(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def residual(self, want_field=False):
        linf, bn = C.c_double(), C.c_double()
        r = np.zeros(self.num_leaf_cells()) if want_field else None
        l2 = lib().ot_residual(self.h, C.byref(linf), C.byref(bn), _dp(r) if want_field else None)
        if want_field:
            return l2, linf.value, bn.value, r
        return l2, linf.value, bn.value

    def solve(self, rel_tol=1e-8, max_cycles=50):
        hist = np.zeros(max_cycles)
        k = lib().ot_solve(self.h, rel_tol, max_cycles, _dp(hist))
        return k, hist[:abs(k)]

    # --- pieces for the pins --------------------------------------------
    def apply_composite(self, phi, with_bterm=True):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        out = np.zeros_like(phi)
        lib().ot_apply_composite(self.h, _dp(phi), _dp(out), 1 if with_bterm else 0)
        return out

    def composite_matrix(self):
        n = self.num_leaf_cells()
        A = np.zeros((n, n))
        b = np.zeros(n)
        lib().ot_composite_matrix(self.h, _dp(A), _dp(b))
        return A, b

    def prolong_test(self, level, coarse):
        coarse = np.ascontiguousarray(coarse, dtype=np.float64)
        nb, n = lib().ot_level_nblocks(self.h, level), self.level_n(level)
        fine = np.zeros(nb * n ** self.dim)
        lib().ot_prolong_test(self.h, level, _dp(coarse), _dp(fine))
        return fine

    def restrict_test(self, level, fine):
        fine = np.ascontiguousarray(fine, dtype=np.float64)
        nb, n = lib().ot_level_nblocks(self.h, level - 1), self.level_n(level - 1)
        coarse = np.zeros(nb * n ** self.dim)
        lib().ot_restrict_test(self.h, level, _dp(fine), _dp(coarse))
        return coarse

    def halfsweep(self, level, color):
        lib().ot_halfsweep(self.h, level, color)

    def level_residual(self, level):
        nb, n = lib().ot_level_nblocks(self.h, level), self.level_n(level)
        out = np.zeros(nb * n ** self.dim)
        lib().ot_level_residual(self.h, level, _dp(out))
        return out

    def set_level(self, level, values, which=0):
        values = np.ascontiguousarray(values, dtype=np.float64)
        lib().ot_set_level(self.h, level, which, _dp(values))

    def level_centers(self, level):
        """Cell centres of a level in canonical order (for building test fields)."""
        bix, _ = self.level_blocks(level)
        n, h = self.level_n(level), self.level_h(level)
        rng = np.arange(n)
        if self.dim == 2:
            yy, xx = np.meshgrid(rng, rng, indexing="ij")
            loc = np.stack([xx.ravel(), yy.ravel()], 1)
        else:
            zz, yy, xx = np.meshgrid(rng, rng, rng, indexing="ij")
            loc = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1)
        out = []
        for b in bix:
            g = b[:self.dim] * n + loc
            out.append(self._lo[:self.dim] + (g + 0.5) * h)
        return np.concatenate(out, 0)
