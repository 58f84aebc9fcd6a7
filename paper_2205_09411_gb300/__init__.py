"""GB300-native octree geometric-multigrid Poisson solver with level-set
Dirichlet boundaries (method of Teunissen & Schiavello, arXiv 2205.09411).

This module is a thin ctypes binding of the CUDA library ``libgmg.so`` (C ABI
in ``include/gmg.h``): it marshals arguments and allocates the device
workspace through PyTorch.  Every step of the solver runs in the library's
CUDA kernels; there is no CPU fallback.  Importing works without a GPU (the
tree and its set-up are host work); calls that need the device raise if the
library or CUDA is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["Tree", "Forest", "load", "build", "GmgError", "FP64", "MIXED", "MIXED_BF16", "LIB_PATH"]

LIB_PATH = _build.LIB
FP64, MIXED, MIXED_BF16 = 0, 1, 2
HOST, DEVICE = 0, 1
WALL_DIRICHLET, WALL_NEUMANN = 0, 1
LSF_KINDS = {"none": 0, "sphere": 1, "capsule": 2, "ellipsoid": 3, "callback": 4, "shape": 5, "grid": 6}

FN = C.CFUNCTYPE(C.c_double, C.POINTER(C.c_double), C.c_void_p)
REFINE_FN = C.CFUNCTYPE(C.c_int, C.c_int, C.POINTER(C.c_int), C.c_void_p)


class Domain(C.Structure):
    _fields_ = [("dim", C.c_int), ("block_n", C.c_int), ("coarse_blocks", C.c_int * 3), ("lo", C.c_double * 3),
                ("h_root", C.c_double), ("max_level", C.c_int), ("max_coarse_cells", C.c_int),
                ("refine", REFINE_FN), ("refine_user", C.c_void_p)]


class Lsf(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 16), ("fn", FN), ("user", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("n_down", C.c_int), ("n_up", C.c_int), ("eps_tol", C.c_double), ("mask_factor", C.c_double),
                ("w_min", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("rel_l2", C.c_double), ("linf", C.c_double), ("bnorm", C.c_double)]


class GmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gmg error %d: %s" % (code, msg))
        self.code = code


_lib = None


def build(force=False, verbose=False):
    """Compile libgmg.so for sm_103a (in-tree)."""
    return _build.build(force=force, verbose=verbose)


def load():
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgmg.so is missing (%s): run __graft_entry__.build() or "
                           "python -m paper_2205_09411_gb300.build" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, dp, ip, sz = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_size_t
    sigs = {
        "gmg_default_params": (None, [C.POINTER(Params)]),
        "gmg_tree_create": (C.c_int, [C.POINTER(Domain), C.POINTER(Params), C.POINTER(vp)]),
        "gmg_tree_destroy": (None, [vp]),
        "gmg_tree_info": (C.c_int, [vp, ip, ip, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "gmg_level_info": (C.c_int, [vp, C.c_int, ip, ip, dp]),
        "gmg_level_blocks": (C.c_int, [vp, C.c_int, ip, ip]),
        "gmg_leaf_centers": (C.c_int, [vp, dp]),
        "gmg_set_walls": (C.c_int, [vp, ip, dp, FN, vp]),
        "gmg_store_stencils": (C.c_int, [vp, C.POINTER(Lsf), FN, vp, C.c_double]),
        "gmg_set_boundary_value": (C.c_int, [vp, FN, vp, C.c_double]),
        "gmg_get_boundary_terms": (C.c_int, [vp, C.c_int, dp]),
        "gmg_workspace_bytes": (C.c_int, [vp, C.POINTER(sz)]),
        "gmg_tree_bind": (C.c_int, [vp, vp, sz]),
        "gmg_set_num_rhs": (C.c_int, [vp, C.c_int]),
        "gmg_num_rhs": (C.c_int, [vp]),
        "gmg_set_rhs": (C.c_int, [vp, vp, C.c_int, vp]),
        "gmg_set_rhs_slots": (C.c_int, [vp, C.c_int, C.c_int, vp, C.c_int, vp]),
        "gmg_get_solution_slots": (C.c_int, [vp, C.c_int, C.c_int, vp, C.c_int, vp]),
        "gmg_iterate": (C.c_int, [vp, C.c_int, ip, C.c_int, dp, dp, vp]),
        "gmg_forest_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(vp)]),
        "gmg_tree_remesh": (C.c_int, [vp, REFINE_FN, vp, C.c_int, C.POINTER(vp)]),
        "gmg_setup_counts": (C.c_int, [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "gmg_setup_on_device": (C.c_int, [vp]),
        "gmg_transfer_solution": (C.c_int, [vp, vp, vp]),
        "gmg_iterate_begin": (C.c_int, [vp, C.c_int, ip, C.c_int, vp]),
        "gmg_iterate_end": (C.c_int, [vp, dp, dp]),
        "gmg_set_level_sweeps": (C.c_int, [vp, C.c_int, C.c_int, C.c_int]),
        "gmg_get_level_sweeps": (C.c_int, [vp, C.c_int, ip, ip]),
        "gmg_num_trees": (C.c_int, [vp]),
        "gmg_forest_tree_info": (C.c_int, [vp, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "gmg_set_solution": (C.c_int, [vp, vp, C.c_int, vp]),
        "gmg_get_solution": (C.c_int, [vp, vp, C.c_int, vp]),
        "gmg_vcycle": (C.c_int, [vp, C.c_int, vp]),
        "gmg_fmg": (C.c_int, [vp, C.c_int, vp]),
        "gmg_efield": (C.c_int, [vp, vp, C.c_int, vp]),
        "gmg_residual": (C.c_int, [vp, dp, dp, vp]),
        "gmg_solve": (C.c_int, [vp, C.c_int, C.c_double, C.c_int, C.POINTER(Stats), vp]),
        "gmg_solve_history": (C.c_int, [vp, C.c_int, C.c_double, C.c_int, dp, C.POINTER(Stats), vp]),
        "gmg_get_level": (C.c_int, [vp, C.c_int, C.c_int, dp, vp]),
        "gmg_get_distances": (C.c_int, [vp, C.c_int, dp]),
        "gmg_get_mask": (C.c_int, [vp, C.c_int, ip]),
        "gmg_num_cut_blocks": (C.c_int, [vp, C.c_int]),
        "gmg_cut_counts": (C.c_int, [vp, C.c_int, ip]),
        "gmg_last_launch_count": (C.c_longlong, [vp]),
        "gmg_profile_enable": (C.c_int, [vp, C.c_int]),
        "gmg_profile_read": (C.c_int, [vp, C.c_int, ip, ip, ip, C.POINTER(C.c_longlong), dp]),
        "gmg_set_option": (C.c_int, [vp, C.c_int, C.c_longlong]),
        "gmg_selftest_barrier_timeout": (C.c_int, [vp, C.c_longlong, vp]),
        "gmg_selftest_conversions": (C.c_int, [vp, vp, C.c_longlong, vp, vp]),
        "gmg_error_string": (C.c_char_p, [C.c_int]),
        "gmg_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# Exceptions raised by Python callbacks while the library runs them: ctypes
# cannot let them cross the C frames, so the callback records the exception,
# returns a neutral value, and _check raises it once the library call is over.
_callback_errors = []


def _check(rc):
    if _callback_errors:
        err = _callback_errors[0]
        _callback_errors.clear()
        raise RuntimeError("a Python callback raised during the library call: %r" % (err,)) from err
    if rc != 0:
        L = load()
        raise GmgError(rc, "%s: %s" % (L.gmg_error_string(rc).decode(), L.gmg_last_error().decode()))


def _fn(f):
    if f is None:
        return FN()

    def cb(xp, _u):
        try:
            return float(f(np.ctypeslib.as_array(xp, shape=(3,)).copy()))
        except BaseException as e:  # noqa: BLE001 - re-raised by _check
            _callback_errors.append(e)
            return float("nan")
    return FN(cb)


def _refine_fn(refine):
    def cb(level, bix, _u):
        try:
            return 1 if refine(level, (bix[0], bix[1], bix[2])) else 0
        except BaseException as e:  # noqa: BLE001 - re-raised by _check
            _callback_errors.append(e)
            return 0
    return REFINE_FN(cb)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def selftest_conversions(x, f, mismatches, stream=None):
    """gmg_selftest_conversions on device tensors: x float64 and f float32 of
    one length, mismatches int64 of 2 (overwritten with the counts)."""
    n = x.numel()
    assert f.numel() == n and mismatches.numel() == 2
    _check(load().gmg_selftest_conversions(C.c_void_p(x.data_ptr()), C.c_void_p(f.data_ptr()), n,
                                           C.c_void_p(mismatches.data_ptr()), _stream_ptr(stream)))


class Tree:
    """One Poisson problem on a block-structured quadtree/octree.

    Life cycle: ``Tree(...)`` (host tree) -> ``set_walls`` -> ``store_stencils``
    (boundary set-up) -> ``bind()`` (device workspace) -> ``set_rhs`` ->
    ``vcycle`` / ``solve`` -> ``solution``.  With ``nrhs`` > 1 the tree holds
    that many right-hand-side slots: leaf arrays are then (nrhs, n_leaf_cells)
    and residuals / statistics are per slot.
    """

    def __init__(self, dim, block_n, coarse_blocks=(1, 1, 1), lo=(0.0, 0.0, 0.0), h_root=None, max_level=1,
                 refine=None, max_coarse_cells=0, n_down=2, n_up=2, eps_tol=1e-8, mask_factor=1.5, w_min=0.0,
                 nrhs=1):
        L = load()
        self.dim = dim
        cb = list(coarse_blocks) + [1] * (3 - len(coarse_blocks))
        lo = list(lo) + [0.0] * (3 - len(lo))
        if h_root is None:
            h_root = 1.0 / (cb[0] * block_n)
        dom = Domain()
        dom.dim, dom.block_n = dim, block_n
        for d in range(3):
            dom.coarse_blocks[d] = int(cb[d])
            dom.lo[d] = float(lo[d])
        dom.h_root, dom.max_level, dom.max_coarse_cells = float(h_root), int(max_level), int(max_coarse_cells)
        if refine is not None:
            self._refine = _refine_fn(refine)
        else:
            self._refine = REFINE_FN()
        dom.refine = self._refine
        prm = Params(n_down, n_up, eps_tol, mask_factor, w_min)
        h = C.c_void_p()
        _check(L.gmg_tree_create(C.byref(dom), C.byref(prm), C.byref(h)))
        self._adopt(h, dim, block_n)
        if nrhs != 1:
            self.set_num_rhs(nrhs)

    def _adopt(self, h, dim, block_n):
        L = load()
        self.h = h
        self.dim = dim
        self._keep = []
        self._ws = None
        lmin, lmax, nleaf, nb = C.c_int(), C.c_int(), C.c_longlong(), C.c_longlong()
        _check(L.gmg_tree_info(self.h, C.byref(lmin), C.byref(lmax), C.byref(nleaf), C.byref(nb)))
        self.lmin, self.lmax, self.n_leaf_cells, self.n_blocks = lmin.value, lmax.value, nleaf.value, nb.value
        self.block_n = block_n
        self.nrhs = 1
        self.ntree = L.gmg_num_trees(self.h)

    @property
    def units(self):
        """(slot, tree) pairs: the independent problems the tree solves."""
        return self.nrhs * self.ntree

    def remesh(self, refine, max_level):
        """A new (unbound) tree on this tree's domain and set-up, refined by
        refine(level, bix) -> bool; blocks present here reuse their set-up."""
        L = load()
        cb = _refine_fn(refine)
        h = C.c_void_p()
        _check(L.gmg_tree_remesh(self.h, cb, None, int(max_level), C.byref(h)))
        t = Tree.__new__(Tree)
        t._adopt(h, self.dim, self.block_n)
        t._keep = list(self._keep) + [cb]
        return t

    def setup_on_device(self):
        """True when the last store_stencils ran its boundary detection on the device."""
        return bool(load().gmg_setup_on_device(self.h))

    def setup_counts(self):
        """(blocks set up, blocks taken from the previous tree)."""
        a, b = C.c_longlong(), C.c_longlong()
        _check(load().gmg_setup_counts(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def transfer_solution_from(self, old, stream=None):
        _check(load().gmg_transfer_solution(old.h, self.h, _stream_ptr(stream)))

    def set_num_rhs(self, nrhs):
        """Right-hand-side slots of the workspace (before bind)."""
        _check(load().gmg_set_num_rhs(self.h, int(nrhs)))
        self.nrhs = int(nrhs)

    def close(self):
        if getattr(self, "h", None):
            load().gmg_tree_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- host-side structure ---------------------------------------------
    def level_blocks(self, level):
        nb = self.level_nblocks(level)
        bix = np.zeros((nb, 3), dtype=np.int32)
        hc = np.zeros(nb, dtype=np.int32)
        _check(load().gmg_level_blocks(self.h, level, bix.ctypes.data_as(C.POINTER(C.c_int)),
                                       hc.ctypes.data_as(C.POINTER(C.c_int))))
        return bix, hc

    def level_info(self, level):
        nb, n, h = C.c_int(), C.c_int(), C.c_double()
        _check(load().gmg_level_info(self.h, level, C.byref(nb), C.byref(n), C.byref(h)))
        return nb.value, n.value, h.value

    def level_nblocks(self, level):
        return self.level_info(level)[0]

    def level_n(self, level):
        return self.level_info(level)[1]

    def level_h(self, level):
        return self.level_info(level)[2]

    def leaf_centers(self):
        x = np.zeros((self.n_leaf_cells, self.dim))
        _check(load().gmg_leaf_centers(self.h, x.ctypes.data_as(C.POINTER(C.c_double))))
        return x

    # --- set-up -------------------------------------------------------------
    def set_walls(self, types, values=None, fn=None):
        t = np.zeros(6, dtype=np.int32)
        t[:len(types)] = types
        v = np.zeros(6)
        if values is not None:
            v[:len(values)] = values
        cb = _fn(fn)
        self._keep.append(cb)
        _check(load().gmg_set_walls(self.h, t.ctypes.data_as(C.POINTER(C.c_int)),
                                    v.ctypes.data_as(C.POINTER(C.c_double)), cb, None))

    def store_stencils(self, lsf=None, phib=0.0):
        """lsf: None, (kind, params) with kind in LSF_KINDS, a callable f(x), or
        ("grid", (values, origin, spacing)) with values[i, j(, k)] the level set
        at origin + (i, j, k) * spacing (interpolated (bi/tri)linearly)."""
        s = Lsf()
        if lsf is None:
            s.kind = 0
        elif callable(lsf):
            s.kind = LSF_KINDS["callback"]
            s.fn = _fn(lsf)
            self._keep.append(s.fn)
        elif lsf[0] == "grid":
            values, origin, spacing = lsf[1]
            values = np.asarray(values, dtype=np.float64)
            assert values.ndim == self.dim
            samples = np.ascontiguousarray(values.transpose())  # x fastest
            self._keep.append(samples)
            s.kind = LSF_KINDS["grid"]
            for d in range(self.dim):
                s.p[d] = float(values.shape[d])
                s.p[3 + d] = float(origin[d])
                s.p[6 + d] = float(spacing[d] if np.ndim(spacing) else spacing)
            s.user = samples.ctypes.data
            s.fn = FN()
        else:
            kind, params = lsf
            s.kind = LSF_KINDS[kind]
            for i, v in enumerate(params):
                s.p[i] = float(v)
            s.fn = FN()
        self._keep.append(s)
        if callable(phib):
            cb = _fn(phib)
            self._keep.append(cb)
            _check(load().gmg_store_stencils(self.h, C.byref(s), cb, None, 0.0))
        else:
            _check(load().gmg_store_stencils(self.h, C.byref(s), FN(), None, float(phib)))

    def set_boundary_value(self, phib):
        """New boundary value (constant or callable f(x)) on the stored boundary:
        boundary terms recomputed from the stored distances, no line search."""
        if callable(phib):
            cb = _fn(phib)
            self._keep.append(cb)
            _check(load().gmg_set_boundary_value(self.h, cb, None, 0.0))
        else:
            _check(load().gmg_set_boundary_value(self.h, FN(), None, float(phib)))

    def boundary_terms(self, level):
        """(blocks, n^dim): the right-hand-side boundary term of every cell of a level."""
        nb, n = self.level_nblocks(level), self.level_n(level)
        out = np.zeros(nb * n ** self.dim)
        _check(load().gmg_get_boundary_terms(self.h, level, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out.reshape(nb, n ** self.dim)

    def num_cut_blocks(self, level):
        return load().gmg_num_cut_blocks(self.h, level)

    def distances(self, level):
        nb, n = self.level_nblocks(level), self.level_n(level)
        out = np.zeros(nb * n ** self.dim * 2 * self.dim)
        _check(load().gmg_get_distances(self.h, level, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out.reshape(nb, n ** self.dim, 2 * self.dim)

    def cut_counts(self, level):
        """(blocks, 2): per block of the level, the cells of colour 0 and 1
        ((x+y+z) even / odd) that the kernels' cut lists hold."""
        out = np.zeros(2 * self.level_nblocks(level), dtype=np.int32)
        _check(load().gmg_cut_counts(self.h, level, out.ctypes.data_as(C.POINTER(C.c_int))))
        return out.reshape(-1, 2)

    def mask(self, level):
        nb, n = self.level_nblocks(level), self.level_n(level)
        out = np.zeros(nb * n ** self.dim, dtype=np.int32)
        _check(load().gmg_get_mask(self.h, level, out.ctypes.data_as(C.POINTER(C.c_int))))
        return out.reshape(nb, n ** self.dim)

    def workspace_bytes(self):
        b = C.c_size_t()
        _check(load().gmg_workspace_bytes(self.h, C.byref(b)))
        return b.value

    def bind(self, device_ptr=None):
        """Bind device memory: a PyTorch allocation (default) or a given pointer."""
        nbytes = self.workspace_bytes()
        if device_ptr is None:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("CUDA device required: the solver has no CPU path")
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            ptr = (self._ws.data_ptr() + 255) // 256 * 256
        else:
            ptr = int(device_ptr)
        _check(load().gmg_tree_bind(self.h, C.c_void_p(ptr), C.c_size_t(nbytes)))

    # --- solve ----------------------------------------------------------------
    def _arr(self, a):
        """(pointer, where) of a float64 numpy array or CUDA tensor."""
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._hold = a
            return C.c_void_p(a.ctypes.data), HOST
        import torch
        assert a.dtype == torch.float64 and a.is_contiguous()
        return C.c_void_p(a.data_ptr()), (DEVICE if a.is_cuda else HOST)

    def _leaf_shape(self, k):
        return (self.n_leaf_cells,) if self.nrhs == 1 and k == 1 else (k, self.n_leaf_cells)

    def set_rhs(self, g, stream=None):
        """g: (n_leaf_cells,) or (nrhs, n_leaf_cells), numpy or torch float64."""
        assert int(np.prod(g.shape)) == self.nrhs * self.n_leaf_cells
        p, where = self._arr(g)
        _check(load().gmg_set_rhs(self.h, p, where, _stream_ptr(stream)))

    def set_rhs_slots(self, slot0, g, stream=None):
        """New right-hand sides for slots slot0 .. slot0 + k - 1 (g: (k, n) or (n,))."""
        k = int(np.prod(g.shape)) // self.n_leaf_cells
        assert k * self.n_leaf_cells == int(np.prod(g.shape))
        p, where = self._arr(g)
        _check(load().gmg_set_rhs_slots(self.h, int(slot0), k, p, where, _stream_ptr(stream)))

    def set_solution(self, phi, stream=None):
        assert int(np.prod(phi.shape)) == self.nrhs * self.n_leaf_cells
        p, where = self._arr(phi)
        _check(load().gmg_set_solution(self.h, p, where, _stream_ptr(stream)))

    def solution(self, out=None, stream=None):
        """Leaf values of every slot: (n_leaf_cells,) for one slot, else (nrhs, n_leaf_cells)."""
        if out is None:
            out = np.zeros(self._leaf_shape(self.nrhs))
        p, where = self._arr(out)
        _check(load().gmg_get_solution(self.h, p, where, _stream_ptr(stream)))
        return out

    def solution_slots(self, slot0, nslots=1, out=None, stream=None):
        if out is None:
            out = np.zeros((nslots, self.n_leaf_cells))
        p, where = self._arr(out)
        _check(load().gmg_get_solution_slots(self.h, int(slot0), int(nslots), p, where, _stream_ptr(stream)))
        return out

    def get_level(self, level, which=0, stream=None):
        """phi (which=0) or b (1) of every cell of a level (slot-major for several slots)."""
        nb, n = self.level_nblocks(level), self.level_n(level)
        out = np.zeros(self.nrhs * nb * n ** self.dim)
        _check(load().gmg_get_level(self.h, level, which, out.ctypes.data_as(C.POINTER(C.c_double)),
                                    _stream_ptr(stream)))
        return out if self.nrhs == 1 else out.reshape(self.nrhs, -1)

    def vcycle(self, n=1, stream=None):
        _check(load().gmg_vcycle(self.h, n, _stream_ptr(stream)))

    def efield(self, out=None, stream=None):
        """E = -grad(phi) on the upper faces of every leaf cell: (n_leaf, dim),
        or (nrhs, n_leaf, dim) for several slots."""
        if out is None:
            shape = (self.n_leaf_cells, self.dim) if self.nrhs == 1 else (self.nrhs, self.n_leaf_cells, self.dim)
            out = np.zeros(shape)
        p, where = self._arr(out)
        _check(load().gmg_efield(self.h, p, where, _stream_ptr(stream)))
        return out

    def fmg(self, n=1, stream=None):
        """n FMG cycles in FP64 (Sec. 2.2)."""
        _check(load().gmg_fmg(self.h, n, _stream_ptr(stream)))

    def residual(self, stream=None):
        """(relative L2, max) of the composite residual: floats for one unit, else
        arrays over the units (slot r, tree i) at r * ntree + i."""
        U = self.units
        r, m = np.zeros(U), np.zeros(U)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        _check(load().gmg_residual(self.h, dp(r), dp(m), _stream_ptr(stream)))
        return (float(r[0]), float(m[0])) if U == 1 else (r, m)

    def iterate(self, precision, active, residual_only=False, stream=None):
        """One solve-loop step on the units with active[u] != 0; returns (rel_l2, linf) arrays."""
        U = self.units
        a = np.ascontiguousarray(np.asarray(active, dtype=np.int32).reshape(U))
        r, m = np.zeros(U), np.zeros(U)
        dp = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
        _check(load().gmg_iterate(self.h, precision, a.ctypes.data_as(C.POINTER(C.c_int)), 1 if residual_only else 0,
                                  dp(r), dp(m), _stream_ptr(stream)))
        return r, m

    def iterate_begin(self, precision, active, residual_only=False, stream=None):
        """Enqueue one solve-loop step (see iterate) without waiting for it."""
        a = np.ascontiguousarray(np.asarray(active, dtype=np.int32).reshape(self.units))
        _check(load().gmg_iterate_begin(self.h, precision, a.ctypes.data_as(C.POINTER(C.c_int)),
                                        1 if residual_only else 0, _stream_ptr(stream)))

    def iterate_end(self):
        """Wait for the step in flight; returns (rel_l2, linf) arrays over the units."""
        r, m = np.zeros(self.units), np.zeros(self.units)
        dp = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
        _check(load().gmg_iterate_end(self.h, dp(r), dp(m)))
        return r, m

    def solve(self, precision=FP64, rel_tol=1e-8, max_cycles=50, stream=None, check=True):
        """Solve every unit to rel_tol.  Returns rc, cycles, rel_l2, linf, bnorm (the
        worst unit's for several units) and, for several units, 'slots' (also
        'units'): per-unit dicts in unit order r * ntree + i."""
        st = (Stats * self.units)()
        rc = load().gmg_solve(self.h, precision, rel_tol, max_cycles, st, _stream_ptr(stream))
        if check:
            _check(rc)
        units = [dict(cycles=x.cycles, rel_l2=x.rel_l2, linf=x.linf, bnorm=x.bnorm) for x in st]
        if self.units == 1:
            return dict(rc=rc, **units[0])
        return dict(rc=rc, cycles=max(x["cycles"] for x in units), rel_l2=max(x["rel_l2"] for x in units),
                    linf=max(x["linf"] for x in units), bnorm=min(x["bnorm"] for x in units), slots=units,
                    units=units)

    def solve_history(self, precision=FP64, rel_tol=1e-8, max_cycles=50, stream=None, check=True):
        """solve() through gmg_solve_history: the same result, plus 'history',
        an array (steps + 1, units) of relative residuals after every step."""
        st = (Stats * self.units)()
        hist = np.full((max_cycles + 1) * self.units, np.nan)
        rc = load().gmg_solve_history(self.h, precision, rel_tol, max_cycles,
                                      hist.ctypes.data_as(C.POINTER(C.c_double)), st, _stream_ptr(stream))
        if check:
            _check(rc)
        hist = hist.reshape(max_cycles + 1, self.units)
        steps = int(np.isfinite(hist[:, 0]).sum())
        units = [dict(cycles=x.cycles, rel_l2=x.rel_l2, linf=x.linf, bnorm=x.bnorm) for x in st]
        out = dict(rc=rc, history=hist[:steps], units=units)
        out.update(units[0] if self.units == 1 else dict(cycles=max(x["cycles"] for x in units)))
        return out

    def tree_leaves(self, i):
        """(offset, count) of tree i's leaf cells in the leaf arrays."""
        off, n = C.c_longlong(), C.c_longlong()
        _check(load().gmg_forest_tree_info(self.h, int(i), C.byref(off), C.byref(n)))
        return off.value, n.value

    OPTIONS = {"graphs": 1, "coarse_coop": 2, "spin_limit": 3, "fused_sweeps": 4, "cta_threads": 5,
               "coop_max_blocks": 6, "inner_cycles": 7, "slots_per_cta": 8, "fmg_steps": 9, "pdl": 10,
               "cluster_tail": 11, "device_setup": 12, "cluster_parts": 13, "level_legs": 14}

    def set_level_sweeps(self, level, n_down, n_up):
        """N_down / N_up red-black sweeps on one level (a tuning schedule)."""
        _check(load().gmg_set_level_sweeps(self.h, int(level), int(n_down), int(n_up)))

    def level_sweeps(self, level):
        a, b = C.c_int(), C.c_int()
        _check(load().gmg_get_level_sweeps(self.h, int(level), C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_option(self, name, value):
        _check(load().gmg_set_option(self.h, self.OPTIONS[name], int(value)))

    def selftest_barrier_timeout(self, spin_limit=1 << 16, stream=None):
        return load().gmg_selftest_barrier_timeout(self.h, int(spin_limit), _stream_ptr(stream))

    def last_launch_count(self):
        return int(load().gmg_last_launch_count(self.h))

    KERNEL_KINDS = ("smooth", "resid_restrict", "fas_rhs", "coarse_solve", "prolong", "restrict_phi",
                    "resid_norm", "norm_reduce", "accumulate", "rhs_copy", "coarse_cluster", "level_leg_down",
                    "level_leg_up")

    def profile(self, enable=True):
        _check(load().gmg_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """[(kind, precision, level, launches, total_ms)] since the last read."""
        cap = 256
        k, p, lv = (np.zeros(cap, dtype=np.int32) for _ in range(3))
        n = np.zeros(cap, dtype=np.int64)
        ms = np.zeros(cap)
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
        cnt = load().gmg_profile_read(self.h, cap, ip(k), ip(p), ip(lv), n.ctypes.data_as(C.POINTER(C.c_longlong)),
                                      ms.ctypes.data_as(C.POINTER(C.c_double)))
        if cnt < 0:
            _check(cnt)
        names = {0: "fp64", 1: "fp32", 2: "bf16"}
        return [(self.KERNEL_KINDS[k[i]], names[int(p[i])], int(lv[i]), int(n[i]), float(ms[i]))
                for i in range(cnt)]


class Forest(Tree):
    """Independent problems in one block structure (gmg_forest_create): the
    trees are set up (walls, stencils) but not bound; the forest copies what
    it needs.  It then behaves as a Tree whose leaf arrays are tree-major
    (``tree_leaves(i)`` gives tree i's range) and whose residuals and
    statistics are per unit (slot r, tree i) = r * ntree + i."""

    def __init__(self, trees, nrhs=1):
        L = load()
        arr = (C.c_void_p * len(trees))(*[t.h for t in trees])
        h = C.c_void_p()
        _check(L.gmg_forest_create(arr, len(trees), C.byref(h)))
        self._adopt(h, trees[0].dim, trees[0].block_n)
        if nrhs != 1:
            self.set_num_rhs(nrhs)
