"""Plain FP64 CPU oracle for the GreeM periodic short-range tree force.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` import this package.  The product
path (``paper_0910_0121_gb300``) never imports it, and the two share no code:
the C source here is an independent restatement of the paper (Eq. 1, Eq. 2,
Sec. 2.2 steps 2-5, Sec. 3.1.2), see ``greem_oracle.c`` for every reading.

This module only marshals numpy arrays into the C library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "greem_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP for timing runs)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.or_g_p3m.restype = _dbl
            L.or_g_p3m.argtypes = [_dbl]
            L.or_pair_accel.restype = None
            L.or_pair_accel.argtypes = [_vp, _dbl, _dbl, _dbl, _vp]
            for f in ("or_g_p3m_d1", "or_g_p3m_d2"):
                getattr(L, f).restype = _dbl
                getattr(L, f).argtypes = [_dbl]
            L.or_quad_accel.restype = None
            L.or_quad_accel.argtypes = [_vp, _vp, _dbl, _vp]
            L.or_list_force_quad.restype = ctypes.c_int
            L.or_list_force_quad.argtypes = [_vp, _vp, ctypes.c_int]
            L.or_wrap.restype = _dbl
            L.or_wrap.argtypes = [_dbl, _dbl]
            L.or_cell_index.restype = _i64
            L.or_cell_index.argtypes = [_dbl, _dbl]
            L.or_morton.restype = ctypes.c_uint64
            L.or_morton.argtypes = [_i64, _i64, _i64]
            L.or_lmin.restype = ctypes.c_int
            L.or_lmin.argtypes = [_dbl, _dbl]
            L.or_direct.restype = ctypes.c_int
            L.or_direct.argtypes = [_vp, _vp, _i64, _dbl, _dbl, _dbl, _vp, ctypes.c_int]
            L.or_direct_at.restype = ctypes.c_int
            L.or_direct_at.argtypes = [_vp, _vp, _i64, _dbl, _dbl, _dbl, _vp, _i64, _vp, ctypes.c_int]
            L.or_tree_build.restype = _vp
            L.or_tree_build.argtypes = [_vp, _vp, _i64, _dbl, _dbl, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int)]
            L.or_tree_free.restype = None
            L.or_tree_free.argtypes = [_vp]
            for f in ("or_tree_n_nodes", "or_tree_n_groups", "or_lists_n_entries"):
                getattr(L, f).restype = _i64
                getattr(L, f).argtypes = [_vp]
            L.or_tree_lmin.restype = ctypes.c_int
            L.or_tree_lmin.argtypes = [_vp]
            L.or_tree_get_sorted.restype = None
            L.or_tree_get_sorted.argtypes = [_vp, _vp, _vp, _vp, _vp]
            for f in ("or_tree_get_nodes", "or_tree_get_moments", "or_tree_get_groups", "or_tree_get_quadrupoles"):
                getattr(L, f).restype = None
                getattr(L, f).argtypes = [_vp, _vp]
            L.or_lists_build.restype = ctypes.c_int
            L.or_lists_build.argtypes = [_vp, _dbl, _vp, _i64]
            L.or_lists_build_eq12.restype = ctypes.c_int
            L.or_lists_build_eq12.argtypes = [_vp, _dbl, _dbl, _vp, _i64]
            L.or_lists_get.restype = None
            L.or_lists_get.argtypes = [_vp, _vp, _vp, _vp, _vp]
            L.or_list_force.restype = ctypes.c_int
            L.or_list_force.argtypes = [_vp, _dbl, _vp, ctypes.c_int]
            L.or_short_force.restype = ctypes.c_int
            L.or_short_force.argtypes = [_vp, _vp, _i64, _dbl, _dbl, _dbl, ctypes.c_int, ctypes.c_int,
                                         _dbl, _vp, ctypes.c_int]
            L.or_let_export.restype = _i64
            L.or_let_export.argtypes = [_vp, _vp, _dbl, _vp, _vp, _i64]
            L.or_max_threads.restype = ctypes.c_int
            L.or_max_threads.argtypes = []
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pos(pos) -> np.ndarray:
    p = np.ascontiguousarray(pos, dtype=np.float64)
    assert p.ndim == 2 and p.shape[1] == 3
    return p


def _mass(mass) -> np.ndarray:
    return np.ascontiguousarray(mass, dtype=np.float32)


# --------------------------------------------------------------------------- scalars
def g_p3m(R: float) -> float:
    """Eq. 2 cutoff function."""
    return lib().or_g_p3m(float(R))


def g_p3m_d1(R: float) -> float:
    """dg/dR of Eq. 2."""
    return lib().or_g_p3m_d1(float(R))


def g_p3m_d2(R: float) -> float:
    """d^2g/dR^2 of Eq. 2."""
    return lib().or_g_p3m_d2(float(R))


def quad_accel(d, q, eta: float) -> np.ndarray:
    """Second-order (quadrupole) part of the acceleration from a mass distribution with
    second moments q = (xx, yy, zz, xy, xz, yz) about its COM at d = COM - x (Sec. 4.1)."""
    dd = np.ascontiguousarray(d, dtype=np.float64)
    qq = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(3)
    lib().or_quad_accel(_ptr(dd), _ptr(qq), float(eta), _ptr(out))
    return out


def pair_accel(d, m: float, eta: float, eps: float = 0.0) -> np.ndarray:
    """Eq. 1 acceleration from a particle at separation d = x_j - x_i."""
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(3)
    lib().or_pair_accel(_ptr(dd), float(m), float(eta), float(eps), _ptr(out))
    return out


def wrap(x: float, L: float) -> float:
    return lib().or_wrap(float(x), float(L))


def cell_index(r: float, L: float) -> int:
    return lib().or_cell_index(float(r), float(L))


def morton(ix: int, iy: int, iz: int) -> int:
    return lib().or_morton(int(ix), int(iy), int(iz))


def lmin(L: float, r_cut: float) -> int:
    return lib().or_lmin(float(L), float(r_cut))


def max_threads() -> int:
    return lib().or_max_threads()


# --------------------------------------------------------------------------- direct sum
def direct(pos, mass, L: float, r_cut: float, eps: float = 0.0, nthreads: int = 0) -> np.ndarray:
    """Brute-force minimum-image sum of Eq. 1 over all pairs, input order, FP64."""
    p, m = _pos(pos), _mass(mass)
    acc = np.zeros((p.shape[0], 3))
    rc = lib().or_direct(_ptr(p), _ptr(m), p.shape[0], float(L), float(r_cut), float(eps), _ptr(acc),
                         int(nthreads))
    if rc:
        raise ValueError(f"oracle direct sum rejected arguments ({rc})")
    return acc


def direct_at(pos, mass, L: float, r_cut: float, idx, eps: float = 0.0, nthreads: int = 0) -> np.ndarray:
    """The brute-force sum of ``direct`` for the particles idx only ([len(idx), 3])."""
    p, m = _pos(pos), _mass(mass)
    ii = np.ascontiguousarray(idx, dtype=np.int64)
    acc = np.zeros((ii.shape[0], 3))
    rc = lib().or_direct_at(_ptr(p), _ptr(m), p.shape[0], float(L), float(r_cut), float(eps), _ptr(ii),
                            ii.shape[0], _ptr(acc), int(nthreads))
    if rc:
        raise ValueError(f"oracle direct sum rejected arguments ({rc})")
    return acc


# --------------------------------------------------------------------------- tree
class Tree:
    """Oracle tree: keys, sort, octree, moments, groups; lists and list force on demand."""

    def __init__(self, pos, mass, L: float, r_cut: float, n_crit: int, n_leaf: int = 10):
        p, m = _pos(pos), _mass(mass)
        self.N = p.shape[0]
        self.L, self.r_cut, self.n_crit, self.n_leaf = float(L), float(r_cut), int(n_crit), int(n_leaf)
        err = ctypes.c_int(0)
        h = lib().or_tree_build(_ptr(p), _ptr(m), self.N, self.L, self.r_cut, self.n_leaf, self.n_crit,
                                ctypes.byref(err))
        if not h:
            raise ValueError(f"oracle tree build rejected arguments ({err.value})")
        self._h = h
        self.theta = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_tree_free(h)
            self._h = None

    @property
    def n_nodes(self) -> int:
        return lib().or_tree_n_nodes(self._h)

    @property
    def n_groups(self) -> int:
        return lib().or_tree_n_groups(self._h)

    @property
    def lmin(self) -> int:
        return lib().or_tree_lmin(self._h)

    def sorted(self):
        """(keys u64, perm i64, wrapped sorted positions [N,3], sorted masses)."""
        key = np.zeros(self.N, np.uint64)
        perm = np.zeros(self.N, np.int64)
        xyz = np.zeros((self.N, 3))
        m = np.zeros(self.N, np.float32)
        lib().or_tree_get_sorted(self._h, _ptr(key), _ptr(perm), _ptr(xyz), _ptr(m))
        return key, perm, xyz, m

    def nodes(self) -> np.ndarray:
        """[n_nodes, 9] int64: level, ix, iy, iz, begin, end, skip, leaf, 0 (preorder)."""
        out = np.zeros((self.n_nodes, 9), np.int64)
        lib().or_tree_get_nodes(self._h, _ptr(out))
        return out

    def moments(self) -> np.ndarray:
        """[n_nodes, 4] float64: M, cx, cy, cz."""
        out = np.zeros((self.n_nodes, 4))
        lib().or_tree_get_moments(self._h, _ptr(out))
        return out

    def quadrupoles(self) -> np.ndarray:
        """[n_nodes, 6] float64: second moments xx, yy, zz, xy, xz, yz about the COM."""
        out = np.zeros((self.n_nodes, 6))
        lib().or_tree_get_quadrupoles(self._h, _ptr(out))
        return out

    def groups(self) -> np.ndarray:
        out = np.zeros(self.n_groups, np.int64)
        lib().or_tree_get_groups(self._h, _ptr(out))
        return out

    def build_lists(self, theta: float, groups=None, theta0=None):
        """Lists with the constant opening angle theta, or, when theta0 is given, with the
        distance-dependent angle of Eq. 12 (Sec. 4.1) capped at theta_max = theta."""
        sel = None if groups is None else np.ascontiguousarray(groups, dtype=np.int64)
        if theta0 is None:
            rc = lib().or_lists_build(self._h, float(theta), None if sel is None else _ptr(sel),
                                      0 if sel is None else sel.shape[0])
        else:
            rc = lib().or_lists_build_eq12(self._h, float(theta0), float(theta), None if sel is None else _ptr(sel),
                                           0 if sel is None else sel.shape[0])
        if rc:
            raise ValueError(f"oracle list build failed ({rc})")
        self.theta = float(theta)
        self._nsel = self.n_groups if sel is None else sel.shape[0]

    def lists(self):
        """(offsets [G+1], kind [E] int8, idx [E] int64, shift [E,3] int8)."""
        ne = lib().or_lists_n_entries(self._h)
        off = np.zeros(self._nsel + 1, np.int64)
        kind = np.zeros(ne, np.int8)
        idx = np.zeros(ne, np.int64)
        sh = np.zeros((ne, 3), np.int8)
        lib().or_lists_get(self._h, _ptr(off), _ptr(kind), _ptr(idx), _ptr(sh))
        return off, kind, idx, sh

    def let_export(self, box, theta: float):
        """Local essential tree for the domain box (int [6]: xlo, xhi, ylo, yhi, zlo, zhi in
        finest cells, half-open) at opening angle theta (Sec. 2.2 step 3): (kind [n] 1 node /
        0 particle, index [n] node or sorted particle), in preorder."""
        b = np.ascontiguousarray(box, dtype=np.int32)
        n = lib().or_let_export(self._h, _ptr(b), float(theta), None, None, 0)
        if n < 0:
            raise ValueError("oracle LET rejected arguments")
        kind = np.zeros(max(n, 1), np.int64)
        idx = np.zeros(max(n, 1), np.int64)
        lib().or_let_export(self._h, _ptr(b), float(theta), _ptr(kind), _ptr(idx), n)
        return kind[:n], idx[:n]

    def list_force(self, eps: float = 0.0, nthreads: int = 0, quad: bool = False) -> np.ndarray:
        """FP64 list force in SORTED order ([N,3]; particles of groups without lists are 0);
        quad adds the second-order terms of node entries (Sec. 4.1; eps must be 0)."""
        acc = np.zeros((self.N, 3))
        if quad:
            if eps != 0.0:
                raise ValueError("the quadrupole terms are for eps = 0")
            lib().or_list_force_quad(self._h, _ptr(acc), int(nthreads))
        else:
            lib().or_list_force(self._h, float(eps), _ptr(acc), int(nthreads))
        return acc

    def list_force_input_order(self, eps: float = 0.0, nthreads: int = 0, quad: bool = False) -> np.ndarray:
        a = self.list_force(eps, nthreads, quad)
        _, perm, _, _ = self.sorted()
        out = np.zeros_like(a)
        out[perm] = a
        return out


def short_force(pos, mass, L: float, r_cut: float, theta: float, n_crit: int, n_leaf: int = 10,
                eps: float = 0.0, nthreads: int = 0) -> np.ndarray:
    """Whole oracle pipeline; FP64 acceleration in input order."""
    p, m = _pos(pos), _mass(mass)
    acc = np.zeros((p.shape[0], 3))
    rc = lib().or_short_force(_ptr(p), _ptr(m), p.shape[0], float(L), float(r_cut), float(theta),
                              int(n_crit), int(n_leaf), float(eps), _ptr(acc), int(nthreads))
    if rc:
        raise ValueError(f"oracle short force failed ({rc})")
    return acc
