"""Thin ctypes binding of libgreem.so (include/greem.h): argument marshalling only.

Every step of the short-range force runs in the library's CUDA kernels; this module
passes torch CUDA tensors as device pointers together with torch's current stream.
It fails loudly when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgreem.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_OOM = -3
ERR_CAPACITY = -4
ERR_TIMEOUT = -5
ERR_NOT_IMPLEMENTED = -6

F32_REL = 0
F64 = 1
FLAG_INDEX_LISTS = 1
FLAG_STAGE_TIMES = 2
FLAG_ADD_PM = 4
FLAG_THETA_EQ12 = 8
FLAG_QUADRUPOLE = 16
ASSIGN_CIC = 0
ASSIGN_TSC = 1

DEBUG_WAIT_POLLS, DEBUG_NODE_CAP, DEBUG_LIST_CAP, DEBUG_STACK_CAP, DEBUG_MAX_ATTEMPTS, DEBUG_START_LEVEL, \
    DEBUG_REPLAY = range(7)

DUMP_KEYS, DUMP_PERM, DUMP_NODES, DUMP_MOMENTS, DUMP_GROUPS, DUMP_LIST_OFFSETS, DUMP_LISTS, DUMP_QUADRUPOLES = range(8)


class GreemError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib().greem_strerror(code).decode() if _lib_loaded() else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("r_cut", ctypes.c_double), ("theta", ctypes.c_double),
                ("eps", ctypes.c_double), ("n_crit", ctypes.c_int), ("n_leaf", ctypes.c_int),
                ("precision", ctypes.c_int), ("list_chunk", ctypes.c_int), ("block_shape", ctypes.c_int),
                ("flags", ctypes.c_uint), ("n_pm", ctypes.c_int), ("assign", ctypes.c_int),
                ("theta0", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_particles", "n_boxes", "n_nodes", "n_groups", "n_list_entries",
                                             "n_interactions", "n_evaluated", "list_capacity",
                                             "kernel_launches")] + \
               [("l_min", ctypes.c_int32), ("retries", ctypes.c_int32)] + \
               [(n, ctypes.c_double) for n in ("ms_keys", "ms_sort", "ms_tree", "ms_groups", "ms_lists",
                                              "ms_force", "ms_total")] + \
               [("n_start_table", ctypes.c_int64), ("n_start_coarse", ctypes.c_int64), ("replayed", ctypes.c_int64)]


_lock = threading.Lock()
_L = None


def _lib_loaded() -> bool:
    return _L is not None


def _lib():
    global _L
    with _lock:
        if _L is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libgreem.so is not built ({LIB_PATH}); run paper_0910_0121_gb300/build.py")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            P = ctypes.POINTER(Params)
            L.greem_params_default.argtypes = [P]
            L.greem_params_default.restype = None
            L.greem_create.argtypes = [ctypes.POINTER(vp), vp]
            L.greem_destroy.argtypes = [vp]
            L.greem_destroy.restype = None
            L.greem_build_tree.argtypes = [vp, vp, vp, i64, P]
            L.greem_short_force.argtypes = [vp, vp, i64, dbl, dbl, dbl, i32, vp]
            L.greem_short_force_ex.argtypes = [vp, vp, vp, i64, P, vp]
            L.greem_short_force_batched.argtypes = [vp, i32, vp, vp, vp, P, vp]
            L.greem_short_force_host.argtypes = [vp, i32, vp, vp, vp, P, vp]
            L.greem_pm_force.argtypes = [vp, vp, vp, i64, dbl, i32, dbl, i32, vp]
            L.greem_graph_capture.argtypes = [vp, vp, vp, i64, P, vp]
            L.greem_graph_launch.argtypes = [vp]
            L.greem_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
            L.greem_debug_dump.argtypes = [vp, i32, vp, i64, ctypes.POINTER(i64)]
            L.greem_autotune.argtypes = [vp, vp, vp, i64, P, vp, i32, vp, P]
            L.greem_debug_dump_group_lists.argtypes = [vp, vp, i64, vp, vp, i64, ctypes.POINTER(i64)]
            L.greem_pair_force_f32.argtypes = [vp, vp, vp, vp, vp, i64, dbl, dbl, vp]
            L.greem_peak_tflops.argtypes = [vp, i32, ctypes.POINTER(dbl)]
            L.greem_kick.argtypes = [vp, vp, vp, i64, dbl]
            L.greem_drift.argtypes = [vp, vp, vp, i64, dbl, dbl]
            L.greem_timestep.argtypes = [vp, vp, vp, i64, dbl, dbl, ctypes.POINTER(dbl)]
            L.greem_softening.argtypes = [dbl, dbl, dbl]
            L.greem_softening.restype = dbl
            L.greem_cosmo_factors.argtypes = [dbl, dbl, dbl, dbl, dbl, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
            L.greem_debug_set.argtypes = [vp, i32, i64]
            L.greem_sample_count.argtypes = [i64, i64, i32, dbl, dbl, dbl, dbl]
            L.greem_sample_count.restype = i64
            L.greem_domain_boxes.argtypes = [vp, i64, i32, i32, i32, vp]
            L.greem_cell_index.argtypes = [vp, vp, i64, dbl, vp, i64, vp]
            L.greem_domain_pack.argtypes = [vp, vp, vp, vp, i64, dbl, vp, i32, vp, vp, vp, vp]
            L.greem_let_export.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, i64, ctypes.POINTER(i64)]
            L.greem_debug_dump_group_entries.argtypes = [vp, vp, i64, vp, vp, vp, i64, ctypes.POINTER(i64)]
            L.greem_strerror.argtypes = [i32]
            L.greem_strerror.restype = ctypes.c_char_p
            for f in ("greem_create", "greem_build_tree", "greem_short_force", "greem_short_force_ex",
                      "greem_short_force_batched", "greem_short_force_host", "greem_pm_force", "greem_graph_capture", "greem_graph_launch",
                      "greem_get_stats", "greem_debug_dump", "greem_autotune", "greem_pair_force_f32",
                      "greem_peak_tflops", "greem_debug_dump_group_lists", "greem_kick", "greem_drift",
                      "greem_timestep", "greem_cosmo_factors", "greem_debug_set",
                      "greem_debug_dump_group_entries", "greem_domain_boxes", "greem_cell_index",
                      "greem_domain_pack", "greem_let_export"):
                getattr(L, f).restype = i32
            _L = L
    return _L


def lib():
    """The loaded C library (raises ImportError when it has not been built)."""
    return _lib()


def _check(rc: int, what: str):
    if rc != OK:
        raise GreemError(rc, what)


def _dev(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a CPU torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def params(L=1.0, r_cut=3.0 / 32, theta=0.5, n_crit=64, n_leaf=10, eps=0.0, precision=F32_REL, list_chunk=0,
           block_shape=0, flags=0, n_pm=0, assign=ASSIGN_TSC, theta0=None) -> Params:
    p = Params()
    _lib().greem_params_default(ctypes.byref(p))
    p.L, p.r_cut, p.theta, p.eps = float(L), float(r_cut), float(theta), float(eps)
    p.n_crit, p.n_leaf, p.precision = int(n_crit), int(n_leaf), int(precision)
    p.list_chunk, p.block_shape, p.flags = int(list_chunk), int(block_shape), int(flags)
    p.n_pm, p.assign = int(n_pm), int(assign)
    if theta0 is not None:
        p.theta0 = float(theta0)
    return p


class Context:
    """greem_ctx bound to a CUDA stream (default: torch's current stream at creation)."""

    def __init__(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(_lib().greem_create(ctypes.byref(h), ctypes.c_void_p(stream.cuda_stream)), "greem_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib().greem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- calls
    def build_tree(self, pos, mass, p: Params):
        import torch
        N = pos.shape[0]
        _check(_lib().greem_build_tree(self._h, _dev(pos, torch.float64, (N, 3), "pos"),
                                       _dev(mass, torch.float32, (N,), "mass"), N, ctypes.byref(p)),
               "greem_build_tree")

    def short_force(self, pos, mass, p: Params, acc=None):
        import torch
        N = pos.shape[0]
        dt = torch.float64 if p.precision == F64 else torch.float32
        if acc is None:
            acc = torch.empty((N, 3), dtype=dt, device=pos.device)
        _check(_lib().greem_short_force_ex(self._h, _dev(pos, torch.float64, (N, 3), "pos"),
                                           _dev(mass, torch.float32, (N,), "mass"), N, ctypes.byref(p),
                                           _dev(acc, dt, (N, 3), "acc")), "greem_short_force_ex")
        return acc

    def short_force_host(self, pos, mass, p: Params, acc=None):
        """greem_short_force_host: independent problems with inputs and results in HOST
        memory (CPU torch tensors; pinned ones let the copies overlap the computation).
        pos, mass: sequences of [N_k,3] float64 and [N_k] float32 tensors; acc: a sequence
        of [N_k,3] tensors (float32, or float64 for F64 precision) or None to allocate
        pinned ones.  Returns the list of acc tensors."""
        import torch
        n = len(pos)
        if len(mass) != n or n < 1:
            raise ValueError("pos and mass must be non-empty sequences of the same length")
        dt = torch.float64 if p.precision == F64 else torch.float32
        if acc is None:
            acc = [torch.empty((x.shape[0], 3), dtype=dt).pin_memory() for x in pos]
        if len(acc) != n:
            raise ValueError("acc must have one tensor per problem")
        vp = ctypes.c_void_p
        ptr_pos, ptr_mass, ptr_acc = (vp * n)(), (vp * n)(), (vp * n)()
        Ns = (ctypes.c_int64 * n)()
        for k in range(n):
            N = pos[k].shape[0]
            ptr_pos[k] = _host(pos[k], torch.float64, (N, 3), "pos").value
            ptr_mass[k] = _host(mass[k], torch.float32, (N,), "mass").value
            ptr_acc[k] = _host(acc[k], dt, (N, 3), "acc").value
            Ns[k] = N
        _check(_lib().greem_short_force_host(self._h, n, ptr_pos, ptr_mass, Ns, ctypes.byref(p), ptr_acc),
               "greem_short_force_host")
        return list(acc)

    def short_force_batched(self, pos, mass, offsets, per_box, acc=None):
        import torch
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        nbox = off.shape[0] - 1
        N = int(off[-1])
        arr = (Params * nbox)(*per_box)
        dt = torch.float64 if per_box[0].precision == F64 else torch.float32
        if acc is None:
            acc = torch.empty((N, 3), dtype=dt, device=pos.device)
        _check(_lib().greem_short_force_batched(self._h, nbox, off.ctypes.data_as(ctypes.c_void_p),
                                                _dev(pos, torch.float64, (N, 3), "pos"),
                                                _dev(mass, torch.float32, (N,), "mass"), arr,
                                                _dev(acc, dt, (N, 3), "acc")), "greem_short_force_batched")
        return acc

    def pm_force(self, pos, mass, L, n_pm, r_cut, assign=ASSIGN_TSC, acc=None):
        """greem_pm_force: the PM (long-range) acceleration, float32 [N,3], input order."""
        import torch
        N = pos.shape[0]
        if acc is None:
            acc = torch.empty((N, 3), dtype=torch.float32, device=pos.device)
        _check(_lib().greem_pm_force(self._h, _dev(pos, torch.float64, (N, 3), "pos"),
                                     _dev(mass, torch.float32, (N,), "mass"), N, float(L), int(n_pm), float(r_cut),
                                     int(assign), _dev(acc, torch.float32, (N, 3), "acc")), "greem_pm_force")
        return acc

    def kick(self, vel, acc, f_kick: float):
        """greem_kick: vel += f_kick * acc (float32 [N,3] device, in place)."""
        import torch
        N = vel.shape[0]
        _check(_lib().greem_kick(self._h, _dev(vel, torch.float32, (N, 3), "vel"), _dev(acc, torch.float32, (N, 3), "acc"),
                                 N, float(f_kick)), "greem_kick")
        return vel

    def drift(self, pos, vel, L: float, f_drift: float):
        """greem_drift: pos += f_drift * vel, wrapped into [0, L) (pos float64, in place)."""
        import torch
        N = pos.shape[0]
        _check(_lib().greem_drift(self._h, _dev(pos, torch.float64, (N, 3), "pos"), _dev(vel, torch.float32, (N, 3), "vel"),
                                  N, float(L), float(f_drift)), "greem_drift")
        return pos

    def timestep(self, vel, acc, eps: float, zeta: float) -> float:
        """greem_timestep: the shared timestep of Eq. 7."""
        import torch
        N = vel.shape[0]
        dt = ctypes.c_double()
        _check(_lib().greem_timestep(self._h, _dev(vel, torch.float32, (N, 3), "vel"),
                                     _dev(acc, torch.float32, (N, 3), "acc"), N, float(eps), float(zeta),
                                     ctypes.byref(dt)), "greem_timestep")
        return dt.value

    def graph_capture(self, pos, mass, p: Params, acc):
        import torch
        N = pos.shape[0]
        dt = torch.float64 if p.precision == F64 else torch.float32
        _check(_lib().greem_graph_capture(self._h, _dev(pos, torch.float64, (N, 3), "pos"),
                                          _dev(mass, torch.float32, (N,), "mass"), N, ctypes.byref(p),
                                          _dev(acc, dt, (N, 3), "acc")), "greem_graph_capture")

    def graph_launch(self) -> int:
        return _lib().greem_graph_launch(self._h)

    def autotune(self, pos, mass, p: Params, acc, candidates=None) -> Params:
        import torch
        N = pos.shape[0]
        best = Params()
        cand = None if candidates is None else (ctypes.c_int * len(candidates))(*candidates)
        dt = torch.float64 if p.precision == F64 else torch.float32
        _check(_lib().greem_autotune(self._h, _dev(pos, torch.float64, (N, 3), "pos"),
                                     _dev(mass, torch.float32, (N,), "mass"), N, ctypes.byref(p),
                                     cand, 0 if cand is None else len(candidates), _dev(acc, dt, (N, 3), "acc"),
                                     ctypes.byref(best)), "greem_autotune")
        return best

    def pair_force_f32(self, xg, xi, xj, mj, r_cut, eps=0.0, acc=None):
        import torch
        P = xg.shape[0]
        if acc is None:
            acc = torch.empty((P, 3), dtype=torch.float32, device=xg.device)
        _check(_lib().greem_pair_force_f32(self._h, _dev(xg, torch.float64, (P, 3), "x_g"),
                                           _dev(xi, torch.float64, (P, 3), "x_i"),
                                           _dev(xj, torch.float64, (P, 3), "x_j"),
                                           _dev(mj, torch.float32, (P,), "m_j"), P, float(r_cut), float(eps),
                                           _dev(acc, torch.float32, (P, 3), "acc")), "greem_pair_force_f32")
        return acc

    def peak_tflops(self, which: int = 0) -> float:
        v = ctypes.c_double()
        _check(_lib().greem_peak_tflops(self._h, int(which), ctypes.byref(v)), "greem_peak_tflops")
        return v.value

    def cell_index(self, pos, L: float, idx=None):
        """greem_cell_index: finest cells (int32 [n,3], device) of pos[idx] (or of all of pos)."""
        import torch
        N = pos.shape[0]
        n = N if idx is None else idx.shape[0]
        cells = torch.empty((n, 3), dtype=torch.int32, device=pos.device)
        if n == 0:
            return cells
        _check(_lib().greem_cell_index(self._h, _dev(pos, torch.float64, (N, 3), "pos"), N, float(L),
                                       None if idx is None else _dev(idx, torch.int64, (n,), "idx"), n,
                                       _dev(cells, torch.int32, (n, 3), "cells")), "greem_cell_index")
        return cells

    def domain_pack(self, pos, mass, ids, L: float, boxes):
        """greem_domain_pack: (pos, mass, ids, counts) packed by destination domain."""
        import torch
        N = pos.shape[0]
        b = np.ascontiguousarray(boxes, dtype=np.int32)
        counts = np.zeros(b.shape[0], np.int64)
        po = torch.empty((N, 3), dtype=torch.float64, device=pos.device)
        mo = torch.empty((N,), dtype=torch.float32, device=pos.device)
        io = torch.empty((N,), dtype=torch.int64, device=pos.device)
        if N:
            _check(_lib().greem_domain_pack(self._h, _dev(pos, torch.float64, (N, 3), "pos"),
                                            _dev(mass, torch.float32, (N,), "mass"),
                                            None if ids is None else _dev(ids, torch.int64, (N,), "ids"), N,
                                            float(L), b.ctypes.data_as(ctypes.c_void_p), b.shape[0],
                                            counts.ctypes.data_as(ctypes.c_void_p), _dev(po, torch.float64),
                                            _dev(mo, torch.float32), _dev(io, torch.int64)), "greem_domain_pack")
        return po, mo, io, counts

    def let_export(self, boxes, self_index: int, with_refs: bool = False):
        """greem_let_export on the last tree: (pos [n,3] f64, mass [n] f32, refs [n] i64 or
        None, counts [ndom]) of the items for every other domain, packed by domain."""
        import torch
        b = np.ascontiguousarray(boxes, dtype=np.int32)
        counts = np.zeros(b.shape[0], np.int64)
        tot = ctypes.c_int64()
        vp = ctypes.c_void_p
        dev = torch.device("cuda", torch.cuda.current_device())
        cap = getattr(self, "_let_cap", 0)
        while True:
            po = torch.empty((max(cap, 1), 3), dtype=torch.float64, device=dev)
            mo = torch.empty((max(cap, 1),), dtype=torch.float32, device=dev)
            ro = torch.empty((max(cap, 1),), dtype=torch.int64, device=dev) if with_refs else None
            rc = _lib().greem_let_export(self._h, b.ctypes.data_as(vp), b.shape[0], int(self_index),
                                         counts.ctypes.data_as(vp), vp(po.data_ptr()), vp(mo.data_ptr()),
                                         None if ro is None else vp(ro.data_ptr()), cap, ctypes.byref(tot))
            if rc == ERR_CAPACITY and tot.value > cap:
                cap = int(tot.value * 1.25) + 1024
                self._let_cap = cap
                continue
            _check(rc, "greem_let_export")
            n = tot.value
            return po[:n], mo[:n], (None if ro is None else ro[:n]), counts

    def debug_set(self, what: int, value: int):
        """greem_debug_set: failure-path controls (DEBUG_* constants)."""
        _check(_lib().greem_debug_set(self._h, int(what), int(value)), "greem_debug_set")

    def stats(self) -> dict:
        s = Stats()
        _check(_lib().greem_get_stats(self._h, ctypes.byref(s)), "greem_get_stats")
        return {n: getattr(s, n) for n, _ in Stats._fields_}

    def dump_group_lists(self, groups):
        """(offsets [n+1], entries [E,5]) of the selected groups' lists, each in preorder."""
        g = np.ascontiguousarray(groups, dtype=np.int64)
        off = np.zeros(g.shape[0] + 1, np.int64)
        n = ctypes.c_int64()
        vp = ctypes.c_void_p
        rc = _lib().greem_debug_dump_group_lists(self._h, g.ctypes.data_as(vp), g.shape[0], off.ctypes.data_as(vp),
                                                None, 0, ctypes.byref(n))
        if rc != OK and n.value == 0:
            raise GreemError(rc, "greem_debug_dump_group_lists")
        ent = np.zeros((max(n.value, 1), 5), np.int64)
        _check(_lib().greem_debug_dump_group_lists(self._h, g.ctypes.data_as(vp), g.shape[0], off.ctypes.data_as(vp),
                                                   ent.ctypes.data_as(vp), n.value, ctypes.byref(n)),
               "greem_debug_dump_group_lists")
        return off, ent[: n.value]

    def dump_group_entries(self, groups, index: bool = False):
        """(offsets [n+1], FP32 entries [E,4], index entries [E,5] or None) of the selected
        groups' lists in the builder's own order (greem_debug_dump_group_entries)."""
        g = np.ascontiguousarray(groups, dtype=np.int64)
        off = np.zeros(g.shape[0] + 1, np.int64)
        n = ctypes.c_int64()
        vp = ctypes.c_void_p
        rc = _lib().greem_debug_dump_group_entries(self._h, g.ctypes.data_as(vp), g.shape[0], off.ctypes.data_as(vp),
                                                  None, None, 0, ctypes.byref(n))
        if rc != OK and n.value == 0:
            raise GreemError(rc, "greem_debug_dump_group_entries")
        ent = np.zeros((max(n.value, 1), 4), np.float32)
        idx = np.zeros((max(n.value, 1), 5), np.int64) if index else None
        _check(_lib().greem_debug_dump_group_entries(self._h, g.ctypes.data_as(vp), g.shape[0],
                                                     off.ctypes.data_as(vp), ent.ctypes.data_as(vp),
                                                     None if idx is None else idx.ctypes.data_as(vp), n.value,
                                                     ctypes.byref(n)), "greem_debug_dump_group_entries")
        return off, ent[: n.value], (None if idx is None else idx[: n.value])

    def dump(self, what: int) -> np.ndarray:
        n = ctypes.c_int64()
        rc = _lib().greem_debug_dump(self._h, int(what), None, 0, ctypes.byref(n))
        if n.value == 0 and rc != OK:
            raise GreemError(rc, "greem_debug_dump")
        buf = np.zeros(max(n.value, 8) // 8 + 1, dtype=np.int64)
        _check(_lib().greem_debug_dump(self._h, int(what), buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes,
                                       ctypes.byref(n)), "greem_debug_dump")
        raw = buf.view(np.uint8)[: n.value]
        if what == DUMP_KEYS:
            return raw.view(np.uint64).copy()
        if what == DUMP_PERM:
            return raw.view(np.uint32).copy()
        if what == DUMP_NODES:
            return raw.view(np.int64).reshape(-1, 9).copy()
        if what == DUMP_MOMENTS:
            return raw.view(np.float64).reshape(-1, 4).copy()
        if what in (DUMP_GROUPS, DUMP_LIST_OFFSETS):
            return raw.view(np.int64).copy()
        if what == DUMP_LISTS:
            return raw.view(np.int64).reshape(-1, 5).copy()
        if what == DUMP_QUADRUPOLES:
            return raw.view(np.float64).reshape(-1, 6).copy()
        raise ValueError(what)


def short_force(pos, mass, L: float, r_cut: float, theta: float, n_crit: int, acc=None):
    """greem_short_force: the whole force with defaults, library-owned context on the
    current device (legacy default stream).  pos float64 [N,3], mass float32 [N] CUDA."""
    import torch
    N = pos.shape[0]
    if acc is None:
        acc = torch.empty((N, 3), dtype=torch.float32, device=pos.device)
    torch.cuda.current_stream().synchronize()
    _check(_lib().greem_short_force(_dev(pos, torch.float64, (N, 3), "pos"), _dev(mass, torch.float32, (N,), "mass"),
                                    N, float(L), float(r_cut), float(theta), int(n_crit),
                                    _dev(acc, torch.float32, (N, 3), "acc")), "greem_short_force")
    return acc


def sample_count(n_total: int, n_local: int, nproc: int, rate: float, t_local: float, t_sum: float,
                 alpha: float) -> int:
    """greem_sample_count: particles to sample for the decomposition (Eq. 3-5)."""
    n = _lib().greem_sample_count(int(n_total), int(n_local), int(nproc), float(rate), float(t_local), float(t_sum),
                                  float(alpha))
    if n < 0:
        raise GreemError(ERR_INVALID_ARG, "greem_sample_count")
    return int(n)


def domain_boxes(cells, grid) -> np.ndarray:
    """greem_domain_boxes: recursive multisection of the sampled cells (int [n,3]) into
    px*py*pz boxes (int32 [p,6])."""
    c = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 3)
    px, py, pz = (int(g) for g in grid)
    out = np.zeros((px * py * pz, 6), np.int32)
    _check(_lib().greem_domain_boxes(c.ctypes.data_as(ctypes.c_void_p), c.shape[0], px, py, pz,
                                     out.ctypes.data_as(ctypes.c_void_p)), "greem_domain_boxes")
    return out


def softening(eps_fin: float, z_crit: float, z: float) -> float:
    """greem_softening: the physical softening of Eq. 6 at redshift z."""
    return _lib().greem_softening(float(eps_fin), float(z_crit), float(z))


def cosmo_factors(a0: float, a1: float, omega_m: float, omega_l: float, h0: float):
    """greem_cosmo_factors: (int dt/a, int dt/a^2) from scale factor a0 to a1."""
    k, d = ctypes.c_double(), ctypes.c_double()
    _check(_lib().greem_cosmo_factors(float(a0), float(a1), float(omega_m), float(omega_l), float(h0), ctypes.byref(k),
                                      ctypes.byref(d)), "greem_cosmo_factors")
    return k.value, d.value
