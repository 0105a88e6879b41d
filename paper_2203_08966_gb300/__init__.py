"""GB300 Barnes-Hut timestep (arXiv 2203.08966, Algorithm 2 with kick-drift-kick leapfrog).

A thin ctypes binding over the C ABI in ``include/nbody.h`` (``libnbody.so`` next to this file,
built by ``build_lib.build()``).  This module only marshals arguments: every step of the method
(box, Morton keys, radix sort, node split, moments, walk, leapfrog) runs in the library's CUDA
kernels.  There is no CPU fallback: importing works without the library, but creating a
``Context`` raises when ``libnbody.so`` is missing or no GPU is present.

Tensors are torch float64 CUDA tensors in the library's structure-of-arrays layout:
``pos`` and ``vel`` of shape (3, N) (rows x, y, z), ``mass`` of shape (N,), ``acc`` (3, N).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnbody.so")

FP64, FP32, FP32_KAHAN, FP64_FAST = 0, 1, 2, 3
WALK_SHAPES = 8  # NBODY_WALK_SHAPES
FLAG_GROUP_MAC = 1  # NBODY_FLAG_GROUP_MAC: grouped acceptance test (Barnes 1990), FP32 forms
FLAG_CELL_GROUPS = 2  # NBODY_FLAG_CELL_GROUPS: FP32 walk groups follow the tree's cells
FLAG_QUADRUPOLE = 4  # NBODY_FLAG_QUADRUPOLE: accepted cells add their quadrupole term
FLAG_CHECK_FINITE = 8  # NBODY_FLAG_CHECK_FINITE: reject NaN / infinite positions and masses
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp32_kahan": FP32_KAHAN, "fp64_fast": FP64_FAST}
# NBODY_SORT_*: how a build sorts (same order in every mode; re-sort from the previous order, §4.4)
SORT_AUTO, SORT_FULL, SORT_RESORT = 0, 1, 2

STATUS = {0: "NBODY_OK", 1: "NBODY_EINVAL", 2: "NBODY_ENOMEM", 3: "NBODY_ECUDA",
          4: "NBODY_ESTACK", 5: "NBODY_ETIMEOUT", 6: "NBODY_ESTATE"}

# Every entry point declared in include/nbody.h.
EXPORTS = ("nbody_create", "nbody_destroy", "nbody_set_params", "nbody_build_tree",
           "nbody_forces", "nbody_step", "nbody_step_host", "nbody_direct_forces", "nbody_sync",
           "nbody_get_keys", "nbody_get_box", "nbody_get_tree", "nbody_get_moments",
           "nbody_get_counters", "nbody_enable_timing", "nbody_get_timings",
           "nbody_last_error", "nbody_get_launch_count", "nbody_sort_keys_noalloc",
           "nbody_forest_create", "nbody_forest_forces", "nbody_forest_step",
           "nbody_autotune", "nbody_set_walk_shape", "nbody_get_walk_shape",
           "nbody_set_walk_limits",
           "nbody_set_sort_mode", "nbody_get_sort_stats", "nbody_measure_fp32_rate",
           "nbody_measure_fp64_rate")


class NBodyError(RuntimeError):
    def __init__(self, status, what, msg=""):
        self.status = status
        super().__init__(f"{what} -> {STATUS.get(status, status)}{': ' + msg if msg else ''}")


class Params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("eps", ctypes.c_double), ("theta", ctypes.c_double),
                ("dt", ctypes.c_double), ("precision", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class TreeRecord(ctypes.Structure):
    _fields_ = [("key", ctypes.c_uint64), ("level", ctypes.c_int32),
                ("child_mask", ctypes.c_int32), ("first", ctypes.c_int64),
                ("count", ctypes.c_int64)]


_RECORD_DTYPE = np.dtype([("key", np.uint64), ("level", np.int32), ("child_mask", np.int32),
                          ("first", np.int64), ("count", np.int64)])

_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libnbody.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with paper_2203_08966_gb300.build_lib.build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    P = ctypes.POINTER(Params)
    sig = {
        "nbody_create": [ctypes.POINTER(vp), i64, P, vp],
        "nbody_destroy": [vp],
        "nbody_set_params": [vp, P],
        "nbody_build_tree": [vp, vp, vp, i64],
        "nbody_forces": [vp, vp, vp, i64, vp],
        "nbody_step": [vp, vp, vp, vp, i64, i32],
        "nbody_step_host": [vp, vp, vp, vp, vp, i64, i32],
        "nbody_direct_forces": [vp, vp, vp, i64, vp, i64, vp],
        "nbody_sync": [vp],
        "nbody_get_keys": [vp, vp, vp],
        "nbody_get_box": [vp, vp],
        "nbody_get_tree": [vp, ctypes.POINTER(i64), vp, i64],
        "nbody_get_moments": [vp, vp, i64],
        "nbody_get_counters": [vp, vp, vp],
        "nbody_enable_timing": [vp, i32],
        "nbody_get_timings": [vp, vp],
        "nbody_last_error": [vp, ctypes.c_char_p, i64],
        "nbody_get_launch_count": [ctypes.POINTER(i64)],
        "nbody_sort_keys_noalloc": [vp, vp, i64, vp, vp, vp],
        "nbody_forest_create": [ctypes.POINTER(vp), i32, vp, P, vp],
        "nbody_forest_forces": [vp, vp, vp, vp],
        "nbody_forest_step": [vp, vp, vp, vp, i32, i32],
        "nbody_autotune": [vp, vp, vp, i64, vp, vp],
        "nbody_get_walk_shape": [vp, vp, vp],
        "nbody_set_walk_shape": [vp, i32],
        "nbody_set_walk_limits": [vp, i32, i64, i32],
        "nbody_set_sort_mode": [vp, i32],
        "nbody_get_sort_stats": [vp, vp, vp],
        "nbody_measure_fp32_rate": [vp, vp],
        "nbody_measure_fp64_rate": [vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    _lib = lib
    return lib


def _dptr(t, dtype, shape=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor of the given dtype (and shape)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, dtype, shape, name):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous numpy {np.dtype(dtype).name} array")
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}")
    return a.ctypes.data_as(ctypes.c_void_p)


class Context:
    """One nbody_ctx: a system of up to ``capacity`` bodies on the current CUDA device.

    All work goes to the CUDA stream that is current when the context is created (or
    ``stream``, a torch.cuda.Stream)."""

    def __init__(self, capacity, G=1.0, eps=0.0, theta=0.5, dt=1e-3, precision=FP32,
                 stream=None, offsets=None, flags=0):
        import torch
        self._lib = load_library()
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.params = Params(G, eps, theta, dt, precision, int(flags))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        sp = ctypes.c_void_p(stream.cuda_stream)
        if offsets is None:
            st = self._lib.nbody_create(ctypes.byref(h), int(capacity), ctypes.byref(self.params),
                                        sp)
            what = "nbody_create"
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            st = self._lib.nbody_forest_create(ctypes.byref(h), int(off.shape[0]) - 1,
                                               off.ctypes.data_as(ctypes.c_void_p),
                                               ctypes.byref(self.params), sp)
            what = "nbody_forest_create"
            capacity = int(off[-1])
            self.offsets = off
        if st != 0:
            raise NBodyError(st, what)
        self._h = h
        self.capacity = int(capacity)

    @classmethod
    def forest(cls, offsets, G=1.0, eps=0.0, theta=0.5, dt=1e-3, precision=FP32, stream=None,
               flags=0):
        """A context for independent systems packed into one set of arrays: system k owns
        bodies offsets[k] .. offsets[k+1] - 1 (nbody_forest_create)."""
        return cls(0, G, eps, theta, dt, precision, stream, offsets=offsets, flags=flags)

    # ---------------------------------------------------------------- plumbing
    def _check(self, st, what):
        if st != 0:
            buf = ctypes.create_string_buffer(256)
            self._lib.nbody_last_error(self._h, buf, 256)
            raise NBodyError(st, what, buf.value.decode(errors="replace"))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nbody_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, G=None, eps=None, theta=None, dt=None, precision=None, flags=None):
        p = self.params
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        new = Params(p.G if G is None else G, p.eps if eps is None else eps,
                     p.theta if theta is None else theta, p.dt if dt is None else dt,
                     p.precision if precision is None else precision,
                     p.flags if flags is None else int(flags))
        self._check(self._lib.nbody_set_params(self._h, ctypes.byref(new)), "nbody_set_params")
        self.params = new

    # ---------------------------------------------------------------- compute
    def build_tree(self, pos, mass):
        import torch
        n = int(mass.shape[0])
        self._check(self._lib.nbody_build_tree(self._h, _dptr(pos, torch.float64, (3, n), "pos"),
                                               _dptr(mass, torch.float64, (n,), "mass"), n),
                    "nbody_build_tree")

    def forces(self, pos, mass, acc=None):
        import torch
        n = int(mass.shape[0])
        if acc is None:
            acc = torch.empty((3, n), dtype=torch.float64, device=pos.device)
        self._check(self._lib.nbody_forces(self._h, _dptr(pos, torch.float64, (3, n), "pos"),
                                           _dptr(mass, torch.float64, (n,), "mass"), n,
                                           _dptr(acc, torch.float64, (3, n), "acc")),
                    "nbody_forces")
        return acc

    def step(self, pos, vel, mass, nsteps=1):
        import torch
        n = int(mass.shape[0])
        self._check(self._lib.nbody_step(self._h, _dptr(pos, torch.float64, (3, n), "pos"),
                                         _dptr(vel, torch.float64, (3, n), "vel"),
                                         _dptr(mass, torch.float64, (n,), "mass"), n,
                                         int(nsteps)), "nbody_step")

    def step_host(self, pos, vel, mass, nsteps=1, acc=None):
        """Host-buffer step on numpy float64 arrays (ideally page-locked), updated in place.

        ``acc`` (3, N), optional, in/out: the acceleration at ``pos`` from the previous call."""
        n = int(mass.shape[0])
        ap = None if acc is None else _hptr(acc, np.float64, (3, n), "acc")
        self._check(self._lib.nbody_step_host(self._h, _hptr(pos, np.float64, (3, n), "pos"),
                                              _hptr(vel, np.float64, (3, n), "vel"), ap,
                                              _hptr(mass, np.float64, (n,), "mass"), n,
                                              int(nsteps)), "nbody_step_host")

    def direct_forces(self, pos, mass, targets=None, acc=None):
        import torch
        n = int(mass.shape[0])
        nt = n if targets is None else int(targets.shape[0])
        if acc is None:
            acc = torch.empty((3, nt), dtype=torch.float64, device=pos.device)
        tp = None if targets is None else _dptr(targets, torch.int64, (nt,), "targets")
        self._check(self._lib.nbody_direct_forces(self._h,
                                                  _dptr(pos, torch.float64, (3, n), "pos"),
                                                  _dptr(mass, torch.float64, (n,), "mass"), n,
                                                  tp, nt,
                                                  _dptr(acc, torch.float64, (3, nt), "acc")),
                    "nbody_direct_forces")
        return acc

    def forest_forces(self, pos, mass, acc=None):
        import torch
        n = self.capacity
        if acc is None:
            acc = torch.empty((3, n), dtype=torch.float64, device=pos.device)
        self._check(self._lib.nbody_forest_forces(self._h,
                                                  _dptr(pos, torch.float64, (3, n), "pos"),
                                                  _dptr(mass, torch.float64, (n,), "mass"),
                                                  _dptr(acc, torch.float64, (3, n), "acc")),
                    "nbody_forest_forces")
        return acc

    def forest_step(self, pos, vel, mass, nsteps=1, use_graph=False):
        import torch
        n = self.capacity
        self._check(self._lib.nbody_forest_step(self._h,
                                                _dptr(pos, torch.float64, (3, n), "pos"),
                                                _dptr(vel, torch.float64, (3, n), "vel"),
                                                _dptr(mass, torch.float64, (n,), "mass"),
                                                int(nsteps), 1 if use_graph else 0),
                    "nbody_forest_step")

    def autotune(self, pos, mass):
        """Times every launch shape of the walk on this input and keeps the fastest; returns
        (chosen shape, per-shape ms)."""
        import torch
        n = self.capacity if getattr(self, "offsets", None) is not None else int(mass.shape[0])
        ms = (ctypes.c_float * WALK_SHAPES)()
        chosen = ctypes.c_int32()
        self._check(self._lib.nbody_autotune(self._h, _dptr(pos, torch.float64, (3, n), "pos"),
                                             _dptr(mass, torch.float64, (n,), "mass"), n,
                                             ms, ctypes.byref(chosen)), "nbody_autotune")
        return int(chosen.value), [float(x) for x in ms]

    def set_walk_shape(self, shape):
        self._check(self._lib.nbody_set_walk_shape(self._h, int(shape)), "nbody_set_walk_shape")

    def set_walk_limits(self, stack_entries=0, max_steps=0, fast_entries=0):
        """Test aid: lowers the walk's stack entries / steps (0 = the defaults); a walk that
        reaches a limit stops and the next sync() raises NBODY_ESTACK.  fast_entries lowers the
        stack of the FP32 walk's fast kernel (deeper groups go to the full-stack walk)."""
        self._check(self._lib.nbody_set_walk_limits(self._h, int(stack_entries), int(max_steps),
                                                    int(fast_entries)),
                    "nbody_set_walk_limits")

    def walk_shape(self):
        """(shape index, threads per block) of the walk for this context's precision."""
        k, t = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.nbody_get_walk_shape(self._h, ctypes.byref(k), ctypes.byref(t)),
                    "nbody_get_walk_shape")
        return int(k.value), int(t.value)

    def set_sort_mode(self, mode):
        """SORT_AUTO, SORT_FULL or SORT_RESORT (the order is the same in every mode)."""
        self._check(self._lib.nbody_set_sort_mode(self._h, int(mode)), "nbody_set_sort_mode")

    def sort_stats(self):
        """(path, removed) of the last build: path 1 = re-sorted from the previous order,
        0 = full sort, -1 = no build yet; removed = bodies the re-sort took out (-1: not tried)."""
        path, removed = ctypes.c_int32(), ctypes.c_int64()
        self._check(self._lib.nbody_get_sort_stats(self._h, ctypes.byref(path),
                                                   ctypes.byref(removed)), "nbody_get_sort_stats")
        return int(path.value), int(removed.value)

    def sync(self):
        self._check(self._lib.nbody_sync(self._h), "nbody_sync")

    # ---------------------------------------------------------------- introspection
    def keys(self, n):
        k = np.zeros(n, dtype=np.uint64)
        ids = np.zeros(n, dtype=np.uint32)
        self._check(self._lib.nbody_get_keys(self._h, k.ctypes.data_as(ctypes.c_void_p),
                                             ids.ctypes.data_as(ctypes.c_void_p)),
                    "nbody_get_keys")
        return k, ids

    def box(self):
        b = np.zeros(5)
        self._check(self._lib.nbody_get_box(self._h, b.ctypes.data_as(ctypes.c_void_p)),
                    "nbody_get_box")
        return b

    def tree(self):
        """Pre-order records (n_nodes, 5) int64: key, level, child mask, first rank, count."""
        nn = ctypes.c_int64()
        self._check(self._lib.nbody_get_tree(self._h, ctypes.byref(nn), None, 0), "nbody_get_tree")
        recs = np.zeros(max(nn.value, 1), dtype=_RECORD_DTYPE)
        self._check(self._lib.nbody_get_tree(self._h, ctypes.byref(nn),
                                             recs.ctypes.data_as(ctypes.c_void_p), nn.value),
                    "nbody_get_tree")
        recs = recs[:nn.value]
        out = np.empty((nn.value, 5), dtype=np.int64)
        out[:, 0] = recs["key"].view(np.int64)
        out[:, 1] = recs["level"]
        out[:, 2] = recs["child_mask"]
        out[:, 3] = recs["first"]
        out[:, 4] = recs["count"]
        return out

    def n_nodes(self):
        nn = ctypes.c_int64()
        self._check(self._lib.nbody_get_tree(self._h, ctypes.byref(nn), None, 0), "nbody_get_tree")
        return nn.value

    def moments(self):
        """(n_nodes, 4) float64: m, x, y, z of every node in pre-order."""
        nn = self.n_nodes()
        out = np.zeros((max(nn, 1), 4))
        self._check(self._lib.nbody_get_moments(self._h, out.ctypes.data_as(ctypes.c_void_p), nn),
                    "nbody_get_moments")
        return out[:nn]

    def counters(self, n):
        pp = np.zeros(n, dtype=np.uint32)
        pc = np.zeros(n, dtype=np.uint32)
        self._check(self._lib.nbody_get_counters(self._h, pp.ctypes.data_as(ctypes.c_void_p),
                                                 pc.ctypes.data_as(ctypes.c_void_p)),
                    "nbody_get_counters")
        return pp, pc

    def enable_timing(self, on=True):
        self._check(self._lib.nbody_enable_timing(self._h, 1 if on else 0), "nbody_enable_timing")

    def timings(self):
        """Device ms of the last call: box+keys, sort, split+moments, walk, whole call."""
        t = np.zeros(5, dtype=np.float32)
        self._check(self._lib.nbody_get_timings(self._h, t.ctypes.data_as(ctypes.c_void_p)),
                    "nbody_get_timings")
        return t


def launch_count() -> int:
    """Kernel launches made by the library so far in this process."""
    v = ctypes.c_int64()
    st = load_library().nbody_get_launch_count(ctypes.byref(v))
    if st != 0:
        raise NBodyError(st, "nbody_get_launch_count")
    return int(v.value)


def measure_fp32_rate(stream=None) -> float:
    """FP32 fused multiply-add rate of the current device in TFLOP/s (a measurement aid; see
    nbody_measure_fp32_rate in include/nbody.h)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    v = ctypes.c_double()
    st = load_library().nbody_measure_fp32_rate(ctypes.c_void_p(stream.cuda_stream),
                                                ctypes.byref(v))
    if st != 0:
        raise NBodyError(st, "nbody_measure_fp32_rate")
    return float(v.value)


def measure_fp64_rate(stream=None) -> float:
    """FP64 fused multiply-add rate of the current device in TFLOP/s (a measurement aid; see
    nbody_measure_fp64_rate in include/nbody.h)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    v = ctypes.c_double()
    st = load_library().nbody_measure_fp64_rate(ctypes.c_void_p(stream.cuda_stream),
                                                ctypes.byref(v))
    if st != 0:
        raise NBodyError(st, "nbody_measure_fp64_rate")
    return float(v.value)
