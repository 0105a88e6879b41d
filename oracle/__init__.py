"""CPU oracle for the Barnes-Hut timestep -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-checkable FP64 reference of what the paper's method computes (the C
source ``nbody_oracle.c`` beside this file cites the passage each function follows).  Only the
test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it; the
library under ``paper_2203_08966_gb300`` never does, and the two share no code.

Array conventions match the library: positions and velocities are (3, N) float64 row-major
(rows x, y, z), masses (N,) float64.

Parity status of each function (what pins it is in ``tests/test_oracle_pins.py``):
    bbox / quantise / keys / interleave  pinned (paper's worked 2-D example, brute force)
    sort_pairs                           pinned (Python sorted())
    resort_insertion (§4.4 re-sort from  pinned (equals sort_pairs from any starting order;
      last step's order)                 exchanges = brute-force inversion count; none when
                                         the starting order is already sorted)
    tree build / records                 pinned (independent prefix-grouping construction,
                                         paper's octal key examples, invariants)
    moments                              pinned (root centre of mass = global centre of mass;
                                         every cell = mass-weighted mean of its children)
    direct                               pinned (Kepler closed forms, Newton's third law)
    tree forces (Barnes-Hut)             pinned (theta = 0 equals direct sum, N = 2 exact,
                                         brute-force recursive walk on small N)
    quadrupoles, quadrupole walk         pinned (two-body closed form, traceless and symmetric,
                                         far-field error third order in size/distance against
                                         second order for the monopole, smaller BH error)
    kdk                                  pinned (time reversibility, second-order convergence,
                                         circular Kepler orbit)
    bh_group (grouped acceptance test,   pinned (groups of one body equal the per-body walk term
      Barnes 1990; not in the paper)     for term, theta = 0 equals direct sum, every body's
                                         count >= its per-body count; cell groups: a partition
                                         of the bodies into <= 32, each inside one tree cell)
    energy                               pinned (two-body closed form)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, no fast-math), in place."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    d = ctypes.c_double
    sig = {
        "orc_set_threads": (None, [ctypes.c_int]),
        "orc_get_threads": (ctypes.c_int, []),
        "orc_bbox": (None, [_f64p, i64, _f64p]),
        "orc_quantise": (None, [_f64p, i64, _f64p, _u32p]),
        "orc_interleave": (ctypes.c_uint64, [_u32p, ctypes.c_int, ctypes.c_int]),
        "orc_keys": (None, [_f64p, i64, _f64p, _u64p]),
        "orc_sort_pairs": (None, [_u64p, i64, _u64p, _i64p]),
        "orc_resort_insertion": (i64, [_u64p, _i64p, i64, _u64p, _i64p]),
        "orc_direct": (None, [_f64p, _f64p, i64, vp, i64, d, d, _f64p]),
        "orc_tree_build": (vp, [_f64p, _f64p, i64]),
        "orc_tree_free": (None, [vp]),
        "orc_tree_stats": (None, [vp, _i64p]),
        "orc_tree_box": (None, [vp, _f64p]),
        "orc_tree_root": (None, [vp, _f64p]),
        "orc_tree_records": (i64, [vp, _i64p, vp]),
        "orc_tree_moments": (i64, [vp, _f64p]),
        "orc_tree_forces": (None, [vp, vp, i64, d, d, d, _f64p, vp, vp]),
        "orc_tree_forces_q": (None, [vp, vp, i64, d, d, d, ctypes.c_int, _f64p, vp, vp]),
        "orc_tree_quads": (i64, [vp, _f64p]),
        "orc_tree_cell_groups": (i64, [vp, i64, _i64p, _i64p]),
        "orc_tree_forces_group": (None, [vp, _i64p, _i64p, i64, d, d, d, _f64p, vp, vp]),
        "orc_bh": (None, [_f64p, _f64p, i64, d, d, d, _f64p, vp, vp]),
        "orc_kdk": (None, [_f64p, _f64p, _f64p, i64, _f64p, d, d, d, d, ctypes.c_int32,
                           ctypes.c_int32]),
        "orc_energy": (None, [_f64p, _f64p, _f64p, i64, d, d, _f64p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _soa(pos):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    assert pos.ndim == 2 and pos.shape[0] == 3
    return pos


def set_threads(t: int) -> None:
    """OpenMP threads for the per-target loops (results do not depend on it)."""
    _load().orc_set_threads(int(t))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def bbox(pos):
    """(o_x, o_y, o_z, L, s): min corner, cube side (largest extent, 1 if zero), s = 2^21 / L."""
    pos = _soa(pos)
    box = np.zeros(5)
    _load().orc_bbox(pos, pos.shape[1], box)
    return box


def quantise(pos, box=None):
    pos = _soa(pos)
    box = bbox(pos) if box is None else np.ascontiguousarray(box, dtype=np.float64)
    q = np.zeros((3, pos.shape[1]), dtype=np.uint32)
    _load().orc_quantise(pos, pos.shape[1], box, q)
    return q


def interleave(coords, bits: int) -> int:
    """Bit interleave of len(coords) coordinates, coordinate 0 most significant (§4.4)."""
    c = np.ascontiguousarray(np.asarray(coords, dtype=np.uint32))
    return int(_load().orc_interleave(c, len(c), int(bits)))


def keys(pos, box=None):
    pos = _soa(pos)
    box = bbox(pos) if box is None else np.ascontiguousarray(box, dtype=np.float64)
    k = np.zeros(pos.shape[1], dtype=np.uint64)
    _load().orc_keys(pos, pos.shape[1], box, k)
    return k


def sort_pairs(k):
    """Sorted keys and original ids, ascending (key, id)."""
    k = np.ascontiguousarray(k, dtype=np.uint64)
    ko = np.zeros_like(k)
    ids = np.zeros(k.shape[0], dtype=np.int64)
    _load().orc_sort_pairs(k, k.shape[0], ko, ids)
    return ko, ids


def resort_insertion(k, prev):
    """Insertion sort (§4.4) of the bodies taken in the order ``prev`` (last step's sorted ids)
    by (key, id): sorted keys, sorted ids and the number of neighbour exchanges it made."""
    k = np.ascontiguousarray(k, dtype=np.uint64)
    prev = np.ascontiguousarray(prev, dtype=np.int64)
    if prev.shape != k.shape:
        raise ValueError("prev must be a permutation of the key indices")
    ko = np.zeros_like(k)
    ids = np.zeros(k.shape[0], dtype=np.int64)
    swaps = int(_load().orc_resort_insertion(k, prev, k.shape[0], ko, ids))
    return ko, ids, swaps


def direct(pos, mass, G=1.0, eps=0.0, targets=None):
    """Direct-sum accelerations (3, nt) of `targets` (all bodies if None), Algorithm 1."""
    pos = _soa(pos)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    n = pos.shape[1]
    if targets is None:
        acc = np.zeros((3, n))
        _load().orc_direct(pos, mass, n, None, n, G, eps, acc)
    else:
        t = np.ascontiguousarray(targets, dtype=np.int64)
        acc = np.zeros((3, t.shape[0]))
        _load().orc_direct(pos, mass, n, _ptr(t), t.shape[0], G, eps, acc)
    return acc


class Tree:
    """Pointer octree built by insertion (Algorithm 2).  Keeps references to pos and mass."""

    def __init__(self, pos, mass):
        self.pos = _soa(pos)
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.n = self.pos.shape[1]
        self._h = _load().orc_tree_build(self.pos, self.mass, self.n)

    def close(self):
        if self._h:
            _load().orc_tree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self):
        s = np.zeros(4, dtype=np.int64)
        _load().orc_tree_stats(self._h, s)
        return dict(nodes=int(s[0]), depth=int(s[1]), buckets=int(s[2]), leaves=int(s[3]))

    def box(self):
        b = np.zeros(5)
        _load().orc_tree_box(self._h, b)
        return b

    def root(self):
        """(m, x, y, z) of the root."""
        r = np.zeros(4)
        _load().orc_tree_root(self._h, r)
        return r

    def records(self, with_leaf_order: bool = False):
        """Pre-order records (n_nodes, 5) int64: key, level, child mask, first rank, count.

        Column 0 holds the hashed-octree key as a uint64 bit pattern."""
        nn = self.stats()["nodes"]
        rec = np.zeros((max(nn, 1), 5), dtype=np.int64)
        order = np.zeros(max(self.n, 1), dtype=np.int64)
        k = _load().orc_tree_records(self._h, rec, _ptr(order) if with_leaf_order else None)
        rec = rec[:k]
        if with_leaf_order:
            return rec, order[:self.n]
        return rec

    def moments(self):
        """(n_nodes, 4) float64: m, x, y, z of every node, in the pre-order of records()."""
        nn = self.stats()["nodes"]
        out = np.zeros((max(nn, 1), 4))
        k = _load().orc_tree_moments(self._h, out)
        return out[:k]

    def quads(self):
        """Quadrupole moments of every node in the order of records(): (n_nodes, 6) as
        (xx, yy, zz, xy, xz, yz) about each node's centre of mass (§2.2)."""
        nn = self.stats()["nodes"]
        out = np.zeros((max(nn, 1), 6))
        k = _load().orc_tree_quads(self._h, out)
        return out[:k]

    def forces(self, G=1.0, eps=0.0, theta=0.5, targets=None, quadrupole=False):
        """Barnes-Hut accelerations (3, nt) and counters pp, pc (nt,) uint32.  quadrupole: accepted
        cells add their quadrupole term (§2.2, softened like the monopole)."""
        if targets is None:
            nt = self.n
            tp = None
        else:
            t = np.ascontiguousarray(targets, dtype=np.int64)
            nt = t.shape[0]
            tp = t
        acc = np.zeros((3, nt))
        pp = np.zeros(nt, dtype=np.uint32)
        pc = np.zeros(nt, dtype=np.uint32)
        _load().orc_tree_forces_q(self._h, _ptr(tp), nt, G, eps, theta, 1 if quadrupole else 0,
                                  acc, _ptr(pp), _ptr(pc))
        return acc, pp, pc


def bh_group(pos, mass, G=1.0, eps=0.0, theta=0.5, group=32, grouping="cells"):
    """Group-walk accelerations (3, N) and counters pp, pc (N,) under the grouped acceptance
    test (Barnes 1990; not in the paper): a cell is accepted for a whole group when its side and
    the distance from its centre of mass to the group's bounding box pass the test.
    grouping="cells": groups follow the tree's cells (a cell of at most `group` bodies whose
    parent holds more, consecutive such siblings merged while they fit, larger buckets cut into
    chunks); grouping="chunks": consecutive runs of `group` bodies in Morton order."""
    pos = _soa(pos)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    n = pos.shape[1]
    t = Tree(pos, mass)
    try:
        if grouping == "cells":
            members = np.zeros(n, dtype=np.int64)
            offsets = np.zeros(n + 1, dtype=np.int64)
            ng = int(_load().orc_tree_cell_groups(t._h, int(group), members, offsets))
        elif grouping == "chunks":
            _, members = sort_pairs(keys(pos))
            members = np.ascontiguousarray(members, dtype=np.int64)
            offsets = np.minimum(np.arange(0, n + group, group, dtype=np.int64), n)
            offsets = np.ascontiguousarray(np.unique(offsets))
            ng = offsets.shape[0] - 1
        else:
            raise ValueError(grouping)
        acc = np.zeros((3, n))
        pp = np.zeros(n, dtype=np.uint32)
        pc = np.zeros(n, dtype=np.uint32)
        _load().orc_tree_forces_group(t._h, members, offsets, ng, G, eps, theta, acc, _ptr(pp),
                                      _ptr(pc))
        return acc, pp, pc
    finally:
        t.close()


def cell_groups(pos, mass, group=32):
    """The groups of bh_group(grouping="cells") as a list of user-id arrays."""
    pos = _soa(pos)
    n = pos.shape[1]
    t = Tree(pos, np.ascontiguousarray(mass, dtype=np.float64))
    try:
        members = np.zeros(n, dtype=np.int64)
        offsets = np.zeros(n + 1, dtype=np.int64)
        ng = int(_load().orc_tree_cell_groups(t._h, int(group), members, offsets))
        return [members[offsets[k]:offsets[k + 1]].copy() for k in range(ng)]
    finally:
        t.close()


def bh(pos, mass, G=1.0, eps=0.0, theta=0.5, quadrupole=False):
    """Barnes-Hut accelerations of all bodies plus (pp, pc) counters (with the cells' quadrupole
    terms when `quadrupole`)."""
    t = Tree(pos, mass)
    try:
        return t.forces(G, eps, theta, quadrupole=quadrupole)
    finally:
        t.close()


def kdk(pos, vel, mass, acc, G=1.0, eps=0.0, theta=0.5, dt=1e-3, nsteps=1, method="bh"):
    """Advance copies of (pos, vel) by nsteps KDK steps.  `acc` = a^(k) at the entry positions.

    Returns (pos, vel, acc) at the end."""
    pos = _soa(pos).copy()
    vel = _soa(vel).copy()
    acc = np.ascontiguousarray(acc, dtype=np.float64).copy()
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    m = {"direct": 0, "bh": 1}[method]
    _load().orc_kdk(pos, vel, mass, pos.shape[1], acc, G, eps, theta, dt, int(nsteps), m)
    return pos, vel, acc


def energy(pos, vel, mass, G=1.0, eps=0.0):
    """(E_kin, E_pot, E_tot), §2.3 with the pair sum over i < j."""
    pos = _soa(pos)
    vel = _soa(vel)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    out = np.zeros(3)
    _load().orc_energy(pos, vel, mass, pos.shape[1], G, eps, out)
    return tuple(float(x) for x in out)


def momentum(vel, mass):
    """Total momentum sum m v (3,)."""
    return (np.asarray(vel) * np.asarray(mass)[None, :]).sum(axis=1)


if __name__ == "__main__":  # pragma: no cover
    build(force=True)
    print(_LIB, file=sys.stderr)
