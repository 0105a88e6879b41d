"""Pins for the CPU oracle: each check ties it to something other than itself -- the paper's
worked examples (tests/golden), closed forms, invariants, or an independent brute-force
construction -- so that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.  CPU only.
"""
import math

import numpy as np
import pytest

import ics
import oracle
from conftest import read_golden

B21 = 21


# ---------------------------------------------------------------- Morton keys (§4.4)

def test_morton_2d_worked_example():
    for x, y, bits, key in read_golden("morton_2d.txt"):
        assert oracle.interleave([int(x), int(y)], int(bits)) == int(key)


def _deinterleave3(key):
    """Inverse of the 3-D interleave (independent: peels bits from the least significant end)."""
    c = [0, 0, 0]
    for b in range(B21):
        for k in (2, 1, 0):
            c[k] |= (key & 1) << b
            key >>= 1
    return c


def test_morton_3d_round_trip_and_order():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        c = [int(v) for v in rng.integers(0, 1 << B21, 3)]
        key = oracle.interleave(c, B21)
        assert key < (1 << 63)
        assert _deinterleave3(key) == c
    # x is the most significant coordinate: the top bit of x outranks everything in y and z
    assert oracle.interleave([1 << 20, 0, 0], B21) > oracle.interleave([0, (1 << 21) - 1, (1 << 21) - 1], B21)
    assert oracle.interleave([0, 1 << 20, 0], B21) > oracle.interleave([0, 0, (1 << 21) - 1], B21)
    assert oracle.interleave([0, 0, 1], B21) == 1
    assert oracle.interleave([0, 1, 0], B21) == 2
    assert oracle.interleave([1, 0, 0], B21) == 4


def test_bbox_and_quantise_closed_forms():
    # box [0, 1]^3 (corners present), so o = 0, L = 1, s = 2^21
    pos = np.array([[0.0, 1.0, 0.5, 0.25, 0.75, 1.0 - 2.0 ** -22],
                    [0.0, 1.0, 0.5, 0.5, 0.125, 0.0],
                    [0.0, 1.0, 0.0, 0.0, 0.0, 0.0]])
    box = oracle.bbox(pos)
    assert list(box) == [0.0, 0.0, 0.0, 1.0, 2.0 ** 21]
    q = oracle.quantise(pos, box)
    assert list(q[0]) == [0, (1 << 21) - 1, 1 << 20, 1 << 19, 3 << 19, (1 << 21) - 1]
    assert list(q[1]) == [0, (1 << 21) - 1, 1 << 20, 1 << 20, 1 << 18, 0]
    # cube side is the largest extent; the other axes keep their own min corner
    pos2 = np.array([[2.0, 6.0], [-1.0, 0.0], [10.0, 10.5]])
    box2 = oracle.bbox(pos2)
    assert list(box2[:4]) == [2.0, -1.0, 10.0, 4.0]
    # all bodies at one point: side 1
    box3 = oracle.bbox(np.ones((3, 5)))
    assert box3[3] == 1.0 and box3[4] == 2.0 ** 21


def test_quantise_monotone_and_in_range():
    pos, _, _ = ics.plummer(5000, 3)
    q = oracle.quantise(pos)
    assert q.max() <= (1 << 21) - 1
    for d in range(3):
        order = np.argsort(pos[d], kind="stable")
        assert np.all(np.diff(q[d][order].astype(np.int64)) >= 0)
        assert q[d][np.argmin(pos[d])] == 0


def test_sort_pairs_matches_python_sort():
    rng = np.random.default_rng(5)
    k = rng.integers(0, 64, 3000).astype(np.uint64)  # many ties
    ks, ids = oracle.sort_pairs(k)
    ref = sorted((int(v), i) for i, v in enumerate(k))
    assert [int(v) for v in ks] == [a for a, _ in ref]
    assert list(ids) == [b for _, b in ref]


# ---------------------------------------------------------------- re-sort from last step's order (§4.4)

def _inversions(k, order):
    """Brute force: pairs (a, b), a before b in `order`, that the (key, id) order puts the other
    way round."""
    c = [(int(k[i]), int(i)) for i in order]
    return sum(1 for a in range(len(c)) for b in range(a + 1, len(c)) if c[a] > c[b])


@pytest.mark.parametrize("start", ["random", "sorted", "reversed", "near"])
def test_resort_insertion_equals_sort_and_counts_inversions(start):
    rng = np.random.default_rng(11)
    n = 400
    k = rng.integers(0, 50, n).astype(np.uint64)       # many equal keys: ties go by id
    ks, ids = oracle.sort_pairs(k)
    if start == "random":
        prev = rng.permutation(n)
    elif start == "sorted":
        prev = ids.copy()
    elif start == "reversed":
        prev = ids[::-1].copy()
    else:  # last step's order after a few bodies moved
        prev = ids.copy()
        for a in rng.integers(0, n - 3, 12):
            prev[a], prev[a + 2] = prev[a + 2], prev[a]
    ko, io, swaps = oracle.resort_insertion(k, prev)
    assert np.array_equal(ko, ks) and np.array_equal(io, ids)
    assert swaps == _inversions(k, prev)
    if start == "sorted":
        assert swaps == 0
    if start == "reversed":
        assert swaps == n * (n - 1) // 2


def test_resort_insertion_after_a_drift_is_cheap():
    """After one small drift of a Plummer sphere last step's order is almost sorted: few
    exchanges (the premise of §4.4), and the result is the sort of the new keys."""
    pos, vel, _ = ics.plummer(20000, 9)
    _, prev = oracle.sort_pairs(oracle.keys(pos))
    pos2 = pos + 5e-4 * vel
    k2 = oracle.keys(pos2)
    ko, io, swaps = oracle.resort_insertion(k2, prev)
    ks, ids = oracle.sort_pairs(k2)
    assert np.array_equal(ko, ks) and np.array_equal(io, ids)
    assert 0 < swaps < 20 * 20000     # a random order would need about n^2 / 4 = 1e8


# ---------------------------------------------------------------- tree (Algorithm 2, §4.2, §4.7)

def _tree_by_prefix(sorted_keys):
    """Independent top-down construction: split the sorted key list by 3-bit prefixes.

    Returns pre-order records (key, level, mask, first, count)."""
    ks = [int(v) for v in sorted_keys]
    out = []

    def rec(lo, hi, level):
        prefix = 0 if level == 0 else ks[lo] >> (3 * (B21 - level))
        hkey = (1 << (3 * level)) | prefix
        count = hi - lo
        if count == 1 or level == B21:
            out.append((hkey, level, 0, lo, count))
            return
        shift = 3 * (B21 - level - 1)
        runs = []
        i = lo
        while i < hi:
            dg = (ks[i] >> shift) & 7
            j = i
            while j < hi and ((ks[j] >> shift) & 7) == dg:
                j += 1
            runs.append((dg, i, j))
            i = j
        mask = 0
        for dg, _, _ in runs:
            mask |= 1 << dg
        out.append((hkey, level, mask, lo, count))
        for _, a, b in runs:
            rec(a, b, level + 1)

    if ks:
        rec(0, len(ks), 0)
    return out


def _records_as_tuples(rec):
    return [(int(np.uint64(r[0].astype(np.uint64))), int(r[1]), int(r[2]), int(r[3]), int(r[4]))
            for r in rec]


@pytest.mark.parametrize("case", ["plummer", "cube", "dupes", "line", "tiny"])
def test_tree_equals_prefix_construction(case):
    if case == "plummer":
        pos, _, m = ics.plummer(3000, 21)
    elif case == "cube":
        pos, _, m = ics.uniform_cube(2000, 22)
    elif case == "dupes":
        pos, _, m = ics.uniform_cube(300, 23)
        pos[:, 100:140] = pos[:, 7:8]          # 41 coincident bodies -> one level-21 bucket
        pos[:, 200] = pos[:, 201]
    elif case == "line":
        x = np.linspace(0.0, 1.0, 257)
        pos = np.stack([x, np.zeros_like(x), np.zeros_like(x)])
        m = np.ones(257)
    else:
        pos = np.array([[0.1, 0.9, 0.11], [0.1, 0.9, 0.1], [0.1, 0.9, 0.1]])
        m = np.ones(3)
    t = oracle.Tree(pos, m)
    rec, order = t.records(with_leaf_order=True)
    ks, ids = oracle.sort_pairs(oracle.keys(pos))
    assert _records_as_tuples(rec) == _tree_by_prefix(ks)
    # the pre-order walk meets the bodies exactly in Morton (key, id) order
    assert np.array_equal(order, ids)
    # invariants: an internal node holds >= 2 bodies and its count is the sum of its children's
    st = t.stats()
    assert st["nodes"] == len(rec)
    internal = rec[rec[:, 2] != 0]
    assert np.all(internal[:, 4] >= 2)
    leaves = rec[rec[:, 2] == 0]
    assert leaves[:, 4].sum() == pos.shape[1]
    assert np.all((leaves[:, 4] == 1) | (leaves[:, 1] == B21))


def test_hashed_keys_golden():
    # one body in every octant of the unit cube: the root's children carry keys 10..17 (octal)
    corners = np.array([[(d >> 2) & 1, (d >> 1) & 1, d & 1] for d in range(8)], dtype=float)
    pos = np.ascontiguousarray((0.25 + 0.5 * corners).T)
    pos = np.concatenate([pos, np.zeros((3, 1)), np.ones((3, 1))], axis=1)  # pin the box to [0,1]
    t = oracle.Tree(pos, np.ones(pos.shape[1]))
    rec = t.records()
    keys_oct = {oct(int(r[0]))[2:] for r in rec}
    golden = read_golden("hashed_keys.txt")
    for parent, digit, child in golden:
        # parent = child >> 3
        assert int(child, 8) >> 3 == int(parent, 8)
        assert (int(parent, 8) << 3) | int(digit) == int(child, 8)
    for parent, digit, child in golden[:8]:
        assert child in keys_oct
    assert rec[0][0] == 1 and rec[0][2] == 0xFF
    # octant of each level-1 cell follows Fig. `hot` (x > y > z)
    for xh, yh, zh, key in read_golden("hot_octants.txt"):
        p = np.array([[0.25 + 0.5 * int(xh)], [0.25 + 0.5 * int(yh)], [0.25 + 0.5 * int(zh)]])
        pp = np.concatenate([p, np.zeros((3, 1)), np.ones((3, 1))], axis=1)
        assert int(oracle.keys(pp)[0]) >> 60 == int(key, 8) & 7
        r = oracle.Tree(pp, np.ones(3)).records()
        assert any(oct(int(x[0]))[2:] == key and int(x[1]) == 1 for x in r)


def test_tree_edge_cases():
    t0 = oracle.Tree(np.zeros((3, 0)), np.zeros(0))
    assert t0.stats()["nodes"] == 0 and len(t0.records()) == 0
    t1 = oracle.Tree(np.array([[1.0], [2.0], [3.0]]), np.array([2.0]))
    r1 = t1.records()
    assert len(r1) == 1 and r1[0][1] == 0 and r1[0][4] == 1
    assert list(t1.root()) == [2.0, 1.0, 2.0, 3.0]
    # all bodies at one point: a chain of one-child nodes down to a level-21 bucket
    t5 = oracle.Tree(np.full((3, 5), 0.3), np.ones(5))
    r5 = t5.records()
    assert len(r5) == 22
    assert [int(r[1]) for r in r5] == list(range(22))
    assert all(int(r[4]) == 5 for r in r5)
    assert t5.stats()["buckets"] == 1


def test_moments_root_is_global_centre_of_mass():
    pos, _, _ = ics.plummer(20000, 31)
    m = np.random.default_rng(1).uniform(0.5, 2.0, 20000)
    t = oracle.Tree(pos, m)
    root = t.root()
    msum = math.fsum(m)
    assert abs(root[0] - msum) <= 1e-14 * msum
    for d in range(3):
        com = math.fsum(m * pos[d]) / msum
        assert abs(root[1 + d] - com) <= 1e-13 * (np.abs(pos[d]).max())


# ---------------------------------------------------------------- forces (eq. motion, Alg. 1)

@pytest.mark.parametrize("eps", [0.0, 0.1])
def test_direct_two_body_closed_form(eps):
    m1, m2, r = 0.3, 0.7, 1.7
    pos = np.array([[0.0, r], [0.0, 0.0], [0.0, 0.0]])
    a = oracle.direct(pos, np.array([m1, m2]), G=2.0, eps=eps)
    k = 2.0 / (r * r + eps * eps) ** 1.5
    assert a[0, 0] == pytest.approx(k * m2 * r, rel=1e-15)      # pulled towards +x
    assert a[0, 1] == pytest.approx(-k * m1 * r, rel=1e-15)
    assert np.all(a[1:] == 0.0)


def test_direct_newton_third_law():
    pos, _, _ = ics.plummer(3000, 41)
    m = np.random.default_rng(2).uniform(0.5, 2.0, 3000) / 3000
    a = oracle.direct(pos, m, eps=0.01)
    net = (a * m).sum(axis=1)
    scale = (np.linalg.norm(a, axis=0) * m).sum()
    assert np.linalg.norm(net) <= 1e-13 * scale


def test_direct_targets_subset():
    pos, _, m = ics.plummer(500, 42)
    full = oracle.direct(pos, m, eps=0.01)
    idx = np.array([0, 17, 499, 250])
    sub = oracle.direct(pos, m, eps=0.01, targets=idx)
    assert np.array_equal(sub, full[:, idx])


# ---------------------------------------------------------------- Barnes-Hut walk (Algorithm 2)

def test_bh_theta_zero_is_direct_sum():
    pos, _, m = ics.plummer(2048, 51)
    a, pp, pc = oracle.bh(pos, m, eps=0.01, theta=0.0)
    ad = oracle.direct(pos, m, eps=0.01)
    assert np.all(pc == 0) and np.all(pp == 2047)
    assert np.abs(a - ad).max() <= 1e-13 * np.abs(ad).max()


def test_bh_two_bodies_exact():
    pos = np.array([[0.0, 1.0], [0.5, -0.25], [2.0, 2.5]])
    m = np.array([1.5, 0.25])
    a, pp, pc = oracle.bh(pos, m, G=1.3, eps=0.05, theta=0.9)
    ad = oracle.direct(pos, m, G=1.3, eps=0.05)
    assert np.array_equal(a, ad)
    assert list(pp) == [1, 1] and list(pc) == [0, 0]


def _brute_walk(pos, m, G, eps, theta):
    """Independent recursive Barnes-Hut on the prefix-built tree, centre of mass taken directly
    over each cell's bodies.  Returns acc (3, n), pp, pc."""
    n = pos.shape[1]
    ks, ids = oracle.sort_pairs(oracle.keys(pos))
    L = oracle.bbox(pos)[3]
    recs = _tree_by_prefix(ks)
    # children lists from pre-order records
    kids = {i: [] for i in range(len(recs))}
    stack = []
    for i, (_, lev, _, first, cnt) in enumerate(recs):
        while stack and not (recs[stack[-1]][3] <= first < recs[stack[-1]][3] + recs[stack[-1]][4]
                             and recs[stack[-1]][1] < lev):
            stack.pop()
        if stack:
            kids[stack[-1]].append(i)
        stack.append(i)
    cm = []
    for (_, lev, _, first, cnt) in recs:
        b = ids[first:first + cnt]
        mm = m[b].sum()
        cm.append((mm, (pos[:, b] * m[b]).sum(axis=1) / mm, b))
    acc = np.zeros((3, n))
    pp = np.zeros(n, dtype=np.int64)
    pc = np.zeros(n, dtype=np.int64)

    def pull(p, xj, mj):
        d = xj - pos[:, p]
        r2 = d @ d + eps * eps
        return G * mj * d / r2 ** 1.5 if r2 > 0 else np.zeros(3)

    def walk(p, node):
        for c in kids[node]:
            lev, cnt = recs[c][1], recs[c][4]
            mm, com, b = cm[c]
            if cnt == 1 or lev == B21:
                for j in b:
                    if j != p:
                        acc[:, p] += pull(p, pos[:, j], m[j])
                        pp[p] += 1
            else:
                ell = L / 2.0 ** lev
                dd = com - pos[:, p]
                if ell * ell < theta * theta * (dd @ dd):
                    acc[:, p] += pull(p, com, mm)
                    pc[p] += 1
                else:
                    walk(p, c)

    for p in range(n):
        if recs and recs[0][4] > 1:
            walk(p, 0)
    return acc, pp, pc


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7, 1.0])
def test_bh_matches_brute_force_walk(theta):
    pos, _, _ = ics.plummer(300, 61)
    m = np.random.default_rng(3).uniform(0.5, 1.5, 300) / 300
    a, pp, pc = oracle.bh(pos, m, G=1.0, eps=0.02, theta=theta)
    ab, ppb, pcb = _brute_walk(pos, m, 1.0, 0.02, theta)
    assert np.array_equal(pp, ppb) and np.array_equal(pc, pcb)
    assert np.abs(a - ab).max() <= 1e-12 * np.abs(ab).max()
    if theta >= 0.5:
        assert pc.sum() > 0


def test_bh_error_decreases_with_theta():
    pos, _, m = ics.plummer(4096, 1)
    ad = oracle.direct(pos, m, eps=0.01)
    errs = []
    for th in (0.7, 0.5, 0.3):
        a, _, _ = oracle.bh(pos, m, eps=0.01, theta=th)
        e = np.sqrt(((a - ad) ** 2).sum(0) / (ad ** 2).sum(0))
        errs.append(np.sqrt((e ** 2).mean()))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 2e-2


def test_bh_coincident_bodies_bucket():
    pos = np.full((3, 4), 0.5)
    pos = np.concatenate([pos, np.array([[2.0], [0.5], [0.5]])], axis=1)
    m = np.ones(5)
    for eps in (0.0, 0.1):
        a, pp, pc = oracle.bh(pos, m, eps=eps, theta=0.5)
        assert np.all(np.isfinite(a))
        assert list(pp[:4]) == [4, 4, 4, 4]
        ad = oracle.direct(pos, m, eps=eps)
        assert np.allclose(a, ad, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- KDK leapfrog (§2.4) and energy (§2.3)

def _circular_pair(eps, r=1.0, m1=0.5, m2=0.5):
    M = m1 + m2
    w = math.sqrt(M / (r * r + eps * eps) ** 1.5)
    pos = np.array([[-m2 / M * r, m1 / M * r], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [-m2 / M * r * w, m1 / M * r * w], [0.0, 0.0]])
    return pos, vel, np.array([m1, m2]), 2 * math.pi / w


@pytest.mark.parametrize("eps", [0.0, 0.2])
def test_kdk_circular_orbit_second_order(eps):
    pos, vel, m, period = _circular_pair(eps)
    errs = []
    for nstep in (200, 400):
        a0 = oracle.direct(pos, m, eps=eps)
        p1, _, _ = oracle.kdk(pos, vel, m, a0, eps=eps, dt=period / nstep, nsteps=nstep,
                              method="direct")
        errs.append(np.abs(p1 - pos).max())
    assert errs[0] < 5e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_kdk_eccentric_kepler_period():
    # e = 0.5, a = 1, G M = 1, start at apocentre: period 2 pi sqrt(a^3 / G M)
    e, a = 0.5, 1.0
    r_apo = a * (1 + e)
    v_apo = math.sqrt((1 - e) / (1 + e) / a)
    m = np.array([1e-12, 1.0])  # test particle around a unit mass, eps = 0
    pos = np.array([[r_apo, 0.0], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [v_apo, 0.0], [0.0, 0.0]])
    nstep = 4000
    acc = oracle.direct(pos, m, eps=0.0)
    p1, _, _ = oracle.kdk(pos, vel, m, acc, eps=0.0, dt=2 * math.pi / nstep, nsteps=nstep,
                          method="direct")
    assert np.abs(p1[:, 0] - pos[:, 0]).max() < 2e-3


def test_kdk_time_reversible():
    pos, vel, m = ics.plummer(64, 71)
    acc = oracle.direct(pos, m, eps=0.05)
    p1, v1, a1 = oracle.kdk(pos, vel, m, acc, eps=0.05, dt=1e-3, nsteps=50, method="direct")
    p2, v2, _ = oracle.kdk(p1, v1, m, a1, eps=0.05, dt=-1e-3, nsteps=50, method="direct")
    assert np.abs(p2 - pos).max() < 1e-12
    assert np.abs(v2 - vel).max() < 1e-12


def test_kdk_bh_step_matches_manual_sequence():
    pos, vel, m = ics.plummer(500, 72)
    eps, th, dt = 0.01, 0.5, 1e-3
    a0, _, _ = oracle.bh(pos, m, eps=eps, theta=th)
    p1, v1, a1 = oracle.kdk(pos, vel, m, a0, eps=eps, theta=th, dt=dt, nsteps=1, method="bh")
    vh = vel + a0 * (0.5 * dt)
    pm = pos + vh * dt
    am, _, _ = oracle.bh(pm, m, eps=eps, theta=th)
    assert np.array_equal(p1, pm)
    assert np.array_equal(a1, am)
    assert np.array_equal(v1, vh + am * (0.5 * dt))


def test_energy_two_body_closed_form():
    pos = np.array([[0.0, 3.0], [0.0, 4.0], [0.0, 0.0]])
    vel = np.array([[1.0, 0.0], [0.0, 2.0], [0.0, 0.0]])
    m = np.array([2.0, 3.0])
    ek, ep, et = oracle.energy(pos, vel, m, G=1.0, eps=0.0)
    assert ek == pytest.approx(0.5 * 2.0 * 1.0 + 0.5 * 3.0 * 4.0, rel=1e-15)
    assert ep == pytest.approx(-6.0 / 5.0, rel=1e-15)
    _, ep2, _ = oracle.energy(pos, vel, m, G=1.0, eps=0.5)
    assert ep2 == pytest.approx(-6.0 / math.sqrt(25.25), rel=1e-15)


def test_energy_and_momentum_drift_plummer():
    """The paper's validation criterion (§2.3, §5): total energy is conserved up to the
    integrator's truncation error; momentum to rounding (direct sum is antisymmetric)."""
    pos, vel, m = ics.plummer(1024, 81)
    eps, dt = 0.01, 1e-3
    e0 = oracle.energy(pos, vel, m, eps=eps)[2]
    p0 = oracle.momentum(vel, m)
    acc = oracle.direct(pos, m, eps=eps)
    p1, v1, _ = oracle.kdk(pos, vel, m, acc, eps=eps, dt=dt, nsteps=20, method="direct")
    e1 = oracle.energy(p1, v1, m, eps=eps)[2]
    assert abs(e1 - e0) / abs(e0) < 1e-4
    assert np.abs(oracle.momentum(v1, m) - p0).max() < 1e-14


def test_moments_every_cell_is_mean_of_children():
    """Algorithm 2 moments: each cell's mass is the sum of its children's, its centre of mass
    their mass-weighted mean; a one-body leaf holds its body exactly."""
    pos, _, _ = ics.plummer(3000, 33)
    m = np.random.default_rng(2).uniform(0.5, 2.0, 3000)
    t = oracle.Tree(pos, m)
    rec, order = t.records(with_leaf_order=True)
    mom = t.moments()
    assert mom.shape == (len(rec), 4)
    level = rec[:, 1]
    for k in range(len(rec)):
        first, count = int(rec[k, 3]), int(rec[k, 4])
        bodies = order[first:first + count]
        msum = math.fsum(m[bodies])
        assert abs(mom[k, 0] - msum) <= 1e-13 * msum
        for d in range(3):
            com = math.fsum(m[bodies] * pos[d, bodies]) / msum
            assert abs(mom[k, 1 + d] - com) <= 1e-12 * max(1.0, abs(com))
        if count == 1:
            b = bodies[0]
            assert list(mom[k]) == [m[b], pos[0, b], pos[1, b], pos[2, b]]
    # children of the root are the records at level 1
    kids = np.nonzero(level == 1)[0]
    assert abs(math.fsum(mom[kids, 0]) - mom[0, 0]) <= 1e-13 * mom[0, 0]


# ---- group walk (grouped acceptance test of Barnes 1990; not in the paper) ----------------

@pytest.mark.parametrize("name", ["plummer", "coincident", "uniform"])
def test_group_walk_of_single_bodies_is_the_per_body_walk(name):
    """With groups of one body the group's box is the body itself, so every decision and every
    term is the per-body walk's: bit-identical forces and counters."""
    if name == "plummer":
        pos, _, mass = ics.plummer(2000, 41)
    elif name == "coincident":
        pos, _, mass = ics.plummer(800, 42)
        pos[:, 50:70] = pos[:, 50:51]
    else:
        pos, _, mass = ics.uniform_cube(700, 43)
    for theta in (0.0, 0.5, 0.9):
        a, pp, pc = oracle.bh(pos, mass, 1.0, 0.01, theta)
        g, gpp, gpc = oracle.bh_group(pos, mass, 1.0, 0.01, theta, group=1)
        assert np.array_equal(a, g)
        assert np.array_equal(pp, gpp) and np.array_equal(pc, gpc)


def test_group_walk_theta_zero_is_direct_sum():
    pos, _, mass = ics.plummer(1500, 44)
    g, gpp, gpc = oracle.bh_group(pos, mass, 1.0, 0.01, 0.0, group=32)
    d = oracle.direct(pos, mass, 1.0, 0.01)
    assert np.all(gpc == 0) and np.all(gpp == 1499)
    assert np.abs(g - d).max() <= 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("theta", [0.3, 0.6, 0.9])
def test_group_walk_refines_every_per_body_list(theta):
    """A cell the group accepts passes the test for every member (its distance to a member is
    at least the distance to the group's box), so each group list splits each per-body list
    further: no body has fewer interactions, and the group forces are at least as accurate in
    aggregate."""
    pos, _, mass = ics.plummer(4000, 45)
    a, pp, pc = oracle.bh(pos, mass, 1.0, 0.01, theta)
    g, gpp, gpc = oracle.bh_group(pos, mass, 1.0, 0.01, theta, group=32)
    assert np.all(gpp.astype(np.int64) + gpc >= pp.astype(np.int64) + pc)
    d = oracle.direct(pos, mass, 1.0, 0.01)
    err = lambda x: np.sqrt(((x - d) ** 2).sum() / (d ** 2).sum())
    assert err(g) <= err(a)


def _cell_groups_from_keys(pos, gmax=32):
    """Brute-force restatement of the cell-grouping rule on sorted Morton keys: a body's cell is
    the largest cell around it with at most gmax bodies; consecutive cells with the same parent
    merge while the group stays within gmax; bodies of a bucket larger than gmax go in chunks."""
    k, order = oracle.sort_pairs(oracle.keys(pos))
    n = len(k)
    if n <= gmax:
        return [set(order.tolist())]
    prefix = lambda a, lev: int(k[a]) >> (3 * (21 - lev)) if lev < 21 else int(k[a])
    def run(a, lev):
        p = prefix(a, lev)
        return sum(1 for b in range(n) if prefix(b, lev) == p)
    groups, cur, cur_parent, cur_cell = [], [], None, None
    a = 0
    while a < n:
        lev = next((l for l in range(1, 22) if run(a, l) <= gmax), None)
        if lev is None:                      # bucket larger than gmax: chunks
            if cur:
                groups.append(cur)
                cur, cur_parent = [], None
            p = int(k[a])
            b = a
            while b < n and int(k[b]) == p:
                b += 1
            for s in range(a, b, gmax):
                groups.append(order[s:min(b, s + gmax)].tolist())
            a = b
            continue
        cell = (lev, prefix(a, lev))
        size = run(a, lev)
        parent = (lev - 1, prefix(a, lev - 1))
        if cur and (parent != cur_parent or len(cur) + size > gmax):
            groups.append(cur)
            cur = []
        cur_parent = parent
        cur.extend(order[a:a + size].tolist())
        a += size
    if cur:
        groups.append(cur)
    return [set(g) for g in groups]


@pytest.mark.parametrize("name", ["plummer", "coincident", "uniform"])
def test_cell_groups_match_brute_force_rule(name):
    if name == "plummer":
        pos, _, mass = ics.plummer(900, 46)
    elif name == "coincident":
        pos, _, mass = ics.plummer(600, 47)
        pos[:, 10:80] = pos[:, 10:11]          # a 70-body bucket
    else:
        pos, _, mass = ics.uniform_cube(700, 48)
    got = [set(g.tolist()) for g in oracle.cell_groups(pos, mass, 32)]
    want = _cell_groups_from_keys(pos, 32)
    assert sorted(map(sorted, got)) == sorted(map(sorted, want))
    assert max(len(g) for g in got) <= 32


# ---- quadrupole moments (§2.2, truncated multipole expansion) ------------------------------

def test_quadrupole_two_body_closed_form():
    """Two masses m at (+-a, 0, 0): about their centre of mass Q_xx = 4 m a^2,
    Q_yy = Q_zz = -2 m a^2, no off-diagonal terms."""
    a, m = 0.7, 0.3
    pos = np.array([[-a, a], [0.0, 0.0], [0.0, 0.0]])
    t = oracle.Tree(pos, np.array([m, m]))
    q = t.quads()[0]   # the root
    t.close()
    assert np.allclose(q, [4 * m * a * a, -2 * m * a * a, -2 * m * a * a, 0, 0, 0], rtol=1e-14,
                       atol=1e-15)


def test_quadrupoles_are_traceless_and_vanish_for_single_bodies():
    pos, _, mass = ics.plummer(500, 61)
    t = oracle.Tree(pos, mass)
    q = t.quads()
    rec = t.records()
    t.close()
    scale = np.abs(q).max(axis=1) + 1e-300
    assert np.all(np.abs(q[:, 0] + q[:, 1] + q[:, 2]) <= 1e-12 * scale)
    single = rec[:, 4] == 1
    assert np.all(q[single] == 0.0)


def test_quadrupole_far_field_error_is_third_order():
    """A small cluster (radius 0.5) seen from a body at distance R: with the cell accepted, the
    monopole's relative error falls as (a/R)^2 (the dipole vanishes about the centre of mass),
    the quadrupole expansion's as (a/R)^3."""
    rng = np.random.default_rng(62)
    k = 30
    u = rng.normal(size=(3, k))
    u *= 0.5 * rng.uniform(0, 1, k) ** (1 / 3) / np.linalg.norm(u, axis=0)
    mass = np.concatenate([rng.uniform(0.5, 1.5, k), [1.0]])
    direction = np.array([1.0, 0.3, 0.2]) / np.linalg.norm([1.0, 0.3, 0.2])
    err = {False: [], True: []}
    for R in (40.0, 80.0, 160.0):
        pos = np.concatenate([u, (R * direction)[:, None]], axis=1)
        d = oracle.direct(pos, mass, 1.0, 0.0, targets=np.array([k]))[:, 0]
        for quad in (False, True):
            t = oracle.Tree(pos, mass)
            a, pp, pc = t.forces(1.0, 0.0, 0.7, targets=np.array([k]), quadrupole=quad)
            t.close()
            assert pc[0] >= 1   # the cluster is seen as cell(s)
            err[quad].append(np.linalg.norm(a[:, 0] - d) / np.linalg.norm(d))
    mono, quad = err[False], err[True]
    for r in (mono[0] / mono[1], mono[1] / mono[2]):
        assert 3.0 < r < 5.0, mono
    for r in (quad[0] / quad[1], quad[1] / quad[2]):
        assert 6.0 < r < 10.0, quad
    assert all(q < m for q, m in zip(quad, mono))


def test_quadrupole_walk_theta_zero_and_smaller_error():
    pos, _, mass = ics.plummer(2500, 63)
    a0, _, _ = oracle.bh(pos, mass, 1.0, 0.01, 0.0)
    q0, _, _ = oracle.bh(pos, mass, 1.0, 0.01, 0.0, quadrupole=True)
    assert np.array_equal(a0, q0)   # no cell is ever accepted
    d = oracle.direct(pos, mass, 1.0, 0.01)
    err = lambda x: np.sqrt(((x - d) ** 2).sum() / (d ** 2).sum())
    for theta in (0.5, 0.7):
        a, pp, pc = oracle.bh(pos, mass, 1.0, 0.01, theta)
        q, qpp, qpc = oracle.bh(pos, mass, 1.0, 0.01, theta, quadrupole=True)
        assert np.array_equal(pp, qpp) and np.array_equal(pc, qpc)   # same lists
        assert err(q) < 0.5 * err(a)
