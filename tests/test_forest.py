"""Forest parity: many independent systems advanced by one set of launches (nbody_forest_*).

Every system of a forest must give what the oracle gives for that system alone: keys and sort
order bit-exact (the forest sorts by system, then key, then index), FP64 forces, counters and
leapfrog states bit-exact, FP32 forces within a relative RMS of 1e-4 of the oracle's Barnes-Hut
at the same theta.  A step replayed from a CUDA graph must equal the same step launched
kernel by kernel, bit for bit.
"""
import numpy as np
import pytest

import ics
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2203_08966_gb300 as nb  # noqa: E402

DEV = "cuda:0"
FP32_TOL = 1e-4


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_rms(a, ref):
    num = ((a - ref) ** 2).sum(axis=0)
    den = (ref ** 2).sum(axis=0)
    ok = den > 0
    return float(np.sqrt(np.mean(num[ok] / den[ok]))) if ok.any() else 0.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def small_forest():
    """Systems of ragged sizes (an empty one, single bodies, a pair, several tiles), each its own
    Plummer sphere placed at its own centre, one with a level-21 bucket."""
    sizes = [1, 2, 0, 3, 64, 100, 1000, 513, 4096, 33]
    parts, vels, masses = [], [], []
    for k, n in enumerate(sizes):
        if n == 0:
            continue
        p, v, m = ics.plummer(max(n, 2), 100 + k)
        p, v, m = p[:, :n].copy(), v[:, :n].copy(), m[:n].copy()
        p += np.array([[3.0 * k], [-1.0 * k], [0.5 * k]])
        if n == 1000:
            p[:, 10:30] = p[:, 10:11]  # 20 coincident bodies
        parts.append(p)
        vels.append(v)
        masses.append(m)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return (np.ascontiguousarray(np.concatenate(parts, axis=1)),
            np.ascontiguousarray(np.concatenate(vels, axis=1)),
            np.ascontiguousarray(np.concatenate(masses)), off)


FOREST = small_forest()


def systems(off):
    return [(int(off[k]), int(off[k + 1])) for k in range(len(off) - 1)]


def test_forest_keys_sorted_by_system_then_key():
    pos, _, mass, off = FOREST
    n = int(off[-1])
    with nb.Context.forest(off, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
        ctx.forest_forces(dev(pos), dev(mass))
        ctx.sync()
        keys, ids = ctx.keys(n)
    for lo, hi in systems(off):
        if hi == lo:
            continue
        ko, io = oracle.sort_pairs(oracle.keys(pos[:, lo:hi]))
        assert np.array_equal(ids[lo:hi], io + lo)
        assert np.array_equal(keys[lo:hi], ko)


def test_forest_fp64_forces_and_counters_bit_exact():
    pos, _, mass, off = FOREST
    n = int(off[-1])
    eps, theta = 0.01, 0.5
    with nb.Context.forest(off, 1.0, eps, theta, 1e-3, nb.FP64) as ctx:
        a = ctx.forest_forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.sync()
        pp, pc = ctx.counters(n)
    for lo, hi in systems(off):
        if hi == lo:
            continue
        ref, rpp, rpc = oracle.bh(pos[:, lo:hi], mass[lo:hi], 1.0, eps, theta)
        assert np.array_equal(a[:, lo:hi], ref), (lo, hi)
        assert np.array_equal(pp[lo:hi], rpp)
        assert np.array_equal(pc[lo:hi], rpc)


@pytest.mark.parametrize("prec", [nb.FP32, nb.FP32_KAHAN])
def test_forest_fp32_forces_within_tolerance(prec):
    pos, _, mass, off = FOREST
    n = int(off[-1])
    eps, theta = 0.01, 0.6
    with nb.Context.forest(off, 1.0, eps, theta, 1e-3, prec) as ctx:
        a = ctx.forest_forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.sync()
        pp, pc = ctx.counters(n)
    agree = []
    for lo, hi in systems(off):
        if hi - lo < 2:
            if hi - lo == 1:
                assert np.all(a[:, lo] == 0.0)
            continue
        ref, rpp, rpc = oracle.bh(pos[:, lo:hi], mass[lo:hi], 1.0, eps, theta)
        assert rel_rms(a[:, lo:hi], ref) <= FP32_TOL, (lo, hi)
        agree.append(np.mean((pp[lo:hi] == rpp) & (pc[lo:hi] == rpc)))
    assert min(agree) >= 0.99


def test_forest_fp64_leapfrog_bit_exact_and_graph_replay_identical():
    pos, vel, mass, off = FOREST
    eps, theta, dt, steps = 0.01, 0.5, 1e-3, 3
    # kernel by kernel
    tp, tv, tm = dev(pos), dev(vel), dev(mass)
    with nb.Context.forest(off, 1.0, eps, theta, dt, nb.FP64) as ctx:
        ctx.forest_step(tp, tv, tm, steps, use_graph=False)
        ctx.sync()
    # replayed graph (one capture, `steps` replays)
    gp, gv = dev(pos), dev(vel)
    with nb.Context.forest(off, 1.0, eps, theta, dt, nb.FP64) as ctx:
        ctx.forest_step(gp, gv, tm, steps, use_graph=True)
        ctx.sync()
    assert torch.equal(tp, gp) and torch.equal(tv, gv)
    p, v = tp.cpu().numpy(), tv.cpu().numpy()
    for lo, hi in systems(off):
        if hi == lo:
            continue
        a0, _, _ = oracle.bh(pos[:, lo:hi], mass[lo:hi], 1.0, eps, theta)
        rp, rv, _ = oracle.kdk(pos[:, lo:hi], vel[:, lo:hi], mass[lo:hi], a0, 1.0, eps, theta,
                               dt, steps)
        assert np.array_equal(p[:, lo:hi], rp), (lo, hi)
        assert np.array_equal(v[:, lo:hi], rv), (lo, hi)


@pytest.mark.parametrize("prec", [nb.FP32_KAHAN])
def test_forest_fp32_graph_replay_identical_to_launches(prec):
    pos, vel, mass, off = ics.forest(24, 11, 256, 4096)
    tp, tv, tm = dev(pos), dev(vel), dev(mass)
    gp, gv = dev(pos), dev(vel)
    with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, prec) as ctx:
        ctx.forest_step(tp, tv, tm, 4, use_graph=False)
        ctx.sync()
    with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, prec) as ctx:
        ctx.forest_step(gp, gv, tm, 2, use_graph=True)
        ctx.forest_step(gp, gv, tm, 2, use_graph=True)   # replays the same graph
        ctx.sync()
    assert torch.equal(tp, gp) and torch.equal(tv, gv)


def test_forest_matches_single_system_contexts():
    """A forest of one system is that system: FP64 forces equal nbody_forces bit for bit."""
    pos, _, mass = ics.plummer(3000, 31)
    off = np.array([0, 3000], dtype=np.int64)
    with nb.Context.forest(off, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
        a = ctx.forest_forces(dev(pos), dev(mass)).cpu().numpy()
    with nb.Context(3000, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
        b = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
    assert np.array_equal(a, b)


def test_forest_rejects_single_system_calls():
    pos, _, mass, off = FOREST
    with nb.Context.forest(off, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
        with pytest.raises(nb.NBodyError):
            ctx.forces(dev(pos), dev(mass))


@pytest.mark.parametrize("prec", [nb.FP64, nb.FP32_KAHAN])
def test_forest_resort_steps_identical_to_full_sort(prec):
    """Re-sorting from the previous step's order (§4.4) inside a forest, launched and replayed
    from a graph, leaves the same states bit for bit as the full sort."""
    pos, vel, mass, off = ics.forest(24, 12, 256, 4096)
    n = int(off[-1])
    out = []
    for mode, graph in ((nb.SORT_FULL, False), (nb.SORT_RESORT, False), (nb.SORT_RESORT, True)):
        tp, tv, tm = dev(pos), dev(vel), dev(mass)
        with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, prec) as ctx:
            ctx.set_sort_mode(mode)
            ctx.forest_step(tp, tv, tm, 4, use_graph=graph)
            ctx.sync()
            path, _ = ctx.sort_stats()
            assert path == (0 if mode == nb.SORT_FULL else 1)
            out.append((tp.cpu().numpy(), tv.cpu().numpy(), ctx.keys(n)))
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])
        assert np.array_equal(o[2][0], out[0][2][0]) and np.array_equal(o[2][1], out[0][2][1])


def test_forest_resort_after_jumps_matches_oracle():
    """Second build of a forest after a tenth of every system's bodies jumped across their
    system: keys and order per system equal the oracle's, systems in order."""
    pos, _, mass, off = FOREST
    n = int(off[-1])
    rng = np.random.default_rng(5)
    p1 = pos.copy()
    for lo, hi in systems(off):
        if hi - lo > 2:
            sel = lo + rng.choice(hi - lo, max(1, (hi - lo) // 10), replace=False)
            c = pos[:, lo:hi].mean(axis=1, keepdims=True)
            p1[:, sel] = 2 * c - p1[:, sel]
    with nb.Context.forest(off, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
        ctx.set_sort_mode(nb.SORT_RESORT)
        ctx.forest_forces(dev(pos), dev(mass))
        ctx.forest_forces(dev(p1), dev(mass))
        ctx.sync()
        assert ctx.sort_stats()[0] == 1
        keys, ids = ctx.keys(n)
    for lo, hi in systems(off):
        if hi == lo:
            continue
        ko, io = oracle.sort_pairs(oracle.keys(p1[:, lo:hi]))
        assert np.array_equal(ids[lo:hi], io + lo)
        assert np.array_equal(keys[lo:hi], ko)
