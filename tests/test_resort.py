"""Re-sort from the previous step's order (temporal coherence, §4.4) against the oracle.

Whatever order the last build left, the re-sort must give the stable sort by (key, index) bit for
bit: the oracle's sort of the current keys, and its insertion re-sort from the same starting
order.  Covered: several leapfrog steps (the case the method is for), orders far from sorted
(the repair of tile seams and the fall-back to the full sort), ties of equal keys, ragged sizes
around the 2048-position tiles, and one to three bodies.  Steps with the re-sort and with the
full sort must leave identical positions and velocities.
"""
import numpy as np
import pytest

import ics
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2203_08966_gb300 as nb  # noqa: E402

DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def assert_sorted_like_oracle(ctx, pos, prev=None):
    n = pos.shape[1]
    keys, ids = ctx.keys(n)
    ko, io = oracle.sort_pairs(oracle.keys(pos))
    assert np.array_equal(keys, ko)
    assert np.array_equal(ids.astype(np.int64), io)
    if prev is not None:  # the paper's route from the same starting order gives the same
        ki, ii, _ = oracle.resort_insertion(oracle.keys(pos), prev)
        assert np.array_equal(keys, ki) and np.array_equal(ids.astype(np.int64), ii)


def test_resort_across_leapfrog_steps():
    """Plummer sphere of 70,000 bodies (above the automatic threshold), 4 steps: from the second
    build on the re-sort runs, takes out a few per cent, and every order is the oracle's."""
    pos, vel, mass = ics.plummer(70000, 21)
    tp, tv, tm = dev(pos), dev(vel), dev(mass)
    with nb.Context(70000, 1.0, 0.005, 0.5, 5e-4, nb.FP32_KAHAN) as ctx:
        ctx.forces(tp, tm)
        assert ctx.sort_stats() == (0, -1)       # first build: nothing to start from
        for _ in range(4):
            _, prev = ctx.keys(70000)
            ctx.step(tp, tv, tm, 1)
            ctx.sync()
            path, removed = ctx.sort_stats()
            assert path == 1 and 0 < removed < 70000 // 10
            assert_sorted_like_oracle(ctx, tp.cpu().numpy(), prev.astype(np.int64))


@pytest.mark.parametrize("prec", [nb.FP64, nb.FP32_KAHAN])
def test_resort_steps_identical_to_full_sort(prec):
    pos, vel, mass = ics.two_plummer(80000, seeds=(4, 5))
    out = []
    for mode in (nb.SORT_AUTO, nb.SORT_FULL):
        tp, tv, tm = dev(pos), dev(vel), dev(mass)
        with nb.Context(80000, 1.0, 0.002, 0.5, 5e-4, prec) as ctx:
            ctx.set_sort_mode(mode)
            ctx.step(tp, tv, tm, 5)
            ctx.sync()
            assert ctx.sort_stats()[0] == (1 if mode == nb.SORT_AUTO else 0)
            out.append((tp.cpu().numpy(), tv.cpu().numpy(), ctx.keys(80000)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2][0], out[1][2][0]) and np.array_equal(out[0][2][1], out[1][2][1])


def _orders(n, rng):
    """Second position sets for a first build of a Plummer sphere: each makes the first build's
    order a different kind of wrong."""
    p0, _, _ = ics.plummer(n, 31)
    out = {}
    p = p0.copy()
    sel = rng.choice(n, n // 10, replace=False)
    p[:, sel] *= -1.0                          # a tenth of the bodies jump across the centre
    out["tenth_reflected"] = p
    p = p0.copy()
    blk = np.argsort(p0[0])[: n // 3]
    p[0, blk] += 3.0                           # a third of the bodies move as a block
    out["third_shifted"] = p
    p = p0.copy()
    p[:, ::7] = p0[:, 3:4]                     # a seventh of the bodies coincide: equal keys
    out["coincident"] = p
    out["unrelated"] = ics.uniform_cube(n, 32)[0]  # no relation to the first order at all
    _, order = oracle.sort_pairs(oracle.keys(p0))
    m = (n // 2) * 2
    p = p0.copy()
    p[:, order[0:m:2]], p[:, order[1:m:2]] = p0[:, order[1:m:2]], p0[:, order[0:m:2]]
    out["sorted_pairs_swapped"] = p            # every neighbour pair of the first order descends
    return p0, out


@pytest.mark.parametrize("n", [2048, 2049, 6143, 20000])
def test_resort_from_far_orders_matches_oracle(n):
    rng = np.random.default_rng(n)
    p0, cases = _orders(n, rng)
    mass = dev(np.full(n, 1.0 / n))
    for name, p in cases.items():
        with nb.Context(n, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
            ctx.set_sort_mode(nb.SORT_RESORT)
            ctx.build_tree(dev(p0), mass)
            _, prev = ctx.keys(n)
            ctx.build_tree(dev(p), mass)
            ctx.sync()
            path, removed = ctx.sort_stats()
            assert path in (0, 1) and 0 <= removed <= n, name
            assert_sorted_like_oracle(ctx, p, prev.astype(np.int64))


def test_auto_mode_falls_back_when_most_bodies_move():
    n = 70000
    p0, _, m = ics.plummer(n, 41)
    with nb.Context(n, 1.0, 0.01, 0.5, 1e-3, nb.FP32) as ctx:
        ctx.build_tree(dev(p0), dev(m))
        p1 = ics.uniform_cube(n, 42)[0]
        ctx.build_tree(dev(p1), dev(m))
        ctx.sync()
        path, removed = ctx.sort_stats()
        assert path == 0 and removed > n // 4
        assert_sorted_like_oracle(ctx, p1)


@pytest.mark.parametrize("n", [1, 2, 3, 33])
def test_resort_tiny(n):
    p0, _, m = ics.plummer(max(n, 2), 51)
    p0, m = p0[:, :n].copy(), m[:n].copy()
    p1 = p0[:, ::-1].copy()
    with nb.Context(n, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
        ctx.set_sort_mode(nb.SORT_RESORT)
        ctx.build_tree(dev(p0), dev(m))
        ctx.build_tree(dev(p1), dev(m))
        ctx.sync()
        assert ctx.sort_stats()[0] == 1
        assert_sorted_like_oracle(ctx, p1)


def test_sort_mode_rejects_unknown():
    with nb.Context(16, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
        with pytest.raises(nb.NBodyError):
            ctx.set_sort_mode(3)
        assert ctx.sort_stats() == (-1, -1)


@pytest.mark.parametrize("n", [2, 100, 2049])
def test_resort_small_systems_steps_identical_to_full_sort(n):
    """Forced re-sorts (every build re-sorts, whatever the size) over leapfrog steps of small
    systems leave the same FP64 states, bit for bit, as the full sort."""
    pos, vel, mass = ics.plummer(max(n, 2), 61)
    pos, vel, mass = pos[:, :n].copy(), vel[:, :n].copy(), mass[:n].copy()
    out = []
    for mode in (nb.SORT_RESORT, nb.SORT_FULL):
        tp, tv, tm = dev(pos), dev(vel), dev(mass)
        with nb.Context(n, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
            ctx.set_sort_mode(mode)
            ctx.step(tp, tv, tm, 5)
            ctx.sync()
            assert ctx.sort_stats()[0] == (1 if mode == nb.SORT_RESORT else 0)
            out.append((tp.cpu().numpy(), tv.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
