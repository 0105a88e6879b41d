"""Launch shapes of the walk: every shape gives every body the same interaction list (identical
counters); FP64 forces are bit-identical in every shape, FP32 forces bit-identical across the
warps-per-block shapes (0..2) and equal to rounding across the shapes that group or buffer the
terms differently (3..7).  The autotuner keeps the fastest shape it measured."""
import numpy as np
import pytest

import ics

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


@pytest.mark.parametrize("prec", [nb.FP64, nb.FP32, nb.FP32_KAHAN])
def test_every_walk_shape_gives_identical_forces_and_counters(prec):
    pos, _, mass = ics.two_plummer(20000, seeds=(4, 5))
    n = mass.shape[0]
    out = []
    with nb.Context(n, 1.0, 0.01, 0.5, 1e-3, prec) as ctx:
        for k in range(nb.WALK_SHAPES):
            ctx.set_walk_shape(k)
            assert ctx.walk_shape()[0] == k
            a = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
            ctx.sync()
            out.append((a, *ctx.counters(n)))
    for k, (a, pp, pc) in enumerate(out):
        assert np.array_equal(pp, out[0][1]) and np.array_equal(pc, out[0][2])
        if prec == nb.FP64 or k < 3:
            assert np.array_equal(a, out[0][0])
        else:
            ref = out[1][0]
            assert np.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum()) <= 1e-6


@pytest.mark.parametrize("prec", [nb.FP64, nb.FP32_KAHAN])
def test_autotune_keeps_the_fastest_shape(prec):
    pos, vel, mass = ics.plummer(30000, 9)
    with nb.Context(30000, 1.0, 0.01, 0.5, 1e-3, prec) as ctx:
        chosen, ms = ctx.autotune(dev(pos), dev(mass))
        assert 0 <= chosen < nb.WALK_SHAPES
        timed = [t for t in ms if t > 0]
        # FP64: the three thread counts; FP32: every shape
        assert len(timed) == (3 if prec == nb.FP64 else nb.WALK_SHAPES)
        assert ms[chosen] == min(timed)
        assert ctx.walk_shape()[0] == chosen
        # stepping after tuning still works (the kept acceleration is recomputed)
        tp, tv = dev(pos), dev(vel)
        ctx.step(tp, tv, dev(mass), 2)
        ctx.sync()
        assert torch.isfinite(tp).all()


def test_forest_autotune_and_graph_use_the_chosen_shape():
    pos, vel, mass, off = ics.forest(16, 12, 512, 4096)
    with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, nb.FP32_KAHAN) as ctx:
        chosen, ms = ctx.autotune(dev(pos), dev(mass))
        # forests: warps per block, buffer size, cell-following groups (no shared far walks)
        assert [k for k, t in enumerate(ms) if t > 0] == [0, 1, 2, 6, 7]
        assert ms[chosen] == min(t for t in ms if t > 0)
        tp, tv = dev(pos), dev(vel)
        ctx.forest_step(tp, tv, dev(mass), 2, use_graph=True)
        ctx.sync()
    ref_p, ref_v = dev(pos), dev(vel)
    with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, nb.FP32_KAHAN) as ctx:
        ctx.set_walk_shape(chosen)  # the same grouping and buffers: the same sums, bit for bit
        ctx.forest_step(ref_p, ref_v, dev(mass), 2, use_graph=False)
        ctx.sync()
    assert torch.equal(tp, ref_p) and torch.equal(tv, ref_v)


def test_autotune_choice_is_kept_per_size_bucket():
    """A tuned choice applies to its size bucket and theta; an explicit shape clears it."""
    pos, _, mass = ics.plummer(5000, 4)
    with nb.Context(5000, 1.0, 0.01, 0.5, 1e-3, nb.FP32_KAHAN) as ctx:
        chosen, _ = ctx.autotune(dev(pos), dev(mass))
        a1 = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.set_walk_shape(chosen)
        a2 = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.sync()
    assert np.array_equal(a1, a2)
