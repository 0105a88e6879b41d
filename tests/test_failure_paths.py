"""Failure detection without a GPU fault: the walk's stack and step guards tripped through the
test-aid limits (nbody_set_walk_limits), the opt-in finite-input check (NBODY_FLAG_CHECK_FINITE),
and the context staying usable after each reported error (the error word is cleared once
nbody_sync has reported it).  The guards stop a walk before any further memory access; no
input here is malformed in a way the library does not check."""
import numpy as np
import pytest

import ics
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2203_08966_gb300 as nb  # noqa: E402

DEV = "cuda:0"
EINVAL, ESTACK = 1, 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_rms(a, ref):
    num = ((a - ref) ** 2).sum(axis=0)
    den = (ref ** 2).sum(axis=0)
    return float(np.sqrt(np.mean(num / den)))


def _expect(status, fn):
    with pytest.raises(nb.NBodyError) as ei:
        fn()
    assert ei.value.status == status


@pytest.mark.parametrize("prec", [nb.FP32, nb.FP32_KAHAN])
@pytest.mark.parametrize("limits", [(40, 0), (0, 3)])
def test_fp32_walk_limits_report_estack_then_recover(prec, limits):
    pos, _, mass = ics.plummer(4096, 1)
    ref, _, _ = oracle.bh(pos, mass, 1.0, 0.01, 0.5)
    tp, tm = dev(pos), dev(mass)
    with nb.Context(4096, 1.0, 0.01, 0.5, 1e-3, prec) as ctx:
        ctx.set_walk_limits(*limits)
        ctx.forces(tp, tm)
        _expect(ESTACK, ctx.sync)
        ctx.sync()                      # reported once: the word was cleared
        ctx.set_walk_limits(0, 0)
        a = ctx.forces(tp, tm).cpu().numpy()
        ctx.sync()
    assert rel_rms(a, ref) <= 1e-4


def test_fp64_walk_step_limit_reports_estack_then_recovers():
    pos, _, mass = ics.plummer(2000, 3)
    ref, rpp, rpc = oracle.bh(pos, mass, 1.0, 0.01, 0.5)
    tp, tm = dev(pos), dev(mass)
    with nb.Context(2000, 1.0, 0.01, 0.5, 1e-3, nb.FP64) as ctx:
        ctx.set_walk_limits(0, 5)
        ctx.forces(tp, tm)
        _expect(ESTACK, ctx.sync)
        ctx.set_walk_limits(0, 0)
        a = ctx.forces(tp, tm).cpu().numpy()
        ctx.sync()
        pp, pc = ctx.counters(2000)
    assert np.array_equal(a, ref) and np.array_equal(pp, rpp) and np.array_equal(pc, rpc)


def test_walk_limits_reject_bad_arguments():
    with nb.Context(16) as ctx:
        for bad in ((1, 0, 0), (32, 0, 0), (0, -1, 0), (0, 0, 63), (0, 0, 1)):
            _expect(EINVAL, lambda: ctx.set_walk_limits(*bad))


@pytest.mark.parametrize("prec", [nb.FP32, nb.FP32_KAHAN])
def test_stack_overflow_walk_keeps_the_lists(prec):
    """The per-body walk's fast kernel gets a stack of 64 ranges instead of 256, so that deep
    groups (theta 0.3) are handed to the full-stack walk: every body keeps its interaction list
    (identical counters); those groups' sums are taken in another order (rounding only)."""
    pos, _, mass = ics.two_plummer(60000, seeds=(4, 5))
    n = mass.shape[0]
    out = []
    for shared in (0, 64):
        with nb.Context(n, 1.0, 0.002, 0.3, 1e-3, prec) as ctx:
            for shape in (1, 6):
                ctx.set_walk_shape(shape)
                ctx.set_walk_limits(0, 0, shared)
                a = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
                ctx.sync()
                out.append((shared, shape, a, *ctx.counters(n)))
    for s0, sh0, a0, pp0, pc0 in out[:2]:
        for s1, sh1, a1, pp1, pc1 in out[2:]:
            if sh1 == sh0:
                assert np.array_equal(pp0, pp1) and np.array_equal(pc0, pc1)
                assert np.sqrt(((a0 - a1) ** 2).sum() / (a0 ** 2).sum()) <= 1e-6


@pytest.mark.parametrize("prec", [nb.FP64, nb.FP32_KAHAN])
@pytest.mark.parametrize("what", ["nan_position", "inf_position", "nan_mass"])
def test_check_finite_rejects_bad_inputs(prec, what):
    pos, vel, mass = ics.plummer(3000, 5)
    bad_pos, bad_mass = pos.copy(), mass.copy()
    if what == "nan_position":
        bad_pos[1, 1234] = np.nan
    elif what == "inf_position":
        bad_pos[2, 7] = -np.inf
    else:
        bad_mass[2999] = np.nan
    flags = nb.FLAG_CHECK_FINITE
    with nb.Context(3000, 1.0, 0.01, 0.5, 1e-3, prec, flags=flags) as ctx:
        _expect(EINVAL, lambda: ctx.forces(dev(bad_pos), dev(bad_mass)))
        _expect(EINVAL, lambda: ctx.build_tree(dev(bad_pos), dev(bad_mass)))
        _expect(EINVAL, lambda: ctx.step(dev(bad_pos), dev(vel), dev(bad_mass), 1))
        # the same context then works on finite inputs, with the check on
        a = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.sync()
    ref, _, _ = oracle.bh(pos, mass, 1.0, 0.01, 0.5)
    assert rel_rms(a, ref) <= (0.0 if prec == nb.FP64 else 1e-4)


def test_check_finite_forest_reports_at_sync():
    sizes = [500, 1000, 33]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    parts = [ics.plummer(s, 30 + k) for k, s in enumerate(sizes)]
    pos = np.concatenate([p[0] for p in parts], axis=1)
    vel = np.concatenate([p[1] for p in parts], axis=1)
    mass = np.concatenate([p[2] for p in parts])
    bad = pos.copy()
    bad[0, 700] = np.inf                  # in the second system
    with nb.Context.forest(off, 1.0, 0.01, 0.5, 1e-3, nb.FP32_KAHAN,
                           flags=nb.FLAG_CHECK_FINITE) as ctx:
        ctx.forest_forces(dev(bad), dev(mass))
        _expect(EINVAL, ctx.sync)
        tp, tv = dev(pos), dev(vel)
        ctx.forest_step(tp, tv, dev(mass), 2)
        ctx.sync()                        # finite inputs: nothing reported
    assert np.isfinite(tp.cpu().numpy()).all()
