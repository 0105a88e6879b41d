"""The grouped acceptance test (NBODY_FLAG_GROUP_MAC; Barnes 1990, not in the paper) against the
oracle's group walk: FP32 forces within a relative RMS of 1e-4, counters equal for >= 99% of
bodies (FP32 and FP64 can break exact ties of the test differently).  Independently of the
oracle: each body's group list refines its per-body list, so no body has fewer interactions
than under the per-body test (exact: both tests use the same monotone FP32 expression)."""
import numpy as np
import pytest

import ics
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2203_08966_gb300 as nb  # noqa: E402

DEV = "cuda:0"
TOL = 1e-4


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_rms(a, ref):
    num = ((a - ref) ** 2).sum(axis=0)
    den = (ref ** 2).sum(axis=0)
    ok = den > 0
    return float(np.sqrt(np.mean(num[ok] / den[ok])))


def rel_global(a, ref):
    return float(np.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum()))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


CASES = {
    "plummer_4096": ics.plummer(4096, 1),
    "two_plummer_20000": ics.two_plummer(20000, seeds=(4, 5)),
    "uniform_1000": ics.uniform_cube(1000, 2),
}


@pytest.mark.parametrize("prec", [nb.FP32, nb.FP32_KAHAN])
@pytest.mark.parametrize("theta", [0.5, 0.8])
@pytest.mark.parametrize("name", sorted(CASES))
def test_group_mac_matches_oracle_group_walk(name, theta, prec):
    pos, _, mass = CASES[name]
    n = mass.shape[0]
    eps = 0.01
    ref, rpp, rpc = oracle.bh_group(pos, mass, 1.0, eps, theta, group=32)
    with nb.Context(n, 1.0, eps, theta, 1e-3, prec, flags=nb.FLAG_GROUP_MAC) as ctx:
        a = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.sync()
        pp, pc = ctx.counters(n)
    assert rel_rms(a, ref) <= TOL
    assert np.mean((pp == rpp) & (pc == rpc)) >= 0.99


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
def test_group_lists_refine_per_body_lists_on_gpu(theta):
    pos, _, mass = ics.plummer(30000, 17)
    n = mass.shape[0]
    with nb.Context(n, 1.0, 0.005, theta, 1e-3, nb.FP32_KAHAN) as ctx:
        a_body = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        bp, bc = ctx.counters(n)
        ctx.set_params(flags=nb.FLAG_GROUP_MAC)
        a_grp = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        gp, gc = ctx.counters(n)
    assert np.all(gp.astype(np.int64) + gc >= bp.astype(np.int64) + bc)
    d = oracle.direct(pos, mass, 1.0, 0.005, targets=np.arange(0, n, 15))
    assert rel_global(a_grp[:, ::15], d) <= rel_global(a_body[:, ::15], d)


def test_group_mac_theta_zero_is_direct_sum():
    pos, _, mass = ics.plummer(3000, 12)
    with nb.Context(3000, 1.0, 0.01, 0.0, 1e-3, nb.FP32_KAHAN, flags=nb.FLAG_GROUP_MAC) as ctx:
        a = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        pp, pc = ctx.counters(3000)
    d = oracle.direct(pos, mass, 1.0, 0.01)
    assert rel_rms(a, d) <= 1e-5
    assert np.all(pp == 2999) and np.all(pc == 0)


def test_group_mac_forest_per_system():
    pos, vel, mass, off = ics.forest(8, 21, 100, 3000)
    with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, nb.FP32_KAHAN,
                           flags=nb.FLAG_GROUP_MAC) as ctx:
        a = ctx.forest_forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.sync()
    for k in range(len(off) - 1):
        lo, hi = int(off[k]), int(off[k + 1])
        ref, _, _ = oracle.bh_group(pos[:, lo:hi], mass[lo:hi], 1.0, 0.01, 0.6, group=32)
        assert rel_rms(a[:, lo:hi], ref) <= TOL, k


def _bucket_case():
    p, v, m = ics.plummer(3000, 7)
    p[:, 100:140] = p[:, 100:101]          # 40 coincident bodies: a bucket larger than a group
    return p, m


@pytest.mark.parametrize("name", ["plummer_4096", "two_plummer_20000", "bucket_40"])
def test_cell_groups_keep_every_interaction_list(name):
    """Grouping by cells changes which bodies share a warp, never a body's list: counters are
    identical to the chunked grouping and forces agree to rounding."""
    if name == "bucket_40":
        pos, mass = _bucket_case()
    else:
        pos, _, mass = CASES[name]
    n = mass.shape[0]
    with nb.Context(n, 1.0, 0.01, 0.6, 1e-3, nb.FP32_KAHAN) as ctx:
        a0 = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        pp0, pc0 = ctx.counters(n)
        ctx.set_params(flags=nb.FLAG_CELL_GROUPS)
        a1 = ctx.forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.sync()
        pp1, pc1 = ctx.counters(n)
    assert np.array_equal(pp0, pp1) and np.array_equal(pc0, pc1)
    assert rel_rms(a1, a0) <= 1e-6


def test_cell_groups_forest_and_graph():
    pos, vel, mass, off = ics.forest(12, 23, 50, 5000)
    n = int(off[-1])
    with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, nb.FP32_KAHAN) as ctx:
        a0 = ctx.forest_forces(dev(pos), dev(mass)).cpu().numpy()
        pp0, pc0 = ctx.counters(n)
    with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, nb.FP32_KAHAN,
                           flags=nb.FLAG_CELL_GROUPS) as ctx:
        a1 = ctx.forest_forces(dev(pos), dev(mass)).cpu().numpy()
        ctx.sync()
        pp1, pc1 = ctx.counters(n)
        tp, tv, tm = dev(pos), dev(vel), dev(mass)
        ctx.forest_step(tp, tv, tm, 2, use_graph=True)
        ctx.sync()
    assert np.array_equal(pp0, pp1) and np.array_equal(pc0, pc1)
    assert rel_rms(a1, a0) <= 1e-6
    rp, rv = dev(pos), dev(vel)
    with nb.Context.forest(off, 1.0, 0.01, 0.6, 1e-3, nb.FP32_KAHAN,
                           flags=nb.FLAG_CELL_GROUPS) as ctx:
        ctx.forest_step(rp, rv, tm, 2, use_graph=False)
        ctx.sync()
    assert torch.equal(tp, rp) and torch.equal(tv, rv)
