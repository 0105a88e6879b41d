"""GPU parity at full size: the 1,048,576-body Plummer sphere and the 16,777,216-body pair of
colliding Plummer spheres in the benchmark's launch configuration (FP32 forces with compensated
accumulation, theta = 0.5, eps = 0.002).  Keys, sort order and tree topology are compared in
full; forces on seeded samples of targets that the oracle walks one by one in its own tree."""
import numpy as np
import pytest

import ics
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2203_08966_gb300 as nb  # noqa: E402

DEV = "cuda:0"


def rel_rms(a, ref):
    num = ((a - ref) ** 2).sum(axis=0)
    den = (ref ** 2).sum(axis=0)
    return float(np.sqrt(np.mean(num / den)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    oracle.set_threads(16)


def _check_system(pos, mass, eps, theta, n_targets, seed, fp64_sample=True):
    n = mass.shape[0]
    tp = torch.from_numpy(pos).to(DEV)
    tm = torch.from_numpy(mass).to(DEV)
    tg = np.sort(np.random.default_rng(seed).choice(n, n_targets, replace=False)).astype(np.int64)
    t = oracle.Tree(pos, mass)
    ref, rpp, rpc = t.forces(1.0, eps, theta, targets=tg)
    with nb.Context(n, 1.0, eps, theta, 5e-4, nb.FP32_KAHAN) as ctx:
        a = ctx.forces(tp, tm)
        keys, ids = ctx.keys(n)
        rec = ctx.tree()
        a32 = a[:, torch.from_numpy(tg).to(DEV)].cpu().numpy()
        pp, pc = ctx.counters(n)
        ko, io = oracle.sort_pairs(oracle.keys(pos))
        assert np.array_equal(keys, ko)
        assert np.array_equal(ids.astype(np.int64), io)
        del ko, io
        assert np.array_equal(rec, t.records())
        err32 = rel_rms(a32, ref)
        assert err32 <= 1e-4
        assert np.mean((pp[tg] == rpp) & (pc[tg] == rpc)) >= 0.99
        if fp64_sample:
            ctx.set_params(precision=nb.FP64)
            a64 = ctx.forces(tp, tm)[:, torch.from_numpy(tg).to(DEV)].cpu().numpy()
            pp, pc = ctx.counters(n)
            assert np.array_equal(a64, ref)
            assert np.array_equal(pp[tg], rpp) and np.array_equal(pc[tg], rpc)
    t.close()
    return err32


def test_plummer_1m():
    w = ics.WORKLOADS["plummer_1m"]
    pos, _, mass = ics.plummer(w["n"], w["seed"])
    err = _check_system(pos, mass, w["eps"], w["theta"], 4096, 3)
    print(f"plummer_1m FP32-Kahan rel. RMS vs oracle BH: {err:.2e}")


def test_two_plummer_16m_bench_configuration():
    w = ics.WORKLOADS["two_plummer_16m"]
    pos, _, mass = ics.two_plummer(w["n"], seeds=w["seeds"])
    err = _check_system(pos, mass, w["eps"], w["theta"], 2048, 9, fp64_sample=False)
    print(f"two_plummer_16m FP32-Kahan rel. RMS vs oracle BH: {err:.2e}")


def test_two_plummer_16m_resort_after_steps():
    """Two leapfrog steps of the benchmark configuration: every build after the first re-sorts
    from the previous build's order (§4.4); the order after the steps is the oracle's sort of the
    new positions, key for key and index for index."""
    w = ics.WORKLOADS["two_plummer_16m"]
    pos, vel, mass = ics.two_plummer(w["n"], seeds=w["seeds"])
    n = mass.shape[0]
    tp, tv, tm = (torch.from_numpy(a).to(DEV) for a in (pos, vel, mass))
    with nb.Context(n, 1.0, w["eps"], w["theta"], w["dt"], nb.FP32_KAHAN) as ctx:
        ctx.step(tp, tv, tm, 2)
        ctx.sync()
        path, removed = ctx.sort_stats()
        assert path == 1 and 0 < removed < n // 10
        keys, ids = ctx.keys(n)
    ko, io = oracle.sort_pairs(oracle.keys(tp.cpu().numpy()))
    assert np.array_equal(keys, ko)
    assert np.array_equal(ids.astype(np.int64), io)


def test_disk_bulge_64m_deep_tree():
    """The deep, imbalanced stress case: exponential disk + Hernquist bulge, N = 67,108,864,
    eps = 0.001, theta = 0.5 (keys, order and tree in full; FP32-Kahan forces on sampled
    targets)."""
    w = ics.WORKLOADS["disk_bulge_64m"]
    pos, _, mass = ics.disk_bulge(w["n"], w["seed"])
    err = _check_system(pos, mass, w["eps"], w["theta"], 1024, 13, fp64_sample=False)
    print(f"disk_bulge_64m FP32-Kahan rel. RMS vs oracle BH: {err:.2e}")
