"""Energy and momentum drift of the GPU forms (§2.3 energy, §2.4 leapfrog) on the 4096-body
Plummer configuration (eps 0.01, theta 0.5, dt 1e-3, 10 steps): the energy of the GPU states,
computed by the oracle, drifts like the oracle's own Barnes-Hut run, within 10% of its relative
drift or 1e-8 (the KDK pin for GPU forms whose forces differ from the oracle by rounding)."""
import numpy as np
import pytest

import ics
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2203_08966_gb300 as nb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def reference():
    w = ics.WORKLOADS["plummer_4k"]
    pos, vel, mass = ics.plummer(w["n"], w["seed"])
    acc0, _, _ = oracle.bh(pos, mass, 1.0, w["eps"], w["theta"])
    rp, rv, _ = oracle.kdk(pos, vel, mass, acc0, 1.0, w["eps"], w["theta"], w["dt"], w["steps"])
    e0 = oracle.energy(pos, vel, mass, 1.0, w["eps"])[2]
    e1 = oracle.energy(rp, rv, mass, 1.0, w["eps"])[2]
    dp = oracle.momentum(rv, mass) - oracle.momentum(vel, mass)
    return w, (pos, vel, mass), e0, (e1 - e0) / abs(e0), dp


@pytest.mark.parametrize("prec", [nb.FP32, nb.FP32_KAHAN, nb.FP64_FAST, nb.FP64])
def test_energy_drift_matches_the_oracle(reference, prec):
    w, (pos, vel, mass), e0, drift_ref, dp_ref = reference
    tp = torch.from_numpy(pos).cuda()
    tv = torch.from_numpy(vel).cuda()
    with nb.Context(w["n"], 1.0, w["eps"], w["theta"], w["dt"], prec) as ctx:
        ctx.step(tp, tv, torch.from_numpy(mass).cuda(), w["steps"])
        ctx.sync()
    p, v = tp.cpu().numpy(), tv.cpu().numpy()
    drift = (oracle.energy(p, v, mass, 1.0, w["eps"])[2] - e0) / abs(e0)
    assert abs(drift - drift_ref) <= max(0.1 * abs(drift_ref), 1e-8), (drift, drift_ref)
    dp = oracle.momentum(v, mass) - oracle.momentum(vel, mass)
    assert np.linalg.norm(dp - dp_ref) <= max(0.1 * np.linalg.norm(dp_ref), 1e-10)
