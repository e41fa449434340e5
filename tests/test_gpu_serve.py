"""Serving: continuous batching with memory-based admission.  Each request's result is
the same alone (srmra_create + srmra_solve) and in the mix."""
import os

import numpy as np
import pytest

from paper_2204_04754_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2204_04754_gb300 import srmra
    if not os.path.exists(srmra.LIB_PATH):
        from paper_2204_04754_gb300 import build
        build.build()
    srmra.lib()
    return srmra


REQS = [(64, 2, 800, 0.3, 5), (32, 4, 1500, 0.6, 3), (48, 2, 600, 0.5, 4),
        (64, 4, 1000, 0.2, 6), (32, 2, 400, 1.0, 2), (96, 4, 500, 0.4, 3)]


def problems():
    return [synth.make_problem(L, K, N, s, seed=synth.seed_for(5, k), n_blobs=8)
            for k, (L, K, N, s, _) in enumerate(REQS)]


def form_of(prec, p):
    """The form a request of problem p runs in on a server of form prec ("auto": the
    polyphase-FFT form where L/K is 8, 16 or 32, else bf16x3)."""
    if prec != "auto":
        return prec
    return "fft32" if p.L // p.K in (8, 16, 32) else "bf16x3"


@pytest.mark.parametrize("prec", ["bf16x3", "fp32", "auto"])
def test_results_same_alone_and_in_the_mix(S, prec):
    """With "auto" the mix holds FFT-form and bf16x3 requests (two batches per step)."""
    probs = problems()
    iters = [r[4] for r in REQS]
    forms = [form_of(prec, p) for p in probs]
    if prec == "auto":
        assert {"fft32", "bf16x3"} <= set(forms), forms
    alone = []
    for p, it, f in zip(probs, iters, forms):
        s = S.Solver(p.L, p.K, p.sigma, p.y, prec=f)
        s.solve(it, 1)
        alone.append(s.state())
        s.close()
    need = [S.srmra_estimate_device_bytes(p.L, p.K, p.N, p.sigma, f)
            for p, f in zip(probs, forms)]
    # room for about three requests at once, and for every request on its own
    budget = max(sum(need[:3]), max(need))
    srv = S.Server(budget, max_active=4, prec=prec)
    # staggered arrivals: two now, the rest while those are running
    ids = [srv.submit(p.L, p.K, p.sigma, p.y, it) for p, it in zip(probs[:2], iters[:2])]
    steps = 0
    pending = list(zip(probs[2:], iters[2:]))
    max_running = 0
    while True:
        if pending and steps % 2 == 1:
            p, it = pending.pop(0)
            ids.append(srv.submit(p.L, p.K, p.sigma, p.y, it))
        running, queued, _ = srv.step()
        max_running = max(max_running, running)
        used, bud = srv.memory()
        assert used <= bud
        steps += 1
        if not pending and running == 0 and queued == 0:
            break
        assert steps < 200
    assert max_running >= 2  # requests overlapped on the device
    for k, (p, rid) in enumerate(zip(probs, ids)):
        r = srv.result(rid, p.L)
        assert r["state"] == 2 and r["latency_ms"] > 0
        xa, r1a, r2a, _, _ = alone[k]
        assert r["x"].tobytes() == xa.tobytes()
        assert r["rho1"].tobytes() == r1a.tobytes() and r["rho2"].tobytes() == r2a.tobytes()
    srv.close()


def test_admission_respects_budget_and_slots(S):
    probs = [synth.make_problem(32, 2, 700, 0.4, seed=synth.seed_for(5, 60 + k)) for k in range(3)]
    need = [S.srmra_estimate_device_bytes(p.L, p.K, p.N, p.sigma, "bf16x3") for p in probs]
    assert len(set(need)) == 1
    srv = S.Server(need[0] + 1, max_active=8, prec="bf16x3")  # room for one at a time
    ids = [srv.submit(p.L, p.K, p.sigma, p.y, 2) for p in probs]
    seen = []
    while True:
        running, queued, _ = srv.step()
        seen.append(running)
        if running == 0 and queued == 0:
            break
    assert max(seen) == 1
    for p, rid in zip(probs, ids):
        assert srv.result(rid, p.L)["state"] == 2
    # slots: a generous budget but one slot
    srv2 = S.Server(100 * need[0], max_active=1, prec="bf16x3")
    for p in probs:
        srv2.submit(p.L, p.K, p.sigma, p.y, 2)
    seen = []
    while True:
        running, queued, _ = srv2.step()
        seen.append(running)
        if running == 0 and queued == 0:
            break
    assert max(seen) == 1
    srv2.close()
    with pytest.raises(S.SrmraError) as e:
        srv.submit(128, 2, 0.3, np.zeros((200000, 64, 64), np.float32), 2)
    assert e.value.status == S.SRMRA_ENOMEM
    srv.close()
