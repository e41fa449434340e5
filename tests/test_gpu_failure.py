"""Failure detection on the GPU, provoked without a fault: a bounded device wait that
runs out (SRMRA_ETIMEOUT), a non-finite log-likelihood (SRMRA_ENUMERIC), and contexts
created and driven from several host threads.

A timeout is provoked with the test hook of srmra_set_wait_limit: one epilogue waits
on a barrier that nothing completes, so its wait runs out after the context's (short)
limit; the kernel then takes its ordinary abort path (drains its own copies and MMAs,
releases TMEM) and sets the status word.  Each test checks that the call reports the
error, that the GPU still answers, and that the same context then computes a correct
iteration (checked against the FP64 oracle) once its state is reset."""
import os
import threading
import time

import numpy as np
import pytest

from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def S():
    from paper_2204_04754_gb300 import srmra
    if not os.path.exists(srmra.LIB_PATH):
        from paper_2204_04754_gb300 import build
        build.build()
    srmra.lib()
    return srmra


def oracle_step_ok(s, p, x, r1, r2, tol):
    """One iteration of `s` from (x, r1, r2) against the dense oracle."""
    s.set_state(x, r1, r2, 1.0, 0)
    ll = s.em_iter(1)[0]
    xg, r1g, r2g, _, _ = s.state()
    xo, r1o, r2o, llo, _ = O.em_iter(p.y, x, r1, r2, p.sigma, p.K)
    assert rel(xg, xo) < tol and rel(r1g, r1o) < tol and rel(r2g, r2o) < tol
    assert abs(ll - llo) < tol * abs(llo)


# (L, K, N, sigma, flags, pass-2 form): the ring cluster form (4 chunks, clusters of 4),
# the interleaved cluster form (9 chunks, one cluster of 9), the per-chunk kernel and
# its compensated M-step, the pair form (4 pairs, clusters of 8) (flags: 8 keeps single
# fp16 M-step operands, 2 turns the clusters off, 4 forces the compensated M-step, 32
# asks for the pair form)
CASES = [(64, 2, 700, 0.3, 8, "ring"), (96, 2, 1000, 0.5, 8, "interleaved"),
         (64, 2, 700, 0.3, 2 | 8, "per_chunk"), (64, 2, 700, 0.3, 4, "per_chunk_comp"),
         (64, 2, 700, 0.3, 32 | 8, "pair")]


@pytest.mark.parametrize("L,K,N,sigma,flags,form", CASES)
def test_pass1_wait_runs_out(S, L, K, N, sigma, flags, form):
    """The pass-1 hook: ETIMEOUT within a second (20 ms limit), then the same context
    gives the oracle's iteration."""
    p = synth.make_problem(L, K, N, sigma, seed=synth.seed_for(3, 500 + L))
    s = S.Solver(p.L, p.K, p.sigma, p.y, prec="bf16x3", x0=p.x0, rho1=p.rho1_0,
                 rho2=p.rho2_0, flags=flags)
    assert s.plan()["p2_form"] == form
    x, r1, r2, _, _ = s.state()
    s.set_wait_limit(20_000_000, test_hook=1)
    t0 = time.perf_counter()
    with pytest.raises(S.SrmraError) as e:
        s.em_iter(1)
    el = time.perf_counter() - t0
    assert e.value.status == S.SRMRA_ETIMEOUT
    assert el < 1.0, el
    s.set_wait_limit(2_000_000_000, test_hook=0)
    oracle_step_ok(s, p, x, r1, r2, 1e-4)
    s.close()


@pytest.mark.parametrize("L,K,N,sigma,flags,form", CASES)
def test_pass2_wait_runs_out(S, L, K, N, sigma, flags, form):
    """The pass-2 hook: in a cluster form the first cluster's rank 0 never builds its
    first weight tile, so the peers' waits for it run out too, and each CTA drains its
    own copies before the cluster leaves (bounded by the fixed 2 s drain limit per
    outstanding slot).  ETIMEOUT, then a correct iteration on the same context."""
    p = synth.make_problem(L, K, N, sigma, seed=synth.seed_for(3, 600 + L))
    s = S.Solver(p.L, p.K, p.sigma, p.y, prec="bf16x3", x0=p.x0, rho1=p.rho1_0,
                 rho2=p.rho2_0, flags=flags)
    assert s.plan()["p2_form"] == form
    x, r1, r2, _, _ = s.state()
    s.set_wait_limit(20_000_000, test_hook=2)
    t0 = time.perf_counter()
    with pytest.raises(S.SrmraError) as e:
        s.em_iter(1)
    el = time.perf_counter() - t0
    print(form, "pass-2 timeout reported after", el, "s")
    assert e.value.status == S.SRMRA_ETIMEOUT
    assert el < 60.0, el
    s.set_wait_limit(2_000_000_000, test_hook=0)
    oracle_step_ok(s, p, x, r1, r2, 1e-4)
    s.close()
    # a fresh context on the same device is unaffected
    s2 = S.Solver(p.L, p.K, p.sigma, p.y, prec="bf16x3", x0=p.x0, rho1=p.rho1_0,
                  rho2=p.rho2_0, flags=flags)
    oracle_step_ok(s2, p, x, r1, r2, 1e-4)
    s2.close()


def test_wait_limit_arguments(S):
    p = synth.make_problem(16, 2, 100, 0.5, seed=5)
    s = S.Solver(p.L, p.K, p.sigma, p.y, prec="bf16x3")
    for lim, hook in [(999, 0), (60_000_000_001, 0), (1_000_000, 3), (1_000_000, -1)]:
        with pytest.raises(S.SrmraError) as e:
            s.set_wait_limit(lim, hook)
        assert e.value.status == S.SRMRA_EINVAL
    s.set_wait_limit(1_000_000, 0)   # a short limit that normal work never reaches
    s.em_iter(2)
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fft32"])
def test_non_finite_estimate_is_reported_then_cleared(S, prec):
    """With SRMRA_FLAG_CHECK_NUMERIC an iteration from an estimate holding a NaN pixel
    returns ENUMERIC; the status word is cleared by that report, so the next iteration
    from a finite estimate succeeds and matches the oracle."""
    p = synth.make_problem(16, 2, 300, 0.4, seed=synth.seed_for(1, 31))
    s = S.Solver(p.L, p.K, p.sigma, p.y, prec=prec, x0=p.x0, rho1=p.rho1_0,
                 rho2=p.rho2_0, flags=S.SRMRA_FLAG_CHECK_NUMERIC)
    x, r1, r2, _, _ = s.state()
    bad = x.copy()
    bad[3, 5] = np.nan
    s.set_state(bad, r1, r2, 1.0, 0)
    with pytest.raises(S.SrmraError) as e:
        s.em_iter(1, loglik=False)   # the flag alone makes the call read the status
    assert e.value.status == S.SRMRA_ENUMERIC
    oracle_step_ok(s, p, x, r1, r2, 1e-4 if prec == "bf16x3" else 1e-5)
    s.close()


def test_non_finite_observation_is_reported(S):
    """A NaN in y reaches every logit of its observation: ENUMERIC at the first
    iteration (float32 form)."""
    p = synth.make_problem(16, 2, 300, 0.4, seed=synth.seed_for(1, 32))
    y = p.y.copy()
    y[7, 2, 2] = np.nan
    s = S.Solver(p.L, p.K, p.sigma, y, prec="fp32", x0=p.x0, rho1=p.rho1_0,
                 rho2=p.rho2_0, flags=S.SRMRA_FLAG_CHECK_NUMERIC)
    with pytest.raises(S.SrmraError) as e:
        s.em_iter(1)
    assert e.value.status == S.SRMRA_ENUMERIC
    s.close()


def test_contexts_from_two_threads(S):
    """Kernel attributes and cluster-occupancy answers are cached per device under a
    lock: two threads that create and run contexts of every form at the same time get
    the same results as one thread alone."""
    p = synth.make_problem(64, 2, 600, 0.4, seed=synth.seed_for(3, 77))
    forms = ["bf16x3", "bf16", "fp32", "fft32"]

    def run(prec):
        s = S.Solver(p.L, p.K, p.sigma, p.y, prec=prec, x0=p.x0, rho1=p.rho1_0,
                     rho2=p.rho2_0)
        s.em_iter(2)
        out = s.state()[0]
        s.close()
        return out

    alone = {f: run(f) for f in forms}
    got = {}
    errs = []

    def worker(fs):
        try:
            for f in fs:
                got[(threading.get_ident(), f)] = run(f)
        except Exception as exc:  # reported below
            errs.append(exc)
    ts = [threading.Thread(target=worker, args=(forms,)),
          threading.Thread(target=worker, args=(forms[::-1],))]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not errs, errs
    assert len(got) == 2 * len(forms)
    for (tid, f), xg in got.items():
        assert np.array_equal(xg, alone[f]), f
