"""Batches (grouped launches + CUDA graph) against the same problems solved one by one
through the single-context path (itself parity-tested against the oracle)."""
import os

import numpy as np
import pytest

from oracle import srmra_oracle as O
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


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (64, 2, 700) and (96, 2, 400) take the compensated M-step (few observations for their
# l^2), (96, 2, 1600) nine pixel chunks in clusters of more than 4, (64, 2, 1200) the
# ring cluster form: one grouped pass-2 launch per kernel
SPECS = [(32, 2, 1500, 0.3), (48, 4, 900, 0.6), (64, 2, 700, 0.2), (32, 4, 2000, 1.0),
         (16, 2, 300, 0.1), (96, 2, 400, 0.5), (96, 2, 1600, 0.5), (64, 2, 1200, 0.3)]


def problems():
    return [synth.make_problem(L, K, N, s, seed=synth.seed_for(4, 50 + k), n_blobs=10)
            for k, (L, K, N, s) in enumerate(SPECS)]


def solver(S, p, prec):
    return S.Solver(p.L, p.K, p.sigma, p.y, prec=prec, x0=p.x0, rho1=p.rho1_0, rho2=p.rho2_0)


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_problems_solved_alone(S, prec, graph):
    probs = problems()
    alone = []
    for p in probs:
        s = solver(S, p, prec)
        s.solve(3, 1)
        alone.append(s.state())
        s.close()
    ss = [solver(S, p, prec) for p in probs]
    if prec == "bf16x3":  # the batch mixes the per-chunk, compensated and cluster forms
        forms = {s.plan()["p2_form"] for s in ss}
        assert {"per_chunk", "per_chunk_comp", "ring", "interleaved"} <= forms, forms
    b = S.Batch(ss, autotune=False, graph=graph)
    ll = b.solve(3, 1)
    for k, s in enumerate(ss):
        x, r1, r2, sbm, t = s.state()
        xa, r1a, r2a, sbma, ta = alone[k]
        # same work decomposition as alone: identical arithmetic, identical bits
        assert x.tobytes() == xa.tobytes() and r1.tobytes() == r1a.tobytes()
        assert t == ta == 3 and sbm == sbma
        assert np.isfinite(ll[k])
    b.close()
    for s in ss:
        s.close()


def test_autotuned_batch_matches_within_tolerance(S):
    probs = problems()
    ss = [solver(S, p, "bf16x3") for p in probs]
    b = S.Batch(ss, autotune=True)
    tun = b.tuning()
    assert tun["p1_scale"] in (1, 2) and tun["p2_scale"] in (1, 2) and tun["ms"] > 0
    assert tun["p1_shift_tile"] in (128, 256)
    print("autotuner", tun)
    b.solve(2, 1)
    for p, s in zip(probs, ss):
        a = solver(S, p, "bf16x3")
        a.solve(2, 1)
        xa = a.state()[0]
        a.close()
        assert rel(s.state()[0], xa) < 1e-5
    b.close()
    for s in ss:
        s.close()


def test_batched_step_against_oracle(S):
    """One batched plain-EM iteration of every problem against the FP64 oracle."""
    probs = problems()
    ss = [solver(S, p, "bf16x3") for p in probs]
    S.srmra_em_iter_batch([s.ctx for s in ss], 1)
    for p, s in zip(probs, ss):
        x, r1, r2, _, t = s.state()
        xo, r1o, r2o, _, _ = O.em_iter(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
        assert t == 1 and rel(x, xo) < 1e-4 and rel(r1, r1o) < 1e-4
        s.close()


def test_batch_pass1_tile_widths(S):
    """Contexts with different pass-1 tile widths (SRMRA_FLAG_P1_TILE128) form a batch
    only with the autotuner, which gives them one width; srmra_batch_tiles reports it."""
    probs = problems()[:3]
    ss = [S.Solver(p.L, p.K, p.sigma, p.y, prec="bf16x3", x0=p.x0, rho1=p.rho1_0,
                   rho2=p.rho2_0, flags=16 if k == 1 else 0) for k, p in enumerate(probs)]
    assert [s.plan()["p1_shift_tile"] for s in ss] == [256, 128, 256]
    with pytest.raises(S.SrmraError) as e:
        S.Batch(ss, autotune=False)
    assert e.value.status == S.SRMRA_EINVAL
    b = S.Batch(ss, autotune=True)
    w = b.tuning()["p1_shift_tile"]
    assert w in (128, 256) and all(s.plan()["p1_shift_tile"] == w for s in ss)
    b.solve(1, 1)
    b.close()
    for s in ss:
        s.close()


def test_batch_with_pair_form_contexts(S):
    """Contexts that ask for the pair form of pass 2 (SRMRA_FLAG_P2_PAIR; it applies to
    bf16x3 problems of up to four pixel chunks without the compensated M-step) batched
    with contexts of the other forms: one grouped launch per form, results identical to
    solving each alone."""
    probs = problems()

    def mk(p):
        return S.Solver(p.L, p.K, p.sigma, p.y, prec="bf16x3", x0=p.x0, rho1=p.rho1_0,
                        rho2=p.rho2_0, flags=S.SRMRA_FLAG_P2_PAIR)
    alone = []
    for p in probs:
        s = mk(p)
        s.solve(3, 1)
        alone.append(s.state())
        s.close()
    ss = [mk(p) for p in probs]
    forms = [s.plan()["p2_form"] for s in ss]
    assert forms.count("pair") == 5 and "interleaved" in forms, forms
    b = S.Batch(ss, autotune=False)
    b.solve(3, 1)
    for k, s in enumerate(ss):
        x, r1, _, _, t = s.state()
        assert x.tobytes() == alone[k][0].tobytes() and r1.tobytes() == alone[k][1].tobytes()
        assert t == 3
    b.close()
    for s in ss:
        s.close()
    # with the autotuner (other observation-range splits for the pair-form launches too)
    ss = [mk(p) for p in probs]
    b = S.Batch(ss, autotune=True)
    b.solve(3, 1)
    for k, s in enumerate(ss):
        assert rel(s.state()[0], alone[k][0]) < 1e-5
    b.close()
    for s in ss:
        s.close()


def test_batch_rejects_mixed_precision_and_duplicates(S):
    probs = problems()[:2]
    a = solver(S, probs[0], "bf16x3")
    b = solver(S, probs[1], "fp32")
    with pytest.raises(S.SrmraError) as e:
        S.Batch([a, b])
    assert e.value.status == S.SRMRA_EINVAL
    with pytest.raises(S.SrmraError) as e:
        S.Batch([a, a])
    assert e.value.status == S.SRMRA_EINVAL
    a.close()
    b.close()
