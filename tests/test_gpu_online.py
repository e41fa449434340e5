"""Online (mini-batch) EM on the GPU (srmra_online_*) against the FP64 oracle's
online_em: the same shards, order and step sizes; x, rho and the batch log-likelihoods
step by step within the float32 tolerance (1e-5 relative); one shard of all
observations with gamma = 1 against a plain EM iteration; the projection; argument
errors."""
import numpy as np
import pytest

from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth
from tests import test_gpu_parity as P

pytestmark = pytest.mark.gpu

S = P.S  # module fixture

CUTS = [0, 200, 450, 600]  # three ragged shards
ORDER = [0, 1, 2, 0, 1, 2]
GAMMAS = [1.0, 0.7, 0.55, 0.45, 0.4, 0.35]


def shard_solvers(S, p, prec):
    return [S.Solver(p.L, p.K, p.sigma, p.y[a:b], prec=prec, x0=p.x0, rho1=p.rho1_0,
                     rho2=p.rho2_0) for a, b in zip(CUTS[:-1], CUTS[1:])]


@pytest.mark.parametrize("prec,L,K,sigma", [("fp32", 16, 2, 0.5), ("fp32", 24, 3, 0.6),
                                            ("fft32", 32, 2, 0.5), ("fft32", 16, 2, 0.5)])
def test_online_steps_match_oracle(S, prec, L, K, sigma):
    p = synth.make_problem(L, K, CUTS[-1], sigma, seed=synth.seed_for(11, L + K))
    shards = shard_solvers(S, p, prec)
    on = S.Online(shards, x0=p.x0, rho1=p.rho1_0, rho2=p.rho2_0)
    batches = [slice(CUTS[k], CUTS[k + 1]) for k in ORDER]
    for t in range(len(ORDER)):
        ll = on.step(ORDER[t], GAMMAS[t])
        x, r1, r2, n = on.state()
        xo, r1o, r2o, llo = O.online_em(p.y, batches[:t + 1], GAMMAS[:t + 1], p.x0, p.rho1_0,
                                        p.rho2_0, p.sigma, p.K)
        assert n == t + 1
        assert P.rel(x, xo) < 1e-5, (t, P.rel(x, xo))
        assert P.rel(r1, r1o) < 1e-5 and P.rel(r2, r2o) < 1e-5, t
        yb = p.y[batches[t]].astype(np.float64)
        scale = (yb ** 2).sum() / (2 * p.sigma ** 2)
        assert abs(ll - llo[-1]) / (abs(llo[-1]) + scale) < 1e-5, t
    on.close()
    for s in shards:
        s.close()


def test_one_full_shard_is_one_em_iteration(S):
    p = synth.make_problem(32, 2, 700, 0.4, seed=synth.seed_for(11, 3))
    a = P.make_solver(S, p)
    ll_a = a.em_iter(1)[0]
    xa, r1a, r2a, _, _ = a.state()
    a.close()
    b = P.make_solver(S, p)
    on = S.Online([b], x0=p.x0, rho1=p.rho1_0, rho2=p.rho2_0)
    ll_b = on.step(0, 1.0)
    xb, r1b, r2b, _ = on.state()
    assert P.rel(xb, xa) < 1e-6 and P.rel(r1b, r1a) < 1e-12 + 1e-6 and P.rel(r2b, r2a) < 1e-6
    assert ll_b == ll_a
    on.close()
    b.close()


def test_online_projection(S):
    p = synth.make_problem(32, 2, 600, 0.5, seed=synth.seed_for(11, 4))
    shards = shard_solvers(S, p, "fp32")
    on = S.Online(shards)
    on.step(0, 1.0)
    x, _, _, _ = on.state()
    on.project(0.5)
    xd, _, _, _ = on.state()
    xo, margin = O.dct_denoise(x, 0.5)
    assert margin > 1e-6
    assert P.rel(xd, xo) < 1e-6
    on.close()
    for s in shards:
        s.close()


def test_online_argument_errors(S):
    p = synth.make_problem(16, 2, 100, 0.5, seed=5)
    a = S.Solver(p.L, p.K, p.sigma, p.y, prec="fp32")
    b = S.Solver(p.L, p.K, 0.7, p.y, prec="fp32")
    with pytest.raises(S.SrmraError) as e:
        S.Online([a, b])
    assert "EINVAL" in str(e.value)
    on = S.Online([a])
    for g in (0.0, 1.5):
        with pytest.raises(S.SrmraError):
            on.step(0, g)
    with pytest.raises(S.SrmraError):
        on.step(3, 0.5)
    on.close()
    a.close()
    b.close()
