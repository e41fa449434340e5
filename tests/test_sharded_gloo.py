"""The sharded EM driver (paper_2204_04754_gb300/sharded.py) over two gloo ranks on the
CPU.  Each rank's solver is a stand-in that runs the FP64 oracle's E-step on its shard
and the oracle's M-step from summed statistics; the driver's all-reduce and the order of
its steps must give the EM iterations of the whole data (Algorithm 2 with projection),
identical on both ranks.  The CUDA library's statistics vector is tested on the GPU in
tests/test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest

from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth

L, K, N, SIGMA = 8, 2, 70, 0.4
CUTS = [0, 31, 70]  # ragged shards
ITERS, F, SBM1 = 4, 2, 0.3


class OracleShard:
    """Solver stand-in: statistics [Z (L^2 x l^2) | c (L^2) | LL] of the shard."""

    def __init__(self, Y, x0, r1, r2):
        self.Y = np.asarray(Y, np.float64).reshape(Y.shape[0], -1)
        self.x, self.r1, self.r2 = np.asarray(x0, np.float64), np.array(r1), np.array(r2)
        self.t, self.F, self.sbm, self.decay = 0, 0, 1.0, 1.0

    def set_schedule(self, F, sigma_bm, decay=2.0 ** -0.1):
        """As the library: mstep_stats projects on this Algorithm 2 schedule."""
        self.F, self.sbm, self.decay = F, sigma_bm, decay

    def stats_length(self):
        return L * L * (L // K) ** 2 + L * L + 1

    def estep_stats(self, out=None):
        W, _, ll = O.estep(self.Y, self.x, self.r1, self.r2, SIGMA, K)
        return np.concatenate([(W.T @ self.Y).ravel(), W.sum(axis=0), [ll]])

    def mstep_stats(self, v, loglik=True):
        S, l2 = L * L, (L // K) ** 2
        Z = np.asarray(v[:S * l2]).reshape(S, l2)
        c = np.asarray(v[S * l2:S * l2 + S])
        self.x, self.r1, self.r2, _, _ = O.mstep_from_sums(Z, c, self.x, K)
        self.t += 1
        if self.F > 0 and self.t % self.F == 0:
            self.x = O.dct_denoise(self.x, self.sbm)[0]
            self.sbm *= self.decay
        return float(v[-1])

    def project(self, sbm):
        self.x = O.dct_denoise(self.x, sbm)[0]


def problem():
    return synth.make_problem(L, K, N, SIGMA, seed=synth.seed_for(31, 1), init="uniform")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2204_04754_gb300 import sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    p = problem()
    sh = OracleShard(p.y[CUTS[rank]:CUTS[rank + 1]], p.x0, p.rho1_0, p.rho2_0)
    lls = sharded.sharded_solve(sh, ITERS, F, sigma_bm1=SBM1)
    q.put((rank, sh.x, sh.r1, sh.r2, lls))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_em_equals_em_on_all_observations():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda r: r[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (_, x0_, a0, b0, ll0), (_, x1_, a1, b1, ll1) = res
    # every rank holds the same estimate (the all-reduce gives both the same sum)
    assert np.array_equal(x0_, x1_) and np.array_equal(a0, a1) and np.array_equal(b0, b1)
    assert ll0 == ll1
    p = problem()
    xo, r1o, r2o, h = O.projected_em(p.y, p.x0, p.rho1_0, p.rho2_0, SIGMA, K, ITERS, F,
                                     sigma_bm1=SBM1)
    assert h["margin"] > 1e-6
    assert np.linalg.norm(x0_ - xo) / np.linalg.norm(xo) < 1e-12
    assert np.abs(a0 - r1o).max() < 1e-12 and np.abs(b0 - r2o).max() < 1e-12
    np.testing.assert_allclose(ll0, h["LL"], rtol=1e-12)
    _ = os


def test_one_shard_is_the_local_iteration():
    """World size 1 (no process group needed for the check): the driver's statistics of
    a single shard holding everything reproduce the oracle's EM iteration."""
    p = problem()
    sh = OracleShard(p.y, p.x0, p.rho1_0, p.rho2_0)
    v = sh.estep_stats()
    ll = sh.mstep_stats(v)
    xo, r1o, r2o, llo, _ = O.em_iter(p.y, p.x0, p.rho1_0, p.rho2_0, SIGMA, K)
    assert np.linalg.norm(sh.x - xo) / np.linalg.norm(xo) < 1e-13
    assert abs(ll - llo) < 1e-10 * abs(llo)
