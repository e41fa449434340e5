"""The data-parallel decomposition over the observations on one GPU: the observations
split into G ragged chunks (one context each, same estimate), the E-step statistics of
the chunks (srmra_estep_stats) summed on the host in a fixed order, the M-step of the sum
(srmra_mstep_stats) against the unsplit EM iteration of the same form and against the
FP64 oracle; the device-memory form of the vectors; and the sharded driver through an
NCCL process group of one rank.

Tolerances: split vs unsplit differ only in the order of float sums over observations
(relative 1e-6 on x and rho for the float32 forms, 1e-5 for bf16x3, whose M-step sums
run in fp16 x fp16 products with float32 accumulation); LL per observation does not
depend on the split, so the LL sums agree to float64 rounding (1e-9).  Against the
oracle: 1e-5 for the float32 forms, 1e-4 for bf16x3 with the compensated M-step (hi +
lo fp16 operands).  The shards and the unsplit context are given the same M-step form
by flag (the automatic choice depends on each context's number of observations).
With single fp16 operands the M-step rounding of this small problem (900
observations) averages over few observations, so only split against unsplit is
checked for that form."""
import os
import socket

import numpy as np
import pytest

from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth
from tests import test_gpu_parity as P

pytestmark = pytest.mark.gpu

S = P.S  # module fixture

CUTS = [0, 250, 601, 900]
TOL_SPLIT = {"fp32": 1e-6, "fft32": 1e-6, "bf16x3": 1e-5}
TOL_ORACLE = {"fp32": 1e-5, "fft32": 1e-5, "bf16x3-comp": 1e-4}
FLAGS = {"bf16x3-comp": 4, "bf16x3-fp16": 8}  # SRMRA_FLAG_MSTEP_COMP / _MSTEP_FP16


def problem(L=32, K=2, sigma=0.5):
    return synth.make_problem(L, K, CUTS[-1], sigma, seed=synth.seed_for(41, L + K),
                              init="uniform")


def shards(S, p, prec, flags=0):
    return [S.Solver(p.L, p.K, p.sigma, p.y[a:b], prec=prec, x0=p.x0, rho1=p.rho1_0,
                     rho2=p.rho2_0, flags=flags) for a, b in zip(CUTS[:-1], CUTS[1:])]


@pytest.mark.parametrize("form,L,K", [("fp32", 32, 2), ("fp32", 24, 3), ("fft32", 32, 2),
                                      ("bf16x3-comp", 32, 2), ("bf16x3-fp16", 32, 2)])
def test_summed_shard_statistics_give_the_iteration(S, form, L, K):
    prec = form.split("-")[0]
    flags = FLAGS.get(form, 0)
    p = problem(L, K)
    sh = shards(S, p, prec, flags)
    vecs = [s.estep_stats() for s in sh]
    assert all(v.shape == (3 * L * L + 1,) for v in vecs)
    total = (vecs[0] + vecs[1]) + vecs[2]
    ll = sh[0].mstep_stats(total)
    x, r1, r2, _, t = sh[0].state()
    assert t == 1
    full = P.make_solver(S, p, prec, flags=flags)
    ll_full = full.em_iter(1)[0]
    xf, r1f, r2f, _, _ = full.state()
    tol = TOL_SPLIT[prec]
    assert P.rel(x, xf) < tol and P.rel(r1, r1f) < tol and P.rel(r2, r2f) < tol, \
        (P.rel(x, xf), P.rel(r1, r1f))
    assert abs(ll - ll_full) < 1e-9 * abs(ll_full)
    # c sums to the number of observations: to float32 rounding, or for bf16x3 with
    # single fp16 weights within the fp16 unit roundoff 2^-11 (a bound for a sum of
    # positive terms each rounded to relative 2^-11)
    ctol = 2.0 ** -11 if form == "bf16x3-fp16" else 1e-5 if prec == "bf16x3" else 1e-6
    assert abs(total[:L * L].sum() - p.N) < ctol * p.N
    xo, r1o, r2o, llo, _ = O.em_iter(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
    if form in TOL_ORACLE:
        tol = TOL_ORACLE[form]
        assert P.rel(x, xo) < tol and P.rel(r1, r1o) < tol and P.rel(r2, r2o) < tol
        assert abs(ll - llo) < 1e-5 * (abs(llo) + (p.y.astype(np.float64) ** 2).sum()
                                       / (2 * p.sigma ** 2))
    for s in sh + [full]:
        s.close()


def test_device_vectors_match_host_vectors(S):
    torch = pytest.importorskip("torch")
    p = problem()
    sh = shards(S, p, "fp32")
    host = [s.estep_stats() for s in sh]
    bufs = [torch.empty(sh[0].stats_length(), dtype=torch.float64, device="cuda")
            for _ in sh]
    for s, b in zip(sh, bufs):
        s.estep_stats(out=b)
    torch.cuda.synchronize()
    for h, b in zip(host, bufs):
        assert np.array_equal(h, b.cpu().numpy())  # same E-step, same reduction order
    tot = (bufs[0] + bufs[1]) + bufs[2]
    ll_dev = sh[1].mstep_stats(tot)
    ll_host = sh[2].mstep_stats((host[0] + host[1]) + host[2])
    xd = sh[1].state()[0]
    xh = sh[2].state()[0]
    assert np.array_equal(xd, xh) and ll_dev == ll_host
    for s in sh:
        s.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_driver_through_nccl_world_of_one(S):
    """The device path of sharded.py (estep into a CUDA tensor, NCCL all-reduce,
    M-step from the tensor, projection) on one rank equals srmra_solve."""
    torch = pytest.importorskip("torch")
    import torch.distributed as dist

    from paper_2204_04754_gb300 import sharded
    p = problem(64, 2, 0.4)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0,
                            world_size=1)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        a = S.Solver(p.L, p.K, p.sigma, p.y, x0=p.x0, rho1=p.rho1_0, rho2=p.rho2_0,
                     stream=stream)
        lls = sharded.sharded_solve(a, 4, 2, sigma_bm1=0.05, device=True)
        b = S.Solver(p.L, p.K, p.sigma, p.y, x0=p.x0, rho1=p.rho1_0, rho2=p.rho2_0,
                     stream=stream)
        llb = b.solve(4, 2, sigma_bm1=0.05)
        xa, r1a, _, sa, ta = a.state()
        xb, r1b, _, sb, tb = b.state()
        assert ta == tb == 4
        # the library applied Algorithm 2's schedule in the M-step of the sharded run
        assert sa == sb == 0.05 * 2.0 ** -0.2
        # four iterations of two float32 runs that differ in the order of their sums:
        # within the float32 form's tolerance
        assert P.rel(xa, xb) < 1e-5 and P.rel(r1a, r1b) < 1e-5, (P.rel(xa, xb), P.rel(r1a, r1b))
        # LL(theta_0): the same E-step at the same estimate; later ones at estimates that
        # differ by float32 rounding
        assert lls[0] == llb[0]
        np.testing.assert_allclose(lls[1:], llb[1:], rtol=1e-6)
        a.close()
        b.close()
    finally:
        dist.destroy_process_group()
    _ = os
