"""Projected EM with the observations sharded over ranks (one process per GPU).

Every rank holds a :class:`~paper_2204_04754_gb300.srmra.Solver` over its own shard of
the observations, all with the same L, K, sigma and starting estimate.  One iteration:

1. ``estep_stats``: the E-step of the shard at the common estimate, reduced to the
   statistics the M-step of Eqs. (x_EM), (rho_EM) reads (3 L^2 + 1 float64 sums over the
   shard's observations; include/srmra.h gives the layout);
2. one all-reduce (sum) of that vector over the ranks;
3. ``mstep_stats`` on the sum on every rank, so that all ranks hold the same estimate;
   on every F-th call it also applies the projection x <- D(x, sigma_BM) and the decay of
   sigma_BM (Algorithm 2) from the schedule the library keeps for the context
   (``set_schedule``), identically on every rank.

The result is the EM iteration over the union of the shards, up to the order of the
float sums.  With ``device=True`` the vector stays in device memory (an NCCL all-reduce);
the solvers must then run on torch's current CUDA stream, so that the collective is
ordered after the E-step kernels and before the M-step kernels.  Otherwise the vector
goes through host memory (any backend, e.g. gloo).
"""
from __future__ import annotations

import numpy as np


def sharded_iteration(solver, group=None, device: bool = False, buffer=None) -> float:
    """One EM iteration over all ranks' shards; returns LL(theta_t) of the union."""
    import torch
    import torch.distributed as dist
    if device:
        if buffer is None:
            buffer = torch.empty(solver.stats_length(), dtype=torch.float64, device="cuda")
        solver.estep_stats(out=buffer)
        dist.all_reduce(buffer, op=dist.ReduceOp.SUM, group=group)
        return solver.mstep_stats(buffer)
    v = torch.from_numpy(np.ascontiguousarray(solver.estep_stats(), dtype=np.float64))
    dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    return solver.mstep_stats(v.numpy())


def sharded_solve(solver, iters: int, F: int, sigma_bm1: float = 1.0,
                  decay: float = 2.0 ** -0.1, group=None, device: bool = False) -> list:
    """Algorithm 2 over the sharded observations: `iters` EM iterations, the projection
    after every F-th (F = 0: none) with sigma_BM starting at sigma_bm1 and multiplied by
    `decay` after each projection (the schedule is handed to the library, whose M-step
    applies it).  Returns the per-iteration LL(theta_t)."""
    buffer = None
    if device:
        import torch
        buffer = torch.empty(solver.stats_length(), dtype=torch.float64, device="cuda")
    solver.set_schedule(F, sigma_bm1, decay)
    return [sharded_iteration(solver, group=group, device=device, buffer=buffer)
            for _ in range(iters)]
