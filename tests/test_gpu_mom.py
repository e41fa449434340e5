"""Projected MoM on the GPU (srmra_mom_*) against the FP64 oracle oracle/mom_oracle.py
on the same seeded inputs: the empirical moments, the objective and its gradient at one
theta, and trajectories of the projected gradient iteration with and without the
denoiser; full-size moments and gradient for the two single-problem workloads; argument
errors.

Tolerances (float32 products, float64 partial sums):
  * M1^, M2^: relative Frobenius error 1e-5 (float32 accumulation of N / splits terms
    of O(1) values: about sqrt(N / splits) 2^-24 relative per partial).
  * f, df/dx, df/drho: 1e-4 relative (R = M2 - M2^ is a difference of O(1) values whose
    float32 rounding, about 1e-6 absolute, is divided by ||R||, which is 1e-2 .. 1e-1 of
    ||M2|| at the starting points used here).
  * trajectories: x and rho within 1e-4 relative after a few steps (the per-step error
    above, carried by a contraction-free but short iteration)."""
import numpy as np
import pytest

from oracle import mom_oracle as M
from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth
from tests import test_gpu_parity as P

pytestmark = pytest.mark.gpu

S = P.S  # module fixture

CASES = [(16, 2, 500, 0.5), (24, 3, 700, 0.4), (32, 2, 1000, 0.3), (40, 5, 333, 0.6)]


def problem(L, K, N, sigma, tag=0):
    return synth.make_problem(L, K, N, sigma, seed=synth.seed_for(21 + tag, L * 7 + K))


def frob_rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L,K,N,sigma", CASES)
def test_empirical_moments(S, L, K, N, sigma):
    p = problem(L, K, N, sigma)
    s = P.make_solver(S, p)
    m = S.Mom(s)
    m1, m2 = m.moments()
    o1, o2 = M.empirical_moments(p.y)
    assert frob_rel(m1, o1) < 1e-5 and frob_rel(m2, o2) < 1e-5, (frob_rel(m1, o1),
                                                                 frob_rel(m2, o2))
    assert np.array_equal(m2, m2.T)  # Y^T Y: the same products in both triangles
    m.close()
    s.close()


def test_moments_of_one_observation(S):
    p = problem(16, 2, 1, 0.5)
    s = P.make_solver(S, p)
    m = S.Mom(s)
    m1, m2 = m.moments()
    y = p.y.astype(np.float64).ravel()
    assert frob_rel(m1, y) < 1e-6 and frob_rel(m2, np.outer(y, y)) < 1e-6
    m.close()
    s.close()


@pytest.mark.parametrize("L,K,N,sigma", CASES)
def test_objective_and_gradient(S, L, K, N, sigma):
    p = problem(L, K, N, sigma)
    rng = np.random.default_rng(L + K)
    r1 = rng.uniform(0.2, 1.0, L)
    r2 = rng.uniform(0.2, 1.0, L)
    r1 /= r1.sum()
    r2 /= r2.sum()
    s = S.Solver(p.L, p.K, p.sigma, p.y, x0=p.x0, rho1=r1, rho2=r2)
    m = S.Mom(s)
    f, gx, g1, g2 = m.eval()
    x, r1g, r2g, _, _ = s.state()
    M1h, M2h = M.empirical_moments(p.y)
    fo, gxo, g1o, g2o = M.gradient(x.astype(np.float64), r1g, r2g, M1h, M2h, p.sigma, p.K)
    assert abs(f - fo) / fo < 1e-4, (f, fo)
    assert P.rel(gx, gxo) < 1e-4, P.rel(gx, gxo)
    assert P.rel(g1, g1o) < 1e-4 and P.rel(g2, g2o) < 1e-4, (P.rel(g1, g1o), P.rel(g2, g2o))
    # eval does not move theta
    x2, r12, r22, _, _ = s.state()
    assert np.array_equal(x, x2) and np.array_equal(r1g, r12) and np.array_equal(r2g, r22)
    m.close()
    s.close()


def step_sizes(p, x, r1, r2, c):
    """Steps that move the largest gradient entry by c (descending, stable here)."""
    M1h, M2h = M.empirical_moments(p.y)
    _, gx, g1, g2 = M.gradient(x, r1, r2, M1h, M2h, p.sigma, p.K)
    return c / np.abs(gx).max(), c / max(np.abs(g1).max(), np.abs(g2).max())


@pytest.mark.parametrize("L,K,N,sigma", CASES[:3])
def test_projected_gradient_trajectory(S, L, K, N, sigma):
    p = problem(L, K, N, sigma, tag=1)
    x0 = p.x0.astype(np.float64)
    mu_x, mu_r = step_sizes(p, x0, p.rho1_0, p.rho2_0, 0.01)
    s = P.make_solver(S, p)
    m = S.Mom(s)
    iters = 6
    fs = m.run(iters, 0, mu_x, mu_r)
    x, r1, r2, _, _ = s.state()
    xo, r1o, r2o, fo = M.projected_mom(p.y, x0, p.rho1_0, p.rho2_0, p.sigma, p.K, iters, 0,
                                       mu_x, mu_r)
    assert all(b < a for a, b in zip(fo, fo[1:]))  # the steps descend
    assert P.rel(fs, fo) < 1e-4, P.rel(fs, fo)
    assert P.rel(x, xo) < 1e-4, P.rel(x, xo)
    assert P.rel(r1, r1o) < 1e-4 and P.rel(r2, r2o) < 1e-4
    assert abs(r1.sum() - 1) < 1e-12 and (r1 >= 0).all() and (r2 >= 0).all()
    m.close()
    s.close()


def test_trajectory_with_denoiser(S):
    L, K = 32, 2
    p = problem(L, K, 800, 0.4, tag=2)
    x0 = p.x0.astype(np.float64)
    mu_x, mu_r = step_sizes(p, x0, p.rho1_0, p.rho2_0, 0.02)
    iters, F, sbm1, decay = 4, 2, 0.05, 0.5
    # the oracle's iteration step by step, checking that no coefficient sits at the
    # hard threshold (where float32 and float64 may keep different coefficients)
    M1h, M2h = M.empirical_moments(p.y)
    x, r1, r2, sbm = x0, p.rho1_0.copy(), p.rho2_0.copy(), sbm1
    for t in range(iters):
        _, gx, g1, g2 = M.gradient(x, r1, r2, M1h, M2h, p.sigma, p.K)
        x = x - mu_x * gx
        r1, r2 = M.project_simplex(r1 - mu_r * g1), M.project_simplex(r2 - mu_r * g2)
        if (t + 1) % F == 0:
            x, margin = O.dct_denoise(x, sbm)
            assert margin > 1e-4, margin
            sbm *= decay
    xo, r1o, r2o, _ = M.projected_mom(p.y, x0, p.rho1_0, p.rho2_0, p.sigma, p.K, iters, F,
                                      mu_x, mu_r, sigma_bm1=sbm1, decay=decay)
    assert np.array_equal(x, xo)
    s = P.make_solver(S, p)
    m = S.Mom(s)
    m.run(iters, F, mu_x, mu_r, sigma_bm1=sbm1, decay=decay)
    xg, r1g, r2g, _, _ = s.state()
    assert P.rel(xg, xo) < 1e-4, P.rel(xg, xo)
    assert P.rel(r1g, r1o) < 1e-4 and P.rel(r2g, r2o) < 1e-4
    m.close()
    s.close()


def test_moments_do_not_depend_on_the_form(S):
    """Every form keeps the float32 centred observations; the moment pass reads only
    those, so its result is the same bit for bit."""
    p = problem(32, 2, 900, 0.5)
    ref = None
    for prec in ("fp32", "bf16x3", "fft32"):
        s = P.make_solver(S, p, prec)
        m = S.Mom(s)
        got = m.moments()
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), prec
        m.close()
        s.close()


def test_run_is_deterministic(S):
    p = problem(24, 3, 600, 0.5, tag=3)
    out = []
    for _ in range(2):
        s = P.make_solver(S, p)
        m = S.Mom(s)
        fs = m.run(5, 0, 1e-3, 1e-3)
        out.append((fs, s.state()[0]))
        m.close()
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("name", ["proj_em_L64_K2_N1e4", "precision_L96_K3_N5e4_s0.2"])
def test_full_size_moments_and_gradient(S, name):
    p = synth.workload_problem(name)
    s = P.make_solver(S, p)
    m = S.Mom(s)
    m1, m2 = m.moments()
    Y = p.y.reshape(p.N, -1).astype(np.float64)
    o1 = Y.mean(axis=0)
    rows = np.random.default_rng(0).choice(Y.shape[1], 24, replace=False)
    o2 = (Y[:, rows].T @ Y) / p.N
    assert frob_rel(m1, o1) < 1e-5
    assert frob_rel(m2[rows], o2) < 1e-5, frob_rel(m2[rows], o2)
    f, gx, g1, g2 = m.eval()
    x, r1, r2, _, _ = s.state()
    M1h, M2h = M.empirical_moments(p.y)
    fo, gxo, g1o, g2o = M.gradient(x.astype(np.float64), r1, r2, M1h, M2h, p.sigma, p.K)
    assert abs(f - fo) / fo < 1e-4
    assert P.rel(gx, gxo) < 1e-4 and P.rel(g1, g1o) < 1e-4 and P.rel(g2, g2o) < 1e-4
    m.close()
    s.close()


def test_argument_errors(S):
    p = problem(12, 2, 50, 0.5)  # L % 8 != 0
    s = P.make_solver(S, p)
    m = S.Mom(s)
    for bad in [dict(iters=-1, F=0), dict(iters=1, F=-1), dict(iters=1, F=0, decay=0.0),
                dict(iters=1, F=1)]:  # the built-in denoiser needs L % 8 == 0
        kw = dict(mu_x=1e-3, mu_rho=1e-3)
        kw.update(bad)
        with pytest.raises(S.SrmraError) as e:
            m.run(**kw)
        assert e.value.status == S.SRMRA_EINVAL
    assert m.run(0, 0, 1e-3, 1e-3).size == 0
    m.close()
    s.close()


def test_non_finite_objective_is_reported_once(S):
    """An estimate whose moments overflow float32 gives ENUMERIC; the status is cleared
    after the report, so the next evaluation at a finite estimate succeeds."""
    p = problem(16, 2, 200, 0.5)
    s = P.make_solver(S, p)
    m = S.Mom(s)
    x, r1, r2, sbm, t = s.state()
    s.set_state(np.full_like(x, 1e30), r1, r2, sbm, t)
    with pytest.raises(S.SrmraError) as e:
        m.eval()
    assert e.value.status == S.SRMRA_ENUMERIC
    s.set_state(x, r1, r2, sbm, t)
    f, gx, _, _ = m.eval()
    assert np.isfinite(f) and np.all(np.isfinite(gx))
    m.close()
    s.close()
