"""Pins of the projected-MoM oracle (oracle/mom_oracle.py) to quantities fixed
independently of its own formulas: element-by-element moments of the model, the exact
moments of a weighted population, finite differences of the objective, the optimality
conditions of the simplex projection; and planted mistakes that these catch."""
import numpy as np
import pytest

from oracle import mom_oracle as M
from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth


def small(L=8, K=2, seed=3):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (L, L))
    r1 = rng.uniform(0.2, 1, L)
    r2 = rng.uniform(0.2, 1, L)
    return x, r1 / r1.sum(), r2 / r2.sum()


def test_model_moments_element_by_element():
    """M1[n] = sum_s rho_s (P R_s x)[n], M2[n, n'] = sum_s rho_s t_s[n] t_s[n'] +
    sigma^2 [n == n'], with P R_s x from the sampling and shift operators, by loops."""
    L, K, sigma = 4, 2, 0.3
    x, r1, r2 = small(L, K)
    l = L // K
    M1 = np.zeros(l * l)
    M2 = np.zeros((l * l, l * l))
    for s1 in range(L):
        for s2 in range(L):
            t = O.sample(O.shift(x, s1, s2), K).ravel()
            w = r1[s1] * r2[s2]
            for n in range(l * l):
                M1[n] += w * t[n]
                for m in range(l * l):
                    M2[n, m] += w * t[n] * t[m]
    M2 += sigma ** 2 * np.eye(l * l)
    m1, m2 = M.model_moments(x, r1, r2, sigma, K)
    np.testing.assert_allclose(m1, M1, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(m2, M2, rtol=1e-13, atol=1e-15)


def test_empirical_moments_of_an_exact_population():
    """Noise-free observations drawn with exact rational weights (each shift repeated in
    proportion to rho): the empirical moments equal the model moments at sigma = 0."""
    L, K = 4, 2
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (L, L))
    c1 = np.array([1, 2, 3, 2])
    c2 = np.array([2, 1, 1, 4])
    Y = []
    for s1 in range(L):
        for s2 in range(L):
            Y += [O.sample(O.shift(x, s1, s2), K)] * int(c1[s1] * c2[s2])
    Y = np.array(Y)
    M1h, M2h = M.empirical_moments(Y)
    m1, m2 = M.model_moments(x, c1 / c1.sum(), c2 / c2.sum(), 0.0, K)
    np.testing.assert_allclose(M1h, m1, rtol=1e-13)
    np.testing.assert_allclose(M2h, m2, rtol=1e-13)


@pytest.mark.parametrize("L,K", [(6, 2), (8, 2), (6, 3)])
def test_gradient_matches_finite_differences(L, K):
    x, r1, r2 = small(L, K, seed=L + K)
    p = synth.make_problem(L, K, 300, 0.4, seed=11)
    M1h, M2h = M.empirical_moments(p.y)
    f, gx, g1, g2 = M.gradient(x, r1, r2, M1h, M2h, 0.4, K)
    assert abs(f - M.objective(x, r1, r2, M1h, M2h, 0.4, K)) < 1e-12 * abs(f)
    rng = np.random.default_rng(1)
    h = 1e-5
    for _ in range(3):
        dx = rng.standard_normal((L, L))
        d1 = rng.standard_normal(L)
        d2 = rng.standard_normal(L)
        fp = M.objective(x + h * dx, r1 + h * d1, r2 + h * d2, M1h, M2h, 0.4, K)
        fm = M.objective(x - h * dx, r1 - h * d1, r2 - h * d2, M1h, M2h, 0.4, K)
        fd = (fp - fm) / (2 * h)
        an = (gx * dx).sum() + g1 @ d1 + g2 @ d2
        assert abs(fd - an) < 1e-6 * (abs(an) + 1e-3), (fd, an)


def test_objective_vanishes_at_the_model_moments():
    x, r1, r2 = small(8, 2)
    m1, m2 = M.model_moments(x, r1, r2, 0.5, 2)
    assert M.objective(x, r1, r2, m1, m2, 0.5, 2) == 0.0
    _, gx, g1, g2 = M.gradient(x, r1, r2, m1, m2, 0.5, 2)
    assert np.abs(gx).max() == 0.0 and np.abs(g1).max() == 0.0 and np.abs(g2).max() == 0.0


def test_simplex_projection():
    rng = np.random.default_rng(2)
    for n in (1, 2, 5, 64):
        for _ in range(20):
            v = rng.standard_normal(n) * rng.uniform(0.1, 3)
            w = M.project_simplex(v)
            assert abs(w.sum() - 1) < 1e-12 and (w >= 0).all()
            # optimality: w = max(v - tau, 0) with one tau (the KKT conditions), found
            # independently by bisection on sum max(v - tau, 0) = 1
            lo, hi = v.min() - 1, v.max()
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if np.maximum(v - mid, 0).sum() > 1:
                    lo = mid
                else:
                    hi = mid
            np.testing.assert_allclose(w, np.maximum(v - 0.5 * (lo + hi), 0), atol=1e-12)
            np.testing.assert_allclose(M.project_simplex(w), w, atol=1e-15)


def test_gradient_step_decreases_the_objective():
    p = synth.make_problem(8, 2, 400, 0.3, seed=12)
    M1h, M2h = M.empirical_moments(p.y)
    x, r1, r2 = p.x0.astype(np.float64), p.rho1_0, p.rho2_0
    f0, gx, g1, g2 = M.gradient(x, r1, r2, M1h, M2h, p.sigma, p.K)
    mu = 1e-3 / (np.abs(gx).max() + 1e-12)
    f1 = M.objective(x - mu * gx, r1, r2, M1h, M2h, p.sigma, p.K)
    assert f1 < f0


def test_lambda_weight_of_the_first_moment_term():
    """Eq. (LS_SR) weighs the first-moment residual by lambda = 1 / (L^2 (1 + sigma^2)).
    With M2^ equal to the model's M2 and M1^ off the model's M1 by a unit vector, the
    objective is lambda alone: 1/32 at L = 4, sigma = 1 (hand-evaluated: 16 * 2 = 32),
    and 1/(64 * 1.25) = 0.0125 at L = 8, sigma = 0.5."""
    for L, K, sigma, lam in [(4, 2, 1.0, 1.0 / 32.0), (8, 2, 0.5, 0.0125)]:
        x, r1, r2 = small(L, K, seed=L)
        m1, m2 = M.model_moments(x, r1, r2, sigma, K)
        e = np.zeros_like(m1)
        e[1] = 1.0
        f = M.objective(x, r1, r2, m1 + e, m2, sigma, K)
        assert abs(f - lam) < 1e-15, (L, sigma, f)
        # and the second-moment term is unweighted: a unit entry of M2^ - M2 adds 1
        E = np.zeros_like(m2)
        E[0, 1] = 1.0
        f2 = M.objective(x, r1, r2, m1, m2 + E, sigma, K)
        assert abs(f2 - 1.0) < 1e-12


def test_planted_mistakes_are_caught(monkeypatch):
    def fails(check):
        try:
            check()
        except AssertionError:
            return True
        return False

    orig = M.gradient
    orig_moments = M.model_moments

    def no_four(x, r1, r2, M1h, M2h, sigma, K):  # the x-gradient with 2 R t_s instead of 4
        f, gx, g1, g2 = orig(x, r1, r2, M1h, M2h, sigma, K)
        return f, 0.5 * gx, g1, g2

    monkeypatch.setattr(M, "gradient", no_four)
    assert fails(lambda: test_gradient_matches_finite_differences(6, 2))
    monkeypatch.setattr(M, "gradient", orig)
    monkeypatch.setattr(M, "model_moments", lambda x, r1, r2, sigma, K: (
        np.outer(r1, r2).ravel() @ O.all_templates(np.asarray(x, float), K),
        O.all_templates(np.asarray(x, float), K).T @ O.all_templates(np.asarray(x, float), K)))
    assert fails(test_model_moments_element_by_element)
    monkeypatch.setattr(M, "model_moments", orig_moments)
    # lambda without the square on sigma, and without the 1/L^2
    monkeypatch.setattr(M, "mom_lambda", lambda L, sigma: 1.0 / (L * L * (1.0 + sigma)))
    assert fails(lambda: (test_lambda_weight_of_the_first_moment_term(),
                          _lambda_at(8, 0.5, 0.0125)))
    monkeypatch.setattr(M, "mom_lambda", lambda L, sigma: 1.0 / (1.0 + sigma * sigma))
    assert fails(test_lambda_weight_of_the_first_moment_term)


def _lambda_at(L, sigma, lam):
    x, r1, r2 = small(L, 2, seed=L)
    m1, m2 = M.model_moments(x, r1, r2, sigma, 2)
    e = np.zeros_like(m1)
    e[0] = 1.0
    assert abs(M.objective(x, r1, r2, m1 + e, m2, sigma, 2) - lam) < 1e-15
