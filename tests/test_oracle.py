"""Pins for the FP64 oracle against things other than itself: explicit operator
matrices, closed forms, invariants the paper states, special cases, and library
routines.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import fft_oracle as FO
from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------- explicit operators

def explicit_P(L, K):
    """Selection matrix P (l^2 x L^2): row n1*l+n2 picks pixel (n1*K, n2*K)."""
    l = L // K
    P = np.zeros((l * l, L * L))
    for n1 in range(l):
        for n2 in range(l):
            P[n1 * l + n2, (n1 * K) * L + n2 * K] = 1.0
    return P


def explicit_R(L, s1, s2):
    """Permutation matrix of the circular translation: (R_s x)[q] = x[q - s]."""
    R = np.zeros((L * L, L * L))
    for q1 in range(L):
        for q2 in range(L):
            R[q1 * L + q2, ((q1 - s1) % L) * L + (q2 - s2) % L] = 1.0
    return R


@pytest.mark.parametrize("L,K", [(4, 1), (4, 2), (6, 2), (6, 3), (8, 2), (8, 4)])
def test_templates_and_adjoint_match_explicit_matrices(L, K):
    rng = np.random.default_rng(L * 10 + K)
    x = rng.standard_normal((L, L))
    l = L // K
    P = explicit_P(L, K)
    T = O.all_templates(x, K)
    for s1 in range(L):
        for s2 in range(L):
            M = P @ explicit_R(L, s1, s2)
            np.testing.assert_array_equal(T[s1 * L + s2], M @ x.ravel())
            v = rng.standard_normal((l, l))
            np.testing.assert_allclose(O.template_adjoint(v, K, s1, s2).ravel(),
                                       M.T @ v.ravel(), rtol=0, atol=1e-15)


def test_synthetic_observations_follow_the_model():
    """Noise-free synthetic observations equal the oracle's templates at the drawn
    shifts (two independent codings of Eq. (1))."""
    p = synth.make_problem(16, 2, 50, 0.0, seed=7)
    T = O.all_templates(p.x_true, p.K)
    for i in range(p.N):
        np.testing.assert_array_equal(p.y[i].ravel(),
                                      T[p.s1[i] * p.L + p.s2[i]].astype(np.float32))


def test_synthetic_generator_is_deterministic():
    a = synth.make_problem(32, 4, 100, 0.2, seed=3)
    b = synth.make_problem(32, 4, 100, 0.2, seed=3)
    assert a.y.tobytes() == b.y.tobytes() and a.x0.tobytes() == b.x0.tobytes()
    assert abs(a.rho1_true.sum() - 1) < 1e-14 and np.all(a.rho1_true > 0)


# ---------------------------------------------------------------- E-step

def brute_force_estep(Y, x, rho1, rho2, sigma, K):
    """Eq. (weights_EM) with explicit P, R_s and naive normalisation (no max trick)."""
    L = x.shape[0]
    P = explicit_P(L, K)
    N = Y.shape[0]
    W = np.zeros((N, L * L))
    LL = 0.0
    for i in range(N):
        tot = 0.0
        for s1 in range(L):
            for s2 in range(L):
                r = Y[i].ravel() - P @ explicit_R(L, s1, s2) @ x.ravel()
                W[i, s1 * L + s2] = rho1[s1] * rho2[s2] * math.exp(-(r @ r) / (2 * sigma ** 2))
                tot += W[i, s1 * L + s2]
        W[i] /= tot
        LL += math.log(tot)
    return W, LL


@pytest.mark.parametrize("L,K,N,sigma", [(4, 1, 3, 1.0), (4, 2, 5, 0.7), (6, 2, 4, 0.9),
                                         (6, 3, 5, 1.2), (8, 2, 3, 1.5)])
def test_estep_matches_brute_force(L, K, N, sigma):
    rng = np.random.default_rng(100 + L + K)
    x = rng.uniform(0, 1, (L, L))
    Y = rng.uniform(0, 1, (N, L // K, L // K))
    r1 = synth.uniform_simplex_draw(L, rng)
    r2 = synth.uniform_simplex_draw(L, rng)
    Wb, LLb = brute_force_estep(Y, x, r1, r2, sigma, K)
    for literal in (True, False):
        W, lse, LL = O.estep(Y, x, r1, r2, sigma, K, literal=literal)
        np.testing.assert_allclose(W, Wb, rtol=1e-12, atol=1e-15)
        assert abs(LL - LLb) <= 1e-12 * abs(LLb)
        np.testing.assert_allclose(W.sum(axis=1), 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("chunk", [None, 1, 3, 7])
def test_chunked_loglik_matches_brute_force(chunk):
    """The chunked Eq. (likelihood_EM) of the oracle equals the brute-force sum over
    observations of log sum_s rho1 rho2 exp(-||y_i - P R_s x||^2 / (2 sigma^2)) (explicit
    P and R_s matrices, naive normalisation), for any chunk size, and the E-step's LL."""
    L, K, N, sigma = 6, 2, 8, 0.7
    rng = np.random.default_rng(321)
    x = rng.uniform(0, 1, (L, L))
    Y = rng.uniform(0, 1, (N, L // K, L // K))
    r1 = synth.uniform_simplex_draw(L, rng)
    r2 = synth.uniform_simplex_draw(L, rng)
    _, LLb = brute_force_estep(Y, x, r1, r2, sigma, K)
    ll = O.loglik(Y, x, r1, r2, sigma, K, chunk=chunk)
    assert abs(ll - LLb) <= 1e-12 * abs(LLb)
    assert abs(ll - O.estep(Y, x, r1, r2, sigma, K)[2]) <= 1e-12 * abs(LLb)


def test_literal_and_expanded_distances_agree():
    p = synth.make_problem(16, 2, 40, 0.3, seed=11)
    T = O.all_templates(p.x0, 2)
    Y = p.y.reshape(p.N, -1).astype(np.float64)
    d1 = O.sq_distances(Y, T, literal=True)
    d2 = O.sq_distances(Y, T, literal=False)
    np.testing.assert_allclose(d2, d1, rtol=1e-11, atol=1e-11)


def test_zero_rho_entries_give_zero_weight():
    """Reading R7: rho[s] = 0 -> weight exactly 0, no NaN."""
    p = synth.make_problem(8, 2, 10, 0.5, seed=5)
    r1 = np.array(p.rho1_0)
    r1[3] = 0.0
    r1 /= r1.sum()
    W, lse, LL = O.estep(p.y, p.x0, r1, p.rho2_0, p.sigma, p.K)
    assert np.all(np.isfinite(W)) and np.isfinite(LL)
    assert np.all(W.reshape(-1, 8, 8)[:, 3, :] == 0.0)


# ---------------------------------------------------------------- M-step

@pytest.mark.parametrize("L,K", [(4, 2), (6, 2), (6, 3), (8, 4)])
def test_mstep_matches_dense_linear_solve(L, K):
    """Eq. (x_EM) assembled as dense L^2 x L^2 A and b (reading R1: P^-1 -> P^T) and
    solved by a general LU; must equal the oracle's diagonal b/A."""
    rng = np.random.default_rng(L * K)
    N = 6
    x = rng.uniform(0, 1, (L, L))
    Y = rng.uniform(0, 1, (N, L // K, L // K))
    r1 = synth.uniform_simplex_draw(L, rng)
    r2 = synth.uniform_simplex_draw(L, rng)
    W, _, _ = O.estep(Y, x, r1, r2, 0.8, K)
    P = explicit_P(L, K)
    A = np.zeros((L * L, L * L))
    b = np.zeros(L * L)
    for s1 in range(L):
        for s2 in range(L):
            M = P @ explicit_R(L, s1, s2)
            ws = W[:, s1 * L + s2]
            A += ws.sum() * (M.T @ M)
            b += M.T @ (Y.reshape(N, -1).T @ ws)
    x_lu = np.linalg.solve(A, b)
    xn, rr1, rr2, bo, Ao = O.mstep(Y, W, x, K)
    np.testing.assert_allclose(xn.ravel(), x_lu, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Ao.ravel(), np.diag(A), rtol=1e-13)
    # rho: marginals of the joint update of Eq. (rho_EM)
    joint = W.sum(axis=0) / W.sum()
    np.testing.assert_allclose(rr1, joint.reshape(L, L).sum(1), rtol=1e-13)
    np.testing.assert_allclose(rr2, joint.reshape(L, L).sum(0), rtol=1e-13)
    assert abs(rr1.sum() - 1) < 1e-14 and abs(rr2.sum() - 1) < 1e-14


def test_mstep_x_is_stationary_point_of_Q():
    """x_{t+1} maximises Eq. (Q) over x: finite-difference gradient vanishes and Q
    decreases under perturbation; the rho update maximises Q over the product
    simplex (perturbations along the simplex decrease it)."""
    p = synth.make_problem(8, 2, 30, 0.4, seed=21)
    W, _, _ = O.estep(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
    xn, r1, r2, _, _ = O.mstep(p.y, W, p.x0, p.K)
    q0 = O.q_function(p.y, W, xn, r1, r2, p.sigma, p.K)
    h = 1e-5
    rng = np.random.default_rng(0)
    for _ in range(6):
        d = rng.standard_normal(xn.shape)
        qp = O.q_function(p.y, W, xn + h * d, r1, r2, p.sigma, p.K)
        qm = O.q_function(p.y, W, xn - h * d, r1, r2, p.sigma, p.K)
        assert abs(qp - qm) / (2 * h) < 1e-6 * abs(q0)
        assert qp < q0 and qm < q0
    for j, k in [(0, 3), (2, 5), (7, 1)]:
        e = np.zeros(8)
        e[j], e[k] = 1e-3, -1e-3
        assert O.q_function(p.y, W, xn, r1 + e, r2, p.sigma, p.K) < q0
        assert O.q_function(p.y, W, xn, r1, r2 + e, p.sigma, p.K) < q0
    q_old = O.q_function(p.y, W, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
    assert q0 >= q_old


def test_onehot_weights_noise_free_reconstruct_x_exactly():
    """Invariant: sigma = 0 observations with one-hot weights at the true
    shifts give x back exactly (all K^2 phases are hit)."""
    p = synth.make_problem(16, 2, 64, 0.0, seed=9)
    L = p.L
    W = np.zeros((p.N, L * L))
    W[np.arange(p.N), p.s1 * L + p.s2] = 1.0
    phases = set(zip((-p.s1) % p.K, (-p.s2) % p.K))
    assert len(phases) == p.K * p.K
    xn, _, _, _, _ = O.mstep(p.y, W, np.zeros((L, L)), p.K)
    np.testing.assert_allclose(xn, p.x_true.astype(np.float64), rtol=0, atol=1e-7)


def test_K1_coverage_is_N_everywhere():
    """K = 1 (classic 2D MRA): every shift samples every pixel, so A[q] = N."""
    p = synth.make_problem(8, 1, 25, 0.5, seed=4)
    _, _, _, _, aux = O.em_iter(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, 1)
    np.testing.assert_allclose(aux["A"], p.N, rtol=1e-13)


def test_rho_is_fixed_point_for_constant_image():
    """Constant x: all templates are equal, so w^{i,s} = rho[s] and Eq. (rho_EM)
    returns rho unchanged (closed form)."""
    rng = np.random.default_rng(2)
    L, K = 8, 2
    Y = rng.standard_normal((20, 4, 4))
    r1 = synth.uniform_simplex_draw(L, rng)
    r2 = synth.uniform_simplex_draw(L, rng)
    _, n1, n2, _, _ = O.em_iter(Y, np.full((L, L), 0.3), r1, r2, 0.5, K)
    np.testing.assert_allclose(n1, r1, rtol=1e-12)
    np.testing.assert_allclose(n2, r2, rtol=1e-12)


def test_worked_example_closed_form():
    """L=2, K=2: EM reduces to a 4-component Gaussian mixture (closed form fixture)."""
    with open(os.path.join(GOLDEN, "worked_example_L2_K2.json")) as f:
        g = json.load(f)
    x = np.array(g["x"])
    Y = np.array(g["y"]).reshape(-1, 1, 1)
    W, lse, LL = O.estep(Y, x, g["rho1"], g["rho2"], g["sigma"], g["K"])
    e = g["expected"]
    np.testing.assert_allclose(W, e["weights"], rtol=1e-13)
    np.testing.assert_allclose(lse, e["lse"], rtol=1e-13)
    xn, r1, r2, LL2, _ = O.em_iter(Y, x, g["rho1"], g["rho2"], g["sigma"], g["K"])
    np.testing.assert_allclose(xn, e["x"], rtol=1e-13)
    np.testing.assert_allclose(r1, e["rho1"], rtol=1e-13)
    np.testing.assert_allclose(r2, e["rho2"], rtol=1e-13)
    assert abs(LL2 - e["loglik"]) < 1e-13 * abs(e["loglik"])


# ---------------------------------------------------------------- invariants

def test_loglik_monotone_without_projection():
    """Sec. 2: an EM iteration never decreases the likelihood."""
    p = synth.make_problem(16, 2, 300, 0.3, seed=12)
    x, r1, r2 = p.x0.astype(np.float64), p.rho1_0, p.rho2_0
    prev = -math.inf
    for _ in range(8):
        x, r1, r2, LL, _ = O.em_iter(p.y, x, r1, r2, p.sigma, p.K)
        assert LL >= prev - 1e-9 * abs(LL)
        prev = LL
    assert O.loglik(p.y, x, r1, r2, p.sigma, p.K) >= prev - 1e-9 * abs(prev)


def test_theorem1_subimage_permutation_and_shift_invariance():
    """Theorem 1: with uniform rho, permuting the K^2 sub-images and translating each on
    the low-resolution grid leaves the likelihood unchanged."""
    p = synth.make_problem(12, 3, 40, 0.4, seed=13)
    x = p.x_true.astype(np.float64)
    ll0 = O.loglik(p.y, x, p.rho1_0, p.rho2_0, p.sigma, p.K)
    xr = FO.polyphase(x, p.K).reshape(p.K * p.K, p.l, p.l)
    rng = np.random.default_rng(1)
    perm = rng.permutation(p.K * p.K)
    moved = np.stack([np.roll(xr[j], shift=tuple(rng.integers(0, p.l, 2)), axis=(0, 1))
                      for j in perm])
    x2 = FO.unpolyphase(moved.reshape(p.K, p.K, p.l, p.l))
    assert not np.allclose(x2, x)
    ll1 = O.loglik(p.y, x2, p.rho1_0, p.rho2_0, p.sigma, p.K)
    assert abs(ll1 - ll0) <= 1e-12 * abs(ll0)


def test_global_shift_equivariance():
    """P R_s R_u x = P R_{s+u} x: with x' = R_u x and rho' = rho(. + u), the weights
    are permuted, w'[i, s] = w[i, s + u], and the likelihood is unchanged."""
    p = synth.make_problem(8, 2, 15, 0.5, seed=14)
    x = p.x0.astype(np.float64)
    r1, r2 = p.rho1_true, p.rho2_true
    u1, u2 = 3, 5
    W, _, LL = O.estep(p.y, x, r1, r2, p.sigma, p.K)
    W2, _, LL2 = O.estep(p.y, O.shift(x, u1, u2), np.roll(r1, -u1), np.roll(r2, -u2),
                         p.sigma, p.K)
    L = p.L
    idx = (((np.arange(L)[:, None] + u1) % L) * L + (np.arange(L)[None, :] + u2) % L).ravel()
    np.testing.assert_allclose(W2, W[:, idx], rtol=1e-10, atol=1e-15)
    assert abs(LL2 - LL) < 1e-12 * abs(LL)


# ---------------------------------------------------------------- second oracle

@pytest.mark.parametrize("L,K,N,sigma", [(16, 2, 500, 0.1), (12, 3, 200, 0.5),
                                         (16, 4, 300, 1.0), (8, 1, 50, 0.3)])
def test_fft_oracle_matches_dense(L, K, N, sigma):
    p = synth.make_problem(L, K, N, sigma, seed=L + K + N)
    a = O.em_iter(p.y, p.x0, p.rho1_true, p.rho2_true, sigma, K)
    b = FO.em_iter_fft(p.y, p.x0, p.rho1_true, p.rho2_true, sigma, K, chunk=97)
    for u, v in zip(a[:3], b[:3]):
        assert np.linalg.norm(u - v) <= 1e-12 * np.linalg.norm(u)
    assert abs(a[3] - b[3]) <= 1e-12 * abs(a[3])
    for key in ("b", "A", "c", "lse"):
        assert np.linalg.norm(a[4][key] - b[4][key]) <= 1e-12 * np.linalg.norm(a[4][key])


@pytest.mark.parametrize("workers", [2, 5])
def test_fft_oracle_thread_split_matches_dense(workers):
    """The observation-range split of the FFT oracle (sums over i formed per range and
    added in order) is the same iteration as the dense definition."""
    p = synth.make_problem(12, 3, 333, 0.4, seed=77)
    a = O.em_iter(p.y, p.x0, p.rho1_true, p.rho2_true, 0.4, 3)
    b = FO.em_iter_fft(p.y, p.x0, p.rho1_true, p.rho2_true, 0.4, 3, chunk=41, workers=workers)
    for u, v in zip(a[:3], b[:3]):
        assert np.linalg.norm(u - v) <= 1e-12 * np.linalg.norm(u)
    assert abs(a[3] - b[3]) <= 1e-12 * abs(a[3])
    np.testing.assert_allclose(b[4]["lse"], a[4]["lse"], rtol=1e-12)


# ---------------------------------------------------------------- denoiser

def test_dct_matrix_is_orthonormal_and_matches_scipy():
    scipy_fft = pytest.importorskip("scipy.fft")
    C = O.dct_matrix(8)
    np.testing.assert_allclose(C @ C.T, np.eye(8), atol=4e-15)
    rng = np.random.default_rng(0)
    blk = rng.standard_normal((8, 8))
    np.testing.assert_allclose(C @ blk @ C.T, scipy_fft.dctn(blk, norm="ortho"), atol=1e-13)


def test_dct_denoise_rules():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (16, 24))[:16, :16]
    # threshold 0 keeps every nonzero coefficient -> identity
    y, _ = O.dct_denoise(x, 0.0)
    np.testing.assert_allclose(y, x, atol=1e-14)
    # Parseval: energy of kept coefficients == energy of output
    C = O.dct_matrix(8)
    y, _ = O.dct_denoise(x, 0.05)
    for a in (0, 8):
        for b in (0, 8):
            X = C @ x[a:a + 8, b:b + 8] @ C.T
            kept = np.abs(X) > 2.7 * 0.05
            kept[0, 0] = True
            assert abs((X[kept] ** 2).sum() - (y[a:a + 8, b:b + 8] ** 2).sum()) < 1e-12
    # a single AC basis function is kept iff its amplitude exceeds 2.7 sigma_BM;
    # the DC coefficient is always kept
    for amp, keep in [(1.0, True), (0.2, False)]:
        X = np.zeros((8, 8))
        X[0, 0] = 5.0
        X[2, 3] = amp
        blk = C.T @ X @ C
        out, margin = O.dct_denoise(blk, 0.1)
        expect = blk if keep else C.T @ np.where(np.arange(64).reshape(8, 8) == 0, X, 0) @ C
        np.testing.assert_allclose(out, expect, atol=1e-13)
        assert abs(margin - min(abs(amp - 0.27), 0.27)) < 1e-12


def test_projected_em_schedule():
    """Algorithm 2 with F: projections after every F-th iteration, sigma_BM follows
    Eq. (decaying_function): sigma_t = 2^(-1/10) sigma_{t-1}, sigma_1 = 1."""
    p = synth.make_problem(16, 2, 50, 0.3, seed=15)
    _, _, _, h = O.projected_em(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K, iters=7, F=2)
    assert len(h["LL"]) == 7
    np.testing.assert_allclose(h["sigma_bm"], [2.0 ** (-k / 10) for k in range(3)], rtol=1e-15)
    _, _, _, h0 = O.projected_em(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K, iters=3, F=0)
    assert h0["sigma_bm"] == []


# ---------------------------------------------------------------- error metric

def test_error_metric_brute_force_vs_fft():
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 1, (12, 12))
    assert O.error_metric(O.shift(x, 4, 7), x) < 1e-15
    xh = x + 0.1 * rng.standard_normal(x.shape)
    e1 = O.error_metric(O.shift(xh, 2, 9), x)
    e2 = FO.error_metric_fft(O.shift(xh, 2, 9), x)
    assert abs(e1 - e2) < 1e-12 and e1 > 0.01
    assert abs(O.snr(np.ones((4, 4)), 0.5) - 4.0) < 1e-15


def test_soft_threshold_is_the_l1_prox_and_nonexpansive():
    """Soft mode = prox of t*||AC coefficients||_1 per block: optimality conditions in the
    DCT domain hold, and the map is non-expansive (Assumption 2 of Sec. 4)."""
    rng = np.random.default_rng(8)
    C = O.dct_matrix(8)
    t = 0.3
    x = rng.uniform(0, 1, (16, 16))
    z, _ = O.dct_denoise(x, t / 2.7, mode="soft")
    for a in (0, 8):
        for b in (0, 8):
            X = C @ x[a:a + 8, b:b + 8] @ C.T
            Zc = C @ z[a:a + 8, b:b + 8] @ C.T
            assert abs(X[0, 0] - Zc[0, 0]) < 1e-12
            m = np.ones((8, 8), bool)
            m[0, 0] = False
            nz = m & (np.abs(Zc) > 1e-12)
            np.testing.assert_allclose(X[nz] - Zc[nz], t * np.sign(Zc[nz]), atol=1e-12)
            assert np.all(np.abs(X[m & ~nz]) <= t + 1e-12)
    for _ in range(5):
        a_ = rng.uniform(0, 1, (16, 16))
        b_ = a_ + 0.1 * rng.standard_normal((16, 16))
        da, _ = O.dct_denoise(a_, 0.1, mode="soft")
        db, _ = O.dct_denoise(b_, 0.1, mode="soft")
        assert np.linalg.norm(da - db) <= np.linalg.norm(a_ - b_) + 1e-12


def test_cycle_spinning_is_translation_equivariant():
    """Averaging over all block offsets makes the denoiser commute with every circular
    shift (exactly, up to rounding); threshold 0 is still the identity."""
    rng = np.random.default_rng(9)
    x = rng.uniform(0, 1, (16, 16))
    for mode in ("hard", "soft"):
        d0, _ = O.dct_denoise(x, 0.1, mode=mode, spin=True)
        d1, _ = O.dct_denoise(O.shift(x, 3, 5), 0.1, mode=mode, spin=True)
        np.testing.assert_allclose(d1, O.shift(d0, 3, 5), atol=1e-13)
        np.testing.assert_allclose(O.dct_denoise(x, 0.0, mode=mode, spin=True)[0], x,
                                   atol=1e-13)
    plain, _ = O.dct_denoise(x, 0.1)
    shifted, _ = O.dct_denoise(O.shift(x, 3, 5), 0.1)
    assert np.linalg.norm(shifted - O.shift(plain, 3, 5)) > 1e-3  # the plain one is not


# ---------------------------------------------------------------------------
# Online EM (reading R13)
# ---------------------------------------------------------------------------


def test_online_em_single_full_batch_is_one_em_iteration():
    p = synth.make_problem(12, 2, 60, 0.5, seed=77, init="uniform")
    xo, r1o, r2o, lls = O.online_em(p.y, [slice(0, p.N)], [0.3], p.x0, p.rho1_0, p.rho2_0,
                                    p.sigma, p.K)
    xe, r1e, r2e, lle, _ = O.em_iter(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
    np.testing.assert_allclose(xo, xe, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(r1o, r1e, rtol=1e-13)
    np.testing.assert_allclose(r2o, r2e, rtol=1e-13)
    assert abs(lls[0] - lle) < 1e-10 * abs(lle)


def test_online_statistics_average_to_the_full_data_ones():
    """With theta frozen, the stochastic-approximation steps with
    gamma_t = n_t / (n_0 + ... + n_t) over a partition of the observations give the
    full-data averages Z / N, c / N (checked against sums computed without batches)."""
    p = synth.make_problem(8, 2, 70, 0.4, seed=78, init="uniform")
    cuts = [0, 13, 40, 41, 70]
    S, seen = None, 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        Zb, cb, _ = O.batch_stats(p.y[a:b], p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
        seen += b - a
        S = O.sa_update(S, (Zb, cb), (b - a) / seen)
    # the full-data sums, term by term from the brute-force weights of each observation
    T = O.all_templates(p.x0, p.K)
    lp = O.log_prior(p.rho1_0, p.rho2_0)
    Y = p.y.reshape(p.N, -1).astype(np.float64)
    Z = np.zeros_like(S[0])
    c = np.zeros_like(S[1])
    for i in range(p.N):
        lg = -((Y[i][None, :] - T) ** 2).sum(axis=1) / (2 * p.sigma ** 2) + lp
        w = np.exp(lg - lg.max())
        w /= w.sum()
        Z += np.outer(w, Y[i])
        c += w
    np.testing.assert_allclose(S[0], Z / p.N, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(S[1], c / p.N, rtol=1e-11, atol=1e-15)


def test_online_em_gamma_one_forgets_the_past():
    """gamma = 1 keeps only the current batch: the step equals an EM iteration on that
    batch alone from the same theta."""
    p = synth.make_problem(8, 2, 50, 0.4, seed=79, init="uniform")
    b0, b1 = slice(0, 20), slice(20, 50)
    x1, r11, r21, _ = O.online_em(p.y, [b0], [1.0], p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
    x2, r12, r22, _ = O.online_em(p.y, [b0, b1], [1.0, 1.0], p.x0, p.rho1_0, p.rho2_0,
                                  p.sigma, p.K)
    xe, r1e, r2e, _, _ = O.em_iter(p.y[b1], x1, r11, r21, p.sigma, p.K)
    np.testing.assert_allclose(x2, xe, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(r12, r1e, rtol=1e-12)
