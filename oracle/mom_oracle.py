"""FP64 CPU oracle for projected MoM in 2D SR-MRA (Algorithm 1 of the paper).

TEST INFRASTRUCTURE ONLY (same rules as ``srmra_oracle``: imported by tests, smoke and
the bench's CPU leg only; shares no code with the CUDA path).

  * Eq. (empiric_MOM), D = 2:  M1^ = (1/N) sum_i y_i,  M2^ = (1/N) sum_i y_i y_i^T.
  * The moments of the model (Sec. 2):  M1 = P C_x rho,
    M2 = P C_x D_rho C_x^T P^T + sigma^2 P P^T, i.e. with the templates
    t_s = P R_s x (the columns of C_x, sampled) and the joint rho_s = rho1[s1] rho2[s2]:
        M1 = sum_s rho_s t_s,   M2 = sum_s rho_s t_s t_s^T + sigma^2 I   (P P^T = I).
  * Eq. (LS_SR):  f = ||M2 - M2^||_F^2 + lambda ||M1 - M1^||^2,
    lambda = 1 / (L^2 (1 + sigma^2)) as the paper sets it.
  * Gradients (derived here; checked against finite differences in the tests), with
    R = M2 - M2^ (symmetric) and r = M1 - M1^:
        df/drho_s = 2 t_s^T R t_s + 2 lambda t_s^T r,
        df/dx     = sum_s rho_s (P R_s)^T (4 R t_s + 2 lambda r),
    and for the product form df/drho1[a] = sum_b df/drho_(a,b) rho2[b], likewise rho2.
  * Algorithm 1 with the reading
    R14 the inner minimiser of Algorithm 1 (F quasi-Newton iterations per outer step, for
        which the paper allows any gradient method) is taken as F steps of the fixed-step
        gradient iteration the paper analyses (Sec. 4, Eq. (pgm)):
        x <- x - mu_x df/dx; rho1, rho2 <- their Euclidean projections onto the
        probability simplex after a step mu_rho of their gradients; then
        x <- D(x, sigma_BM) and sigma_BM <- 2^(-1/10) sigma_BM (Eq. decaying_function).
"""
from __future__ import annotations

import numpy as np

from oracle import srmra_oracle as O


def empirical_moments(Y: np.ndarray):
    """Eq. (empiric_MOM) for d = 1, 2 over the flattened observations."""
    Y = np.asarray(Y, np.float64).reshape(Y.shape[0], -1)
    N = Y.shape[0]
    return Y.sum(axis=0) / N, (Y.T @ Y) / N


def model_moments(x, rho1, rho2, sigma, K):
    """M1 = sum_s rho_s t_s, M2 = sum_s rho_s t_s t_s^T + sigma^2 I."""
    T = O.all_templates(np.asarray(x, np.float64), K)          # (L^2, l^2)
    rho = np.outer(rho1, rho2).ravel()
    M1 = rho @ T
    M2 = (T * rho[:, None]).T @ T + sigma ** 2 * np.eye(T.shape[1])
    return M1, M2


def mom_lambda(L: int, sigma: float) -> float:
    return 1.0 / (L * L * (1.0 + sigma * sigma))


def objective(x, rho1, rho2, M1h, M2h, sigma, K) -> float:
    """Eq. (LS_SR)."""
    L = np.asarray(x).shape[0]
    M1, M2 = model_moments(x, rho1, rho2, sigma, K)
    return float(((M2 - M2h) ** 2).sum() + mom_lambda(L, sigma) * ((M1 - M1h) ** 2).sum())


def gradient(x, rho1, rho2, M1h, M2h, sigma, K):
    """(f, df/dx (L x L), df/drho1 (L), df/drho2 (L))."""
    x = np.asarray(x, np.float64)
    L = x.shape[0]
    l = L // K
    lam = mom_lambda(L, sigma)
    T = O.all_templates(x, K)
    rho = np.outer(rho1, rho2).ravel()
    M1 = rho @ T
    M2 = (T * rho[:, None]).T @ T + sigma ** 2 * np.eye(T.shape[1])
    R = M2 - M2h
    r = M1 - M1h
    f = float((R ** 2).sum() + lam * (r ** 2).sum())
    U = T @ R                                                   # rows R t_s
    g_rho = 2.0 * (U * T).sum(axis=1) + 2.0 * lam * (T @ r)     # df/drho_s
    G = g_rho.reshape(L, L)
    g1 = G @ np.asarray(rho2, np.float64)
    g2 = G.T @ np.asarray(rho1, np.float64)
    gx = np.zeros((L, L))
    for s1 in range(L):
        for s2 in range(L):
            s = s1 * L + s2
            v = rho[s] * (4.0 * U[s] + 2.0 * lam * r)
            gx += O.template_adjoint(v.reshape(l, l), K, s1, s2)
    return f, gx, g1, g2


def project_simplex(v: np.ndarray) -> np.ndarray:
    """Euclidean projection onto {w >= 0, sum w = 1}: with u = v sorted decreasingly and
    k the largest index with u_k > (u_1 + ... + u_k - 1) / k, the threshold is
    tau = (u_1 + ... + u_k - 1) / k and w = max(v - tau, 0)."""
    v = np.asarray(v, np.float64)
    u = np.sort(v)[::-1]
    css = np.cumsum(u)
    k = np.arange(1, v.size + 1)
    ok = u - (css - 1.0) / k > 0
    kk = k[ok][-1]
    tau = (css[kk - 1] - 1.0) / kk
    return np.maximum(v - tau, 0.0)


def projected_mom(Y, x0, rho1, rho2, sigma, K, iters, F, mu_x, mu_rho, sigma_bm1=1.0,
                  decay=2.0 ** -0.1):
    """Algorithm 1 with reading R14.  Returns (x, rho1, rho2, objective per step)."""
    M1h, M2h = empirical_moments(Y)
    x = np.asarray(x0, np.float64)
    r1 = np.asarray(rho1, np.float64)
    r2 = np.asarray(rho2, np.float64)
    sbm = float(sigma_bm1)
    fs = []
    for t in range(iters):
        f, gx, g1, g2 = gradient(x, r1, r2, M1h, M2h, sigma, K)
        fs.append(f)
        x = x - mu_x * gx
        r1 = project_simplex(r1 - mu_rho * g1)
        r2 = project_simplex(r2 - mu_rho * g2)
        if F > 0 and (t + 1) % F == 0:
            x, _ = O.dct_denoise(x, sbm)
            sbm *= decay
    return x, r1, r2, fs
