"""Plain FP64 CPU oracle for projected EM in 2D SR-MRA (Shani, Tirer, Giryes, Bendory).

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline / reference leg, and
by nothing else.  It shares no code with the CUDA path (``paper_2204_04754_gb300``),
and it never imports it.

It computes, in float64, what the paper defines:

  * Eq. (1), data model:  y_i = P R_{s_i} x + eps_i, with
        (R_s x)[q1,q2] = x[q1 - s1, q2 - s2]   (indices mod L, s1 on axis 0)
        (P z)[n1,n2]   = z[n1*K, n2*K].
  * Eq. (likelihood_EM):  log p = sum_i log sum_s rho[s] exp(-||y_i - P R_s x||^2 / (2 sigma^2)),
    without the Gaussian normalising constant (the paper omits it too).
  * Eq. (Q) and Eq. (weights_EM): w^{i,s} = C_i rho[s] exp(-||y_i - P R_s x||^2/(2 sigma^2)),
    sum_s w^{i,s} = 1.
  * Eq. (x_EM): A x = b with A = sum_{i,s} w R_s^T P^T P R_s, b = sum_{i,s} w R_s^T P^T y_i.
  * Eq. (rho_EM): rho[s] = sum_i w^{i,s} / sum_i sum_s' w^{i,s'}.
  * Eq. (decaying_function): sigma_BM_t = 2^(-1/10) sigma_BM_{t-1}, sigma_BM_1 = 1.
  * Algorithm 2 (projected EM): F EM steps, then x <- D(x, sigma_BM), then decay.

Readings where the paper is silent or ambiguous:
  R1  "P^{-1}" in Eq. (x_EM) is read as P^T (zero-filling adjoint); P has no inverse.
  R2  rho is the product rho1 (x) rho2 (Sec. 2 parameter set, and the diagonal of D_rho
      in the moment formulas); Eq. (rho_EM) is evaluated for the joint, and rho1, rho2
      are its marginals.
  R3  shift indices 1..L in the sums are taken as 0..L-1 (the same set modulo L).
  R4  s1 acts on the first array index (rows), s2 on the second; arrays are row-major.
  R5  the subscript w_k in Eq. (rho_EM) is the current iteration's weights w_t.
  R6  a pixel with zero coverage (A[q] = 0) keeps its previous value.
  R7  rho[s] = 0 gives log rho = -inf, logit -inf, weight exactly 0.
  R8  the log-likelihood omits the constant -(N l^2 / 2) log(2 pi sigma^2).
  R9  the denoiser D is a block-DCT hard threshold (BM3D is third-party and not part of
      the method): non-overlapping 8x8 blocks anchored at pixel (0,0), orthonormal 2D
      DCT-II, the DC coefficient always kept, an AC coefficient kept iff
      |c| > 2.7 * sigma_BM (ties are zeroed), no clipping.
  R10 the projection runs after the M-step of every F-th iteration; F = 0 means none.
  R11 the loops of Algorithms 1 and 2 run for a fixed number of iterations (the paper
      leaves the stopping rule open).
  R13 online EM (the online strategy the paper suggests for large N, Sec. 6, without an
      algorithm): mini-batch EM with stochastic-approximation sufficient statistics.
      The statistics of Eqs. (x_EM) and (rho_EM) are the per-shift sums
      Z[s] = sum_i w^{i,s} y_i and c[s] = sum_i w^{i,s}; step t takes a batch B_t,
      averages them over it (Z_B / |B_t|, c_B / |B_t|), sets
      S_t = (1 - gamma_t) S_{t-1} + gamma_t S_{B_t} (gamma_0 = 1), and runs the M-step
      on S_t.  The M-step is scale-free in (Z, c), so a single batch of all N
      observations with gamma = 1 is one EM iteration.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Forward operator, Eq. (1)
# ---------------------------------------------------------------------------


def shift(x: np.ndarray, s1: int, s2: int) -> np.ndarray:
    """R_s x: (R_s x)[q] = x[q - s] with indices mod L (circular translation)."""
    return np.roll(x, shift=(s1, s2), axis=(0, 1))


def sample(z: np.ndarray, K: int) -> np.ndarray:
    """P z: the L/K x L/K equally spaced samples z[n1*K, n2*K]."""
    return z[::K, ::K]


def sample_adjoint(v: np.ndarray, K: int) -> np.ndarray:
    """P^T v: zero-filled upsampling, v[n] placed at pixel n*K (reading R1)."""
    l = v.shape[0]
    out = np.zeros((l * K, l * K), dtype=np.float64)
    out[::K, ::K] = v
    return out


def template(x: np.ndarray, K: int, s1: int, s2: int) -> np.ndarray:
    """P R_s x, the noiseless observation for shift s = (s1, s2)."""
    return sample(shift(x, s1, s2), K)


def template_adjoint(v: np.ndarray, K: int, s1: int, s2: int) -> np.ndarray:
    """(P R_s)^T v = R_s^T P^T v = R_{-s} P^T v (R_s is a permutation)."""
    return shift(sample_adjoint(v, K), -s1, -s2)


def all_templates(x: np.ndarray, K: int) -> np.ndarray:
    """Rows T[s] = vec(P R_s x) for s = s1*L + s2 (row-major shift index)."""
    x = np.asarray(x, dtype=np.float64)
    L = x.shape[0]
    l = L // K
    T = np.empty((L * L, l * l))
    for s1 in range(L):
        for s2 in range(L):
            T[s1 * L + s2] = template(x, K, s1, s2).ravel()
    return T


# ---------------------------------------------------------------------------
# E-step: Eq. (likelihood_EM), Eq. (weights_EM)
# ---------------------------------------------------------------------------


def log_prior(rho1: np.ndarray, rho2: np.ndarray) -> np.ndarray:
    """log rho[s] = log rho1[s1] + log rho2[s2], flattened as s = s1*L + s2 (R2, R7)."""
    with np.errstate(divide="ignore"):
        return (np.log(np.asarray(rho1, np.float64))[:, None]
                + np.log(np.asarray(rho2, np.float64))[None, :]).ravel()


def sq_distances(Y: np.ndarray, T: np.ndarray, literal: bool = False) -> np.ndarray:
    """d[i,s] = ||y_i - T_s||^2.

    literal=True forms the difference elementwise (the definition as printed);
    literal=False uses ||y||^2 - 2<y,T> + ||T||^2 with a library matmul for <y,T>.
    The two are the same number up to rounding order; a test pins one to the other.
    """
    Y = np.asarray(Y, np.float64)
    if literal:
        return ((Y[:, None, :] - T[None, :, :]) ** 2).sum(axis=2)
    return ((Y * Y).sum(1)[:, None] - 2.0 * (Y @ T.T) + (T * T).sum(1)[None, :])


def logsumexp_rows(a: np.ndarray) -> np.ndarray:
    """log sum_j exp(a[i,j]) per row, stable; rows may hold -inf entries (R7)."""
    m = a.max(axis=1)
    with np.errstate(invalid="ignore"):
        return m + np.log(np.exp(a - m[:, None]).sum(axis=1))


def estep(Y: np.ndarray, x: np.ndarray, rho1: np.ndarray, rho2: np.ndarray,
          sigma: float, K: int, literal: bool = False):
    """E-step of Sec. 2: logits, per-observation log-normaliser, weights, log-likelihood.

    Returns (W, lse, LL) where W[i,s] = w^{i,s} of Eq. (weights_EM), lse[i] is
    log sum_s rho[s] exp(-d[i,s]/(2 sigma^2)) and LL = sum_i lse[i] is Eq.
    (likelihood_EM) for the current parameters (reading R8).
    """
    Y = np.asarray(Y, np.float64).reshape(Y.shape[0], -1)
    T = all_templates(x, K)
    d = sq_distances(Y, T, literal=literal)
    logits = -d / (2.0 * sigma * sigma) + log_prior(rho1, rho2)[None, :]
    lse = logsumexp_rows(logits)
    W = np.exp(logits - lse[:, None])
    return W, lse, float(lse.sum())


def loglik(Y, x, rho1, rho2, sigma, K, chunk: int | None = None) -> float:
    """Eq. (likelihood_EM) (without its constant) for parameters (x, rho)."""
    Y = np.asarray(Y, np.float64).reshape(Y.shape[0], -1)
    T = all_templates(x, K)
    lp = log_prior(rho1, rho2)[None, :]
    total = 0.0
    step = Y.shape[0] if chunk is None else chunk
    for a in range(0, Y.shape[0], step):
        d = sq_distances(Y[a:a + step], T)
        total += float(logsumexp_rows(-d / (2.0 * sigma * sigma) + lp).sum())
    return total


def q_function(Y, W, x, rho1, rho2, sigma, K) -> float:
    """Eq. (Q): sum_{i,s} w^{i,s} (log rho[s] - ||y_i - P R_s x||^2 / (2 sigma^2))."""
    Y = np.asarray(Y, np.float64).reshape(Y.shape[0], -1)
    T = all_templates(x, K)
    d = sq_distances(Y, T)
    lp = log_prior(rho1, rho2)[None, :]
    with np.errstate(invalid="ignore"):
        term = np.where(W > 0, W * (lp - d / (2.0 * sigma * sigma)), 0.0)
    return float(term.sum())


# ---------------------------------------------------------------------------
# M-step: Eq. (x_EM), Eq. (rho_EM)
# ---------------------------------------------------------------------------


def mstep_from_sums(Z: np.ndarray, c: np.ndarray, x_prev: np.ndarray, K: int):
    """M-step from the per-shift sums Z[s] = sum_i w^{i,s} y_i and c[s] = sum_i w^{i,s}.

    b = sum_s (P R_s)^T Z[s] and A = sum_s c[s] (P R_s)^T (P R_s) 1 (A is the diagonal
    of the matrix in Eq. (x_EM), since R_s^T P^T P R_s is a 0/1 diagonal projector);
    x = b / A where A > 0, else the previous value (R6).  rho from Eq. (rho_EM) on the
    joint, then its marginals (R2).  Returns (x, rho1, rho2, b, A).
    """
    x_prev = np.asarray(x_prev, np.float64)
    L = x_prev.shape[0]
    l = L // K
    b = np.zeros((L, L))
    A = np.zeros((L, L))
    ones = np.ones((l, l))
    for s1 in range(L):
        for s2 in range(L):
            s = s1 * L + s2
            b += template_adjoint(Z[s].reshape(l, l), K, s1, s2)
            A += c[s] * template_adjoint(ones, K, s1, s2)
    x = np.where(A > 0, b / np.where(A > 0, A, 1.0), x_prev)
    rho_joint = (c / c.sum()).reshape(L, L)
    return x, rho_joint.sum(axis=1), rho_joint.sum(axis=0), b, A


def mstep(Y: np.ndarray, W: np.ndarray, x_prev: np.ndarray, K: int):
    """M-step given the full weight matrix W (N x L^2)."""
    Y = np.asarray(Y, np.float64).reshape(Y.shape[0], -1)
    Z = W.T @ Y
    c = W.sum(axis=0)
    return mstep_from_sums(Z, c, x_prev, K)


def em_iter(Y, x, rho1, rho2, sigma, K, chunk: int | None = None, literal: bool = False):
    """One EM iteration theta_t -> theta_{t+1}.

    Returns (x_{t+1}, rho1_{t+1}, rho2_{t+1}, LL(theta_t), aux) where aux holds lse,
    c, b, A.  With `chunk`, observations are processed `chunk` at a time and the sums
    over i (Z, c, LL) are accumulated across chunks; each chunk evaluates the same
    formulas.
    """
    Y = np.asarray(Y, np.float64).reshape(Y.shape[0], -1)
    N = Y.shape[0]
    step = N if chunk is None else chunk
    L = np.asarray(x).shape[0]
    S = L * L
    Z = np.zeros((S, Y.shape[1]))
    c = np.zeros(S)
    lse_all = np.empty(N)
    for a in range(0, N, step):
        W, lse, _ = estep(Y[a:a + step], x, rho1, rho2, sigma, K, literal=literal)
        Z += W.T @ Y[a:a + step]
        c += W.sum(axis=0)
        lse_all[a:a + step] = lse
    xn, r1, r2, b, A = mstep_from_sums(Z, c, x, K)
    return xn, r1, r2, float(lse_all.sum()), dict(lse=lse_all, c=c, b=b, A=A)


# ---------------------------------------------------------------------------
# Denoiser: block-DCT hard threshold (reading R9)
# ---------------------------------------------------------------------------


def dct_matrix(B: int = 8) -> np.ndarray:
    """Orthonormal DCT-II matrix C[k,n] = a_k cos(pi (2n+1) k / (2B))."""
    n = np.arange(B)
    k = n[:, None]
    C = np.cos(math.pi * (2 * n[None, :] + 1) * k / (2.0 * B))
    C[0, :] *= math.sqrt(1.0 / B)
    C[1:, :] *= math.sqrt(2.0 / B)
    return C


def dct_denoise(x: np.ndarray, sigma_bm: float, thr: float = 2.7, B: int = 8,
                mode: str = "hard", spin: bool = False):
    """D(x, sigma_BM): per BxB block, X = C x C^T, threshold the AC coefficients at
    t = thr*sigma_BM, keep DC, invert.
      mode 'hard': keep an AC coefficient iff |X| > t (reading R9);
      mode 'soft': X <- sign(X) max(|X| - t, 0), the proximal operator of t*||AC(DCT x)||_1
                   on each block (a convex prox, the setting of Sec. 4's Assumption 2);
      spin:        average of the block denoiser over all B^2 circular offsets of the block
                   grid (cycle spinning): D(x) = mean_d R_{-d} D_0(R_d x).
    Returns (x_denoised, margin) with margin = min over AC coefficients of | |X| - t |
    (the distance to a hard-threshold flip)."""
    x = np.asarray(x, np.float64)
    L = x.shape[0]
    if L % B:
        raise ValueError("image side must be a multiple of the block size")
    if spin:
        acc = np.zeros_like(x)
        margin = math.inf
        for d1 in range(B):
            for d2 in range(B):
                y, mg = dct_denoise(shift(x, d1, d2), sigma_bm, thr, B, mode, False)
                acc += shift(y, -d1, -d2)
                margin = min(margin, mg)
        return acc / (B * B), margin
    C = dct_matrix(B)
    t = thr * sigma_bm
    out = np.empty_like(x)
    margin = math.inf
    ac = np.ones((B, B), dtype=bool)
    ac[0, 0] = False
    for a in range(0, L, B):
        for b in range(0, L, B):
            X = C @ x[a:a + B, b:b + B] @ C.T
            if mode == "hard":
                keep = np.abs(X) > t
                keep[0, 0] = True
                Xd = X * keep
            elif mode == "soft":
                Xd = np.sign(X) * np.maximum(np.abs(X) - t, 0.0)
                Xd[0, 0] = X[0, 0]
            else:
                raise ValueError(mode)
            margin = min(margin, float(np.min(np.abs(np.abs(X[ac]) - t))))
            out[a:a + B, b:b + B] = C.T @ Xd @ C
    return out, margin


# ---------------------------------------------------------------------------
# Algorithm 2: projected EM
# ---------------------------------------------------------------------------


def projected_em(Y, x0, rho1, rho2, sigma, K, iters, F, sigma_bm1=1.0,
                 decay=2.0 ** -0.1, chunk=None, em_step=None, mode="hard", spin=False,
                 thr=2.7):
    """Algorithm 2: repeat {F EM steps (Eqs. weights_EM, x_EM, rho_EM);
    x <- D(x, sigma_BM); sigma_BM <- decay * sigma_BM}, for `iters` EM steps total.
    F = 0 runs plain EM (no projection).  Returns (x, rho1, rho2, history) where
    history holds LL(theta_t) per iteration, the sigma_BM used per projection and the
    smallest threshold margin met."""
    step = em_step or (lambda x_, r1_, r2_: em_iter(Y, x_, r1_, r2_, sigma, K, chunk=chunk))
    x = np.asarray(x0, np.float64)
    r1 = np.asarray(rho1, np.float64)
    r2 = np.asarray(rho2, np.float64)
    sbm = float(sigma_bm1)
    hist = dict(LL=[], sigma_bm=[], margin=math.inf)
    for t in range(iters):
        x, r1, r2, LL, _ = step(x, r1, r2)
        hist["LL"].append(LL)
        if F > 0 and (t + 1) % F == 0:
            x, mg = dct_denoise(x, sbm, thr=thr, mode=mode, spin=spin)
            hist["sigma_bm"].append(sbm)
            hist["margin"] = min(hist["margin"], mg)
            sbm *= decay
    return x, r1, r2, hist


# ---------------------------------------------------------------------------
# Online EM (reading R13)
# ---------------------------------------------------------------------------


def batch_stats(Yb, x, rho1, rho2, sigma, K):
    """E-step on a batch: the per-observation averages Z_B / n, c_B / n of the
    sufficient statistics, and the batch log-likelihood terms lse_i."""
    Yb = np.asarray(Yb, np.float64).reshape(Yb.shape[0], -1)
    n = Yb.shape[0]
    W, lse, _ = estep(Yb, x, rho1, rho2, sigma, K)
    return (W.T @ Yb) / n, W.sum(axis=0) / n, lse


def sa_update(S, Sb, gamma):
    """Stochastic-approximation step S <- (1 - gamma) S + gamma S_B on (Z, c)."""
    if S is None:
        return Sb
    return tuple((1.0 - gamma) * a + gamma * b for a, b in zip(S, Sb))


def online_em(Y, batches, gammas, x0, rho1, rho2, sigma, K, F=0, sigma_bm1=1.0,
              decay=2.0 ** -0.1):
    """Online EM (R13): for each step t, an E-step on the observations Y[batches[t]]
    (an index array or a slice), the update of the statistics with gammas[t]
    (gamma_0 is taken as 1), the M-step of Eqs. (x_EM), (rho_EM) on them, and every
    F-th step the projection of Algorithm 2.  Returns (x, rho1, rho2, batch LLs)."""
    x = np.asarray(x0, np.float64)
    r1 = np.asarray(rho1, np.float64)
    r2 = np.asarray(rho2, np.float64)
    S = None
    lls = []
    sbm = float(sigma_bm1)
    for t, (bt, g) in enumerate(zip(batches, gammas)):
        Zb, cb, lse = batch_stats(Y[bt], x, r1, r2, sigma, K)
        S = sa_update(S, (Zb, cb), 1.0 if t == 0 else g)
        x, r1, r2, _, _ = mstep_from_sums(S[0], S[1], x, K)
        lls.append(float(lse.sum()))
        if F > 0 and (t + 1) % F == 0:
            x, _ = dct_denoise(x, sbm)
            sbm *= decay
    return x, r1, r2, lls


# ---------------------------------------------------------------------------
# Reporting quantities (Sec. 5)
# ---------------------------------------------------------------------------


def error_metric(xhat: np.ndarray, x: np.ndarray) -> float:
    """error(xhat) = min_s ||R_s xhat - x||_F / ||x||_F, brute force over all L^2 shifts."""
    xhat = np.asarray(xhat, np.float64)
    x = np.asarray(x, np.float64)
    L = x.shape[0]
    best = math.inf
    for s1 in range(L):
        for s2 in range(L):
            best = min(best, float(np.linalg.norm(shift(xhat, s1, s2) - x)))
    return best / float(np.linalg.norm(x))


def snr(x: np.ndarray, sigma: float) -> float:
    """SNR = ||x||_F^2 / (L^2 sigma^2)."""
    x = np.asarray(x, np.float64)
    return float((x * x).sum() / (x.size * sigma * sigma))
