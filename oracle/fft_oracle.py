"""Second FP64 CPU oracle for one EM iteration, via the polyphase decomposition.

TEST INFRASTRUCTURE ONLY (same rules as ``srmra_oracle``: imported by tests, smoke and
the bench's CPU leg only; shares no code with the CUDA path).

It follows the proof of Theorem 1 (Sec. 2): with the K^2 sub-images
    x_r[l1, l2] = x[r1 + l1*K, r2 + l2*K],   r in [0,K)^2,
the template P R_s x of shift s = t*K - r (mod L, per axis) is the low-resolution
circular translate of x_r by t:  (P R_s x)[n] = x_r[n - t]  (indices mod l = L/K).
Hence
  * <y_i, P R_s x> is the circular cross-correlation of y_i with x_r at lag t,
    evaluated with 2D FFTs of size l x l;
  * ||P R_s x||^2 = ||x_r||^2 takes only K^2 values;
  * the right-hand side of Eq. (x_EM) on sub-image r is
        b_r[m] = sum_i sum_t w^{i,(r,t)} y_i[m + t],
    a correlation of the weight map w_{i,r,.} with y_i, also done with FFTs;
  * the diagonal of A on sub-image r is sum_t c[(r,t)] with c[s] = sum_i w^{i,s}.
The weights, rho update (Eq. rho_EM, marginals of the joint) and log-likelihood are
those of Sec. 2.  Observations are processed in chunks; the sums over i are
accumulated across chunks.  This formulation never builds the L^2 x l^2 template
matrix nor the N x L^2 weight matrix, so it runs at the full workload sizes.
"""
from __future__ import annotations

import numpy as np


def polyphase(x: np.ndarray, K: int) -> np.ndarray:
    """Sub-images xr[r1, r2, l1, l2] = x[r1 + l1*K, r2 + l2*K]."""
    L = x.shape[0]
    l = L // K
    return np.asarray(x, np.float64).reshape(l, K, l, K).transpose(1, 3, 0, 2)


def unpolyphase(xr: np.ndarray) -> np.ndarray:
    """Inverse of `polyphase`."""
    K, _, l, _ = xr.shape
    return xr.transpose(2, 0, 3, 1).reshape(l * K, l * K)


def shift_of(K: int, L: int) -> np.ndarray:
    """S[r, t] = (t*K - r) mod L: the full-resolution shift of phase r and lag t."""
    l = L // K
    r = np.arange(K)[:, None]
    t = np.arange(l)[None, :]
    return (t * K - r) % L


def _estep_sums(Y, Xf, nu, lp, inv2s2, K, l, chunk):
    """The sums over the observations Y (n x l x l, float64) that the M-step reads:
    G[r] = sum_i conj(FFT2(w_{i,r,.})) * FFT2(y_i), c[r, t] = sum_i w^{i,(r,t)}, and
    lse_i (Eqs. weights_EM and likelihood_EM, Sec. 2)."""
    N = Y.shape[0]
    G = np.zeros((K, K, l, l), dtype=np.complex128)
    c = np.zeros((K, K, l, l))
    lse = np.empty(N)
    for a in range(0, N, chunk):
        Yc = Y[a:a + chunk]
        n = Yc.shape[0]
        Yf = np.fft.fft2(Yc)                               # (n,l,l)
        corr = np.fft.ifft2(Yf[:, None, None] * np.conj(Xf)[None]).real   # (n,K,K,l,l)
        yy = (Yc * Yc).sum(axis=(1, 2))
        d = yy[:, None, None, None, None] - 2.0 * corr + nu[None, :, :, None, None]
        logits = (-d * inv2s2 + lp[None]).reshape(n, -1)
        m = logits.max(axis=1)
        with np.errstate(invalid="ignore"):
            lse_c = m + np.log(np.exp(logits - m[:, None]).sum(axis=1))
        W = np.exp(logits - lse_c[:, None]).reshape(n, K, K, l, l)
        lse[a:a + n] = lse_c
        c += W.sum(axis=0)
        G += (np.conj(np.fft.fft2(W)) * Yf[:, None, None]).sum(axis=0)
    return G, c, lse


def em_iter_fft(Y, x, rho1, rho2, sigma, K, chunk: int | None = None, workers: int = 1):
    """One EM iteration. Returns (x_{t+1}, rho1_{t+1}, rho2_{t+1}, LL(theta_t), aux)
    with aux = dict(lse, c (joint, L x L), b (L x L), A (L x L)).

    workers > 1 splits the observations into that many contiguous ranges whose sums
    over i (a plain regrouping of the sums in Eqs. x_EM and rho_EM) are formed by
    threads and added in range order, so that large problems check in seconds."""
    x = np.asarray(x, np.float64)
    L = x.shape[0]
    l = L // K
    N = Y.shape[0]
    Y = np.asarray(Y, np.float64).reshape(N, l, l)
    if chunk is None:
        chunk = max(1, (1 << 26) // (L * L * 16))
    xr = polyphase(x, K)                                   # (K,K,l,l)
    Xf = np.fft.fft2(xr)
    nu = (xr * xr).sum(axis=(2, 3))                        # ||x_r||^2, (K,K)
    S = shift_of(K, L)                                     # (K, l)
    with np.errstate(divide="ignore"):
        lr1 = np.log(np.asarray(rho1, np.float64))[S]      # (K, l) over (r1, t1)
        lr2 = np.log(np.asarray(rho2, np.float64))[S]      # (K, l) over (r2, t2)
    lp = lr1[:, None, :, None] + lr2[None, :, None, :]     # (K,K,l,l)
    inv2s2 = 1.0 / (2.0 * sigma * sigma)
    workers = max(1, min(int(workers), N))
    if workers == 1:
        G, c, lse = _estep_sums(Y, Xf, nu, lp, inv2s2, K, l, chunk)
    else:
        from concurrent.futures import ThreadPoolExecutor
        cuts = [N * k // workers for k in range(workers + 1)]
        with ThreadPoolExecutor(workers) as ex:
            parts = list(ex.map(lambda k: _estep_sums(Y[cuts[k]:cuts[k + 1]], Xf, nu, lp,
                                                      inv2s2, K, l, chunk),
                                range(workers)))
        G = parts[0][0].copy()
        c = parts[0][1].copy()
        for Gp, cp_, _ in parts[1:]:
            G += Gp
            c += cp_
        lse = np.concatenate([q[2] for q in parts])
    b_r = np.fft.ifft2(G).real                             # (K,K,l,l)
    A_r = c.sum(axis=(2, 3))                               # (K,K)
    xr_new = np.where(A_r[:, :, None, None] > 0,
                      b_r / np.where(A_r > 0, A_r, 1.0)[:, :, None, None], xr)
    cs = np.zeros((L, L))
    cs[S[:, None, :, None], S[None, :, None, :]] = c
    rho_joint = cs / cs.sum()
    b = unpolyphase(b_r)
    A = unpolyphase(np.broadcast_to(A_r[:, :, None, None], (K, K, l, l)))
    return (unpolyphase(xr_new), rho_joint.sum(axis=1), rho_joint.sum(axis=0),
            float(lse.sum()), dict(lse=lse, c=cs.ravel(), b=b, A=A))


def error_metric_fft(xhat: np.ndarray, x: np.ndarray) -> float:
    """error(xhat) = min_s ||R_s xhat - x|| / ||x|| using an FFT cross-correlation:
    ||R_s xhat - x||^2 = ||xhat||^2 + ||x||^2 - 2 <R_s xhat, x>."""
    xhat = np.asarray(xhat, np.float64)
    x = np.asarray(x, np.float64)
    corr = np.fft.ifft2(np.fft.fft2(x) * np.conj(np.fft.fft2(xhat))).real
    d2 = (xhat * xhat).sum() + (x * x).sum() - 2.0 * corr.max()
    return float(np.sqrt(max(d2, 0.0)) / np.linalg.norm(x))
