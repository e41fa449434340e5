"""Seeded synthetic inputs for 2D SR-MRA (shared by the oracle tests, the GPU tests
and the benchmark).

This module only *generates data*; it holds none of the EM arithmetic.  It draws

  * a ground-truth image x in [0,1]^{L x L}: a sum of periodic (wrapped) Gaussian
    blobs, optionally plus a layer of wrapped axis-aligned rectangles, min-max
    scaled to [0,1] (the paper's images have pixel values in [0,1], Sec. 5);
  * shift distributions rho1, rho2 on the L-simplex: two-component wrapped,
    discretised Gaussian mixtures (non-uniform, as the model of Sec. 1 allows);
  * N observations following the data model of Eq. (1):
        y_i[n1,n2] = x[(n1*K - s1_i) mod L, (n2*K - s2_i) mod L] + eps_i[n1,n2],
    with s1_i ~ rho1, s2_i ~ rho2 i.i.d. and eps_i ~ N(0, sigma^2) i.i.d.;
  * the initial guess used by the workloads: nearest-neighbour upsampling of the
    mean observation, and uniform rho.

Everything is drawn in float64 from numpy's PCG64 and handed out as float32 bytes
(images, observations) and float64 (distributions), so that every consumer ingests
the same values.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 20220411


def seed_for(config: int, instance: int = 0) -> int:
    """Seed convention: base seed + 100 * config + instance."""
    return BASE_SEED + 100 * int(config) + int(instance)


def _wrapped_gauss_1d(L: int, mu: float, std: float) -> np.ndarray:
    """Periodic Gaussian bump on Z_L (sum over a few periods)."""
    n = np.arange(L, dtype=np.float64)
    out = np.zeros(L)
    for k in range(-3, 4):
        out += np.exp(-0.5 * ((n - mu + k * L) / std) ** 2)
    return out


def blob_image(L: int, n_blobs: int, rng: np.random.Generator,
               n_rects: int = 0) -> np.ndarray:
    """Sum of wrapped Gaussian blobs (+ optional wrapped rectangles), scaled to [0,1]."""
    img = np.zeros((L, L))
    for _ in range(n_blobs):
        c1, c2 = rng.uniform(0, L, size=2)
        std = rng.uniform(1.0, 3.0)
        amp = rng.uniform(0.5, 1.0)
        img += amp * np.outer(_wrapped_gauss_1d(L, c1, std), _wrapped_gauss_1d(L, c2, std))
    for _ in range(n_rects):
        lo, hi = max(1, L // 16), max(1, L // 4)
        h, w = rng.integers(lo, hi + 1, size=2)
        a1, a2 = rng.integers(0, L, size=2)
        val = rng.uniform(0.0, 1.0)
        rows = (a1 + np.arange(h)) % L
        cols = (a2 + np.arange(w)) % L
        img[np.ix_(rows, cols)] += val
    mn, mx = img.min(), img.max()
    if mx > mn:
        img = (img - mn) / (mx - mn)
    return img


def mixture_distribution(L: int, rng: np.random.Generator) -> np.ndarray:
    """Two-component wrapped discretised Gaussian mixture on {0..L-1}, normalised."""
    w = rng.uniform(0.2, 0.8, size=2)
    w = w / w.sum()
    p = np.zeros(L)
    for k in range(2):
        mu = rng.uniform(0, L)
        std = rng.uniform(L / 16.0, L / 6.0)
        g = _wrapped_gauss_1d(L, mu, std)
        p += w[k] * g / g.sum()
    return p / p.sum()


def uniform_simplex_draw(L: int, rng: np.random.Generator) -> np.ndarray:
    """The paper's alternative: U[0,1] entries normalised onto the simplex (Sec. 5)."""
    p = rng.uniform(0.0, 1.0, size=L)
    return p / p.sum()


def observe(x: np.ndarray, K: int, s1: np.ndarray, s2: np.ndarray,
            noise: np.ndarray) -> np.ndarray:
    """Data model of Eq. (1): sample x on the K-spaced grid after a circular shift."""
    L = x.shape[0]
    l = L // K
    n = np.arange(l) * K
    rows = (n[None, :] - s1[:, None]) % L          # (N, l)
    cols = (n[None, :] - s2[:, None]) % L          # (N, l)
    clean = x[rows[:, :, None], cols[:, None, :]]  # (N, l, l)
    return clean + noise


@dataclasses.dataclass
class Problem:
    """One seeded SR-MRA instance (float32 image/observations, float64 rho)."""
    L: int
    K: int
    N: int
    sigma: float
    x_true: np.ndarray      # (L, L) float32
    rho1_true: np.ndarray   # (L,) float64
    rho2_true: np.ndarray   # (L,) float64
    s1: np.ndarray          # (N,) int64
    s2: np.ndarray          # (N,) int64
    y: np.ndarray           # (N, l, l) float32, C-contiguous
    x0: np.ndarray          # (L, L) float32 initial guess
    rho1_0: np.ndarray      # (L,) float64 initial guess (uniform)
    rho2_0: np.ndarray

    @property
    def l(self) -> int:
        return self.L // self.K


def make_problem(L: int, K: int, N: int, sigma: float, seed: int,
                 n_blobs: int = 6, n_rects: int = 0,
                 init: str = "mean_upsample") -> Problem:
    """Draw one instance. `init` = 'mean_upsample' (workload default) or
    'uniform' (the paper's experimental init: U[0,1] pixels min-max scaled)."""
    if L % K:
        raise ValueError("K must divide L")
    rng = np.random.Generator(np.random.PCG64(seed))
    x = blob_image(L, n_blobs, rng, n_rects=n_rects)
    rho1 = mixture_distribution(L, rng)
    rho2 = mixture_distribution(L, rng)
    s1 = rng.choice(L, size=N, p=rho1)
    s2 = rng.choice(L, size=N, p=rho2)
    l = L // K
    noise = rng.standard_normal((N, l, l)) * sigma
    y64 = observe(x, K, s1, s2, noise)
    y = np.ascontiguousarray(y64.astype(np.float32))
    if init == "mean_upsample":
        m = y.astype(np.float64).mean(axis=0)                  # (l, l)
        x0 = np.repeat(np.repeat(m, K, axis=0), K, axis=1)     # nearest neighbour
    elif init == "uniform":
        x0 = rng.uniform(0.0, 1.0, size=(L, L))
        x0 = (x0 - x0.min()) / (x0.max() - x0.min())
    else:
        raise ValueError(init)
    uni = np.full(L, 1.0 / L)
    return Problem(L=L, K=K, N=N, sigma=float(sigma),
                   x_true=x.astype(np.float32), rho1_true=rho1, rho2_true=rho2,
                   s1=s1.astype(np.int64), s2=s2.astype(np.int64), y=y,
                   x0=np.ascontiguousarray(x0.astype(np.float32)),
                   rho1_0=uni.copy(), rho2_0=uni.copy())


# The five workloads of the benchmark plan, as (name -> generator arguments).
# Images: blob images; config 2 adds a rectangle layer.
WORKLOADS = {
    "plain_em_L16_K2_N500": dict(L=16, K=2, N=500, sigma=0.1, n_blobs=6,
                                 iters=20, F=0, config=1),
    "proj_em_L64_K2_N1e4": dict(L=64, K=2, N=10_000, sigma=0.3, n_blobs=40,
                                n_rects=8, iters=30, F=1, config=2),
    "precision_L96_K3_N5e4_s0.2": dict(L=96, K=3, N=50_000, sigma=0.2,
                                       n_blobs=6, iters=40, F=1, config=3),
    "precision_L96_K3_N5e4_s1.0": dict(L=96, K=3, N=50_000, sigma=1.0,
                                       n_blobs=6, iters=40, F=1, config=3),
}


# the largest request of the serving mix, as a single problem
WORKLOADS["largest_request_L128_K2_N1e5"] = dict(L=128, K=2, N=100_000, sigma=0.5,
                                                 n_blobs=6, iters=30, F=1, config=5)
WORKLOADS["batched_64"] = dict(count=64, iters=30, F=1, config=4, prec="bf16x3")
WORKLOADS["serve"] = dict(rate=50.0, iters=30, F=1, config=5, prec="bf16x3")


def workload_problem(name: str, N: int | None = None, instance: int = 0) -> Problem:
    """Build the seeded problem of a named workload (optionally with fewer observations)."""
    w = WORKLOADS[name]
    n = w["N"] if N is None else N
    return make_problem(w["L"], w["K"], n, w["sigma"], seed_for(w["config"], instance),
                        n_blobs=w.get("n_blobs", 6), n_rects=w.get("n_rects", 0))


def batched_instances(count: int = 64, seed: int = seed_for(4)):
    """Uneven instances for the batched workload: L in {32,48,64,96}, K in {2,4},
    N ~ U[1000, 20000], sigma ~ U[0.1, 1.0]; each with its own blob image and rho."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for k in range(count):
        L = int(rng.choice([32, 48, 64, 96]))
        K = int(rng.choice([2, 4]))
        N = int(rng.integers(1000, 20001))
        sigma = float(rng.uniform(0.1, 1.0))
        specs.append(dict(L=L, K=K, N=N, sigma=sigma, seed=seed_for(4, k)))
    return specs


def snr(x: np.ndarray, sigma: float) -> float:
    """SNR = ||x||_F^2 / (L^2 sigma^2) as defined in Sec. 5."""
    return float(np.sum(np.asarray(x, np.float64) ** 2) / (x.size * sigma ** 2))


__all__ = ["Problem", "make_problem", "workload_problem", "WORKLOADS", "seed_for",
           "batched_instances", "snr", "observe", "blob_image",
           "mixture_distribution", "uniform_simplex_draw"]
