"""GPU parity of the polyphase-FFT form (SRMRA_FFT32) against the FP64 oracles: per
iteration x, rho, LL, lse[i] and c[s] element by element within the float32 tolerance
(1e-5 relative) on the dense float32 form's parity problems and a projected run; its
error next to the dense float32 form's on harder starts; the same problem through a
batch; and the sizes it refuses."""
import numpy as np
import pytest

from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth
from tests import test_gpu_parity as P

pytestmark = pytest.mark.gpu

P.TOL.setdefault("fft32", 1e-5)
S = P.S  # module fixture

CASES = [
    (16, 2, 500, 0.1),    # l = 8 (the plain-EM workload)
    (32, 2, 700, 0.4),    # l = 16
    (64, 2, 700, 0.3),    # l = 32
    (24, 3, 333, 0.5),    # l = 8, K = 3, N % 8 != 0
    (32, 4, 129, 0.6),    # l = 8, K = 4
    (8, 1, 130, 0.5),     # K = 1: classic 2D MRA
    # odd N: the last observation pair of the last block holds one observation
    (64, 2, 701, 0.3),    # l = 32
    (32, 2, 333, 0.4),    # l = 16
]


@pytest.mark.parametrize("L,K,N,sigma", CASES)
def test_em_step_parity_fft32(S, L, K, N, sigma):
    """The dense float32 form's parity problems (same seeds and start)."""
    p = synth.make_problem(L, K, N, sigma, seed=synth.seed_for(1, L * 7 + K))
    P.check_one_step(S, p, steps=3, prec="fft32", oracle="fft")


@pytest.mark.parametrize("L,K,N,sigma", [(16, 2, 500, 0.1), (64, 2, 700, 0.3)])
def test_fft32_error_matches_fp32_form(S, L, K, N, sigma):
    """From a uniform random start at high SNR the first step is poorly conditioned and
    neither float32 form reaches 1e-5 (both ~1e-5 to 5e-5 on x).  The FFT form's error
    against the float64 oracle is then no larger than the dense float32 form's."""
    from oracle import fft_oracle as FO
    p = synth.make_problem(L, K, N, sigma, seed=synth.seed_for(9, L + K), init="uniform")
    err = {}
    for prec in ("fp32", "fft32"):
        s = P.make_solver(S, p, prec)
        x0, r1, r2, _, _ = s.state()
        s.em_iter(1)
        x, a1, a2, _, _ = s.state()
        s.close()
        xo, r1o, r2o, _, _ = FO.em_iter_fft(p.y, x0, r1, r2, p.sigma, p.K)
        err[prec] = (P.rel(x, xo), max(P.rel(a1, r1o), P.rel(a2, r2o)))
    print(L, K, N, sigma, err)
    assert err["fft32"][0] <= 1.5 * err["fp32"][0] + 1e-6
    assert err["fft32"][1] <= 1.5 * err["fp32"][1] + 1e-6


def test_precision_workload_shapes_fft32(S):
    """L=96, K=3 (l = 32), sigma = 0.2 on 1000 observations with the workload's own
    start.  (From a uniform random start at this sigma, 7 of the 9 sub-images receive
    posterior mass below 1e-20: float32 weights underflow there, both float32 forms
    leave those pixels as uncovered, and the float64 oracle divides by A_r ~ 1e-120 —
    a degenerate case, not a parity case.)"""
    p = synth.workload_problem("precision_L96_K3_N5e4_s0.2", N=1000)
    P.check_one_step(S, p, steps=2, prec="fft32", oracle="fft")


def test_projected_steps_fft32(S):
    p = synth.make_problem(64, 2, 900, 0.3, seed=synth.seed_for(9, 99), n_blobs=12, n_rects=4,
                           init="uniform")
    P.check_one_step(S, p, steps=3, prec="fft32", oracle="fft", F=1)


def test_full_size_sampled_fft32(S):
    """The bench workload (L64 K2 N1e4): lse of a sample of observations against the
    oracle's direct formula, and rho on the simplex."""
    p = synth.workload_problem("proj_em_L64_K2_N1e4")
    s = S.Solver(p.L, p.K, p.sigma, p.y, prec="fft32", x0=p.x0, rho1=p.rho1_0, rho2=p.rho2_0)
    s.em_iter(1)
    lse, _ = s.estep()
    _, r1, r2, _, _ = s.state()
    s.close()
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(p.N, size=64, replace=False))
    _, lse_o, _ = O.estep(p.y[idx], p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K)
    yscale = (p.y[idx].astype(np.float64) ** 2).sum(axis=(1, 2)) / (2 * p.sigma ** 2)
    err = np.max(np.abs(lse[idx] - lse_o) / (1 + np.abs(lse_o) + yscale))
    assert err < 1e-5
    assert abs(r1.sum() - 1) < 1e-12 and abs(r2.sum() - 1) < 1e-12


def test_fft32_agrees_with_fp32_form(S):
    """Five EM iterations (no projection) from the same start: the two float32 forms
    compute the same function with different rounding."""
    p = synth.make_problem(64, 2, 1500, 0.5, seed=synth.seed_for(9, 7), init="uniform")
    out = []
    for prec in ("fp32", "fft32"):
        s = P.make_solver(S, p, prec)
        ll = s.em_iter(5)
        out.append((s.state(), ll))
        s.close()
    (xa, r1a, r2a, _, _), lla = out[0]
    (xb, r1b, r2b, _, _), llb = out[1]
    assert P.rel(xb, xa) < 1e-4 and P.rel(r1b, r1a) < 1e-4 and P.rel(r2b, r2a) < 1e-4
    assert np.max(np.abs(llb - lla) / np.abs(lla)) < 1e-5


def test_fft32_batch_equals_alone(S):
    probs = [synth.make_problem(L, K, N, s, seed=synth.seed_for(9, 40 + k), init="uniform")
             for k, (L, K, N, s) in enumerate([(64, 2, 600, 0.4), (32, 4, 800, 0.5),
                                                (48, 3, 500, 0.3)])]
    alone = []
    for p in probs:
        s = P.make_solver(S, p, "fft32")
        s.solve(3, 1)
        alone.append(s.state())
        s.close()
    solvers = [P.make_solver(S, p, "fft32") for p in probs]
    b = S.Batch(solvers, autotune=False)
    b.solve(3, 1)
    for k, s in enumerate(solvers):
        x, r1, r2, _, _ = s.state()
        assert x.tobytes() == alone[k][0].tobytes()
        assert r1.tobytes() == alone[k][1].tobytes() and r2.tobytes() == alone[k][2].tobytes()
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("L,K", [(12, 2), (40, 1), (128, 2)])
def test_fft32_refuses_other_sizes(S, L, K):
    p = synth.make_problem(L, K, 50, 0.5, seed=1)
    with pytest.raises(S.SrmraError) as e:
        S.Solver(p.L, p.K, p.sigma, p.y, prec="fft32")
    assert "EINVAL" in str(e.value)
