"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs.  Tolerances are those the method targets: relative L2 error of x and
rho within 1e-5 for the float32 form (per iteration, and after full runs); the
log-likelihood and per-observation lse within the float32 rounding of a logit."""
import math
import os

import numpy as np
import pytest

from oracle import fft_oracle as FO
from oracle import srmra_oracle as O
from paper_2204_04754_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def S():
    from paper_2204_04754_gb300 import srmra
    if not os.path.exists(srmra.LIB_PATH):
        from paper_2204_04754_gb300 import build
        build.build()
    srmra.lib()
    return srmra


def make_solver(S, p, prec="fp32", **kw):
    return S.Solver(p.L, p.K, p.sigma, p.y, prec=prec, x0=p.x0, rho1=p.rho1_0,
                    rho2=p.rho2_0, **kw)


def check_one_step(S, p, steps, prec="fp32", chunk=None, oracle="dense", F=0):
    """Restart the oracle from the GPU state before every iteration and compare
    x, rho, LL, lse[i] and c[s] element by element."""
    tol = TOL[prec]
    yscale = (p.y.astype(np.float64) ** 2).sum(axis=(1, 2)) / (2 * p.sigma ** 2)
    s = make_solver(S, p, prec)
    sbm = 1.0
    worst = dict(x=0.0, rho=0.0, ll=0.0, lse=0.0, c=0.0)
    for it in range(steps):
        x, r1, r2, _, _ = s.state()
        ll = s.em_iter(1)[0]
        fn = O.em_iter if oracle == "dense" else FO.em_iter_fft
        xo, r1o, r2o, llo, aux = fn(p.y, x, r1, r2, p.sigma, p.K, chunk=chunk)
        xg, r1g, r2g, _, _ = s.state()
        lse, c = s.estep()
        if F:
            s.project(sbm)
            xo_d, margin = O.dct_denoise(xg, sbm)
            xg_d = s.state()[0]
            worst["x_denoised"] = max(worst.get("x_denoised", 0.0), rel(xg_d, xo_d))
            assert margin > 1e-6 * sbm, "threshold tie: pick another seed"
            sbm *= 2.0 ** -0.1
        worst["x"] = max(worst["x"], rel(xg, xo))
        worst["rho"] = max(worst["rho"], rel(r1g, r1o), rel(r2g, r2o))
        # LL and lse are differences of terms of size ||y_i||^2 / (2 sigma^2); their
        # float32 rounding is relative to that scale, not to the (possibly ~0) result
        worst["ll"] = max(worst["ll"], abs(ll - llo) / (abs(llo) + yscale.sum()))
        worst["lse"] = max(worst["lse"], float(np.max(np.abs(lse - aux["lse"]) /
                                                      (1.0 + np.abs(aux["lse"]) + yscale))))
        worst["c"] = max(worst["c"], float(np.max(np.abs(c - aux["c"]))) / p.N)
        assert abs(r1g.sum() - 1) < 1e-12 and abs(r2g.sum() - 1) < 1e-12
    s.close()
    print(p.L, p.K, p.N, p.sigma, worst)
    assert worst["x"] < tol and worst["rho"] < tol
    assert worst["ll"] < tol and worst["lse"] < tol and worst["c"] < tol
    if F:
        assert worst["x_denoised"] < tol
    return worst


# (L, K, N, sigma): several tiles, ragged tails, K = 1, K = L, odd low-res sizes
CASES = [
    (16, 2, 500, 0.1),     # the plain-EM workload (l = 8)
    (12, 3, 333, 0.4),     # ragged shift tile (S = 144), l^2 = 16, N % 128 != 0
    (12, 2, 257, 0.3),     # l^2 = 36 (not a multiple of 16)
    (8, 1, 130, 0.5),      # K = 1: classic 2D MRA
    (20, 4, 129, 0.6),     # l = 5
    (6, 6, 40, 0.3),       # K = L: l = 1
    (64, 2, 700, 0.3),     # l = 32: four 256-pixel chunks (cluster of 4)
    (48, 1, 300, 0.8),     # l^2 = 2304: nine chunks, two chunk groups
]


@pytest.mark.parametrize("L,K,N,sigma", CASES)
def test_em_step_parity_fp32(S, L, K, N, sigma):
    p = synth.make_problem(L, K, N, sigma, seed=synth.seed_for(1, L * 7 + K))
    check_one_step(S, p, steps=3)


def test_single_observation(S):
    p = synth.make_problem(16, 2, 1, 0.2, seed=31)
    check_one_step(S, p, steps=2)


def test_worked_example_closed_form(S):
    """The L = 2, K = 2 closed-form fixture (a 4-component Gaussian mixture)."""
    import json
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "worked_example_L2_K2.json")))
    y = np.array(g["y"], np.float32).reshape(-1, 1, 1)
    s = S.Solver(2, 2, g["sigma"], y, x0=np.array(g["x"], np.float32), rho1=g["rho1"],
                 rho2=g["rho2"])
    ll = s.em_iter(1)[0]
    x, r1, r2, _, _ = s.state()
    e = g["expected"]
    assert rel(x, e["x"]) < 1e-6 and rel(r1, e["rho1"]) < 1e-6 and rel(r2, e["rho2"]) < 1e-6
    assert abs(ll - e["loglik"]) < 1e-6 * abs(e["loglik"])
    s.close()


def test_zero_rho_entries(S):
    """rho entries that are exactly 0 give weight 0 and no NaN (reading R7)."""
    p = synth.make_problem(16, 2, 200, 0.3, seed=41)
    r1 = np.array(p.rho1_true)
    r1[:5] = 0.0
    r1 /= r1.sum()
    s = S.Solver(p.L, p.K, p.sigma, p.y, x0=p.x0, rho1=r1, rho2=p.rho2_0)
    ll = s.em_iter(1)[0]
    xo, r1o, r2o, llo, _ = O.em_iter(p.y, p.x0, r1, p.rho2_0, p.sigma, p.K)
    x, g1, g2, _, _ = s.state()
    assert np.all(g1[:5] == 0.0)
    assert rel(x, xo) < 1e-5 and rel(g1, r1o) < 1e-5 and abs(ll - llo) < 1e-5 * abs(llo)
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fft32"])
def test_pixels_without_coverage_keep_their_value(S, prec):
    """With zero prior weight on every even first-axis shift, the sub-images of phase
    r1 = 0 get no coverage (A = 0): their pixels keep the previous value exactly
    (reading R6) and the others follow the oracle."""
    p = synth.make_problem(32, 2, 300, 0.4, seed=43)
    r1 = np.array(p.rho1_true)
    r1[0::2] = 0.0
    r1 /= r1.sum()
    s = S.Solver(p.L, p.K, p.sigma, p.y, prec=prec, x0=p.x0, rho1=r1, rho2=p.rho2_0)
    s.em_iter(1)
    x, g1, _, _, _ = s.state()
    s.close()
    xo, r1o, _, _, aux = O.em_iter(p.y, p.x0, r1, p.rho2_0, p.sigma, p.K)
    assert np.all(aux["A"][0::2] == 0.0) and np.all(aux["A"][1::2] > 0.0)
    assert np.array_equal(x[0::2], p.x0[0::2])  # first-axis pixels q1 = 0 mod 2
    tol = {"fp32": 1e-5, "fft32": 1e-5, "bf16x3": 1e-4}[prec]
    assert rel(x[1::2], xo[1::2]) < tol and rel(g1, r1o) < tol


def test_full_plain_em_run_fp32(S):
    """20 plain EM iterations at L=16, K=2, N=500, sigma=0.1 from the same start:
    x, rho after the run and the LL trajectory match the oracle; LL never decreases.

    The run starts from the paper's initial guess (U[0,1] pixels, min-max scaled;
    Sec. 5).  The mean-upsampled guess makes all K^2 sub-images equal; with uniform
    rho exact EM never leaves that set (the symmetry of Theorem 1), but the set is
    unstable, so how a run leaves it is decided by rounding alone."""
    w = synth.WORKLOADS["plain_em_L16_K2_N500"]
    p = synth.make_problem(w["L"], w["K"], w["N"], w["sigma"], synth.seed_for(1),
                           n_blobs=w["n_blobs"], init="uniform")
    s = make_solver(S, p)
    ll = s.em_iter(w["iters"])
    x, r1, r2, _, t = s.state()
    xo, r1o, r2o, h = O.projected_em(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K,
                                     iters=w["iters"], F=0)
    assert t == w["iters"]
    assert rel(x, xo) < TOL["fp32"] and rel(r1, r1o) < TOL["fp32"] and rel(r2, r2o) < TOL["fp32"]
    np.testing.assert_allclose(ll, h["LL"], rtol=1e-6)
    assert np.all(np.diff(ll) >= -1e-6 * np.abs(ll[1:]))
    s.close()


def test_projected_em_one_step_parity_fp32(S):
    """EM step + built-in DCT projection, oracle restarted from the GPU state."""
    p = synth.make_problem(64, 2, 1500, 0.3, seed=synth.seed_for(2, 5), n_blobs=40, n_rects=8)
    check_one_step(S, p, steps=3, F=1)


def test_projected_em_full_run_fp32(S):
    """Algorithm 2 with F = 1 for 8 iterations: the oracle run (same start) and the GPU
    run agree when no DCT coefficient lies near the threshold (the oracle reports
    its smallest margin)."""
    p = synth.make_problem(32, 2, 800, 0.3, seed=synth.seed_for(2, 9), n_blobs=20, n_rects=4,
                           init="uniform")
    s = make_solver(S, p)
    ll = s.solve(8, 1)
    x, r1, r2, sbm, t = s.state()
    xo, r1o, r2o, h = O.projected_em(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K, iters=8, F=1)
    assert h["margin"] > 1e-4
    assert abs(sbm - 2.0 ** (-8 / 10)) < 1e-15 and t == 8
    assert rel(x, xo) < TOL["fp32"] and rel(r1, r1o) < TOL["fp32"]
    np.testing.assert_allclose(ll, h["LL"], rtol=1e-6)
    s.close()


def test_full_size_projected_workload_one_iteration(S):
    """L=64, K=2, N=10^4, sigma=0.3 at full size: one iteration against the FFT
    oracle (element-wise on x, rho, lse, c)."""
    p = synth.workload_problem("proj_em_L64_K2_N1e4")
    check_one_step(S, p, steps=1, oracle="fft")


def test_projected_workload_full_run_30_iterations(S):
    """The projected-EM workload (L = 64, K = 2, N = 1e4, sigma = 0.3) at full size over
    its 30 iterations of Algorithm 2 (F = 1, sigma_BM_1 = 1, Eq. decaying_function) from
    the workload's initial guess: the GPU run against the FP64 oracle's own run (its
    polyphase-FFT formulation, pinned to the dense one), which reports the smallest
    distance of any DCT coefficient to the threshold (a coefficient closer than the
    two runs' difference could be kept by one and zeroed by the other)."""
    p = synth.workload_problem("proj_em_L64_K2_N1e4")
    s = make_solver(S, p)
    ll = s.solve(30, 1)
    x, r1, r2, sbm, t = s.state()
    s.close()
    step = lambda x_, a, b: FO.em_iter_fft(p.y, x_, a, b, p.sigma, p.K,
                                           workers=os.cpu_count() or 1)
    xo, r1o, r2o, h = O.projected_em(p.y, p.x0, p.rho1_0, p.rho2_0, p.sigma, p.K, iters=30,
                                     F=1, em_step=step)
    errs = (rel(x, xo), rel(r1, r1o), rel(r2, r2o),
            float(np.max(np.abs(np.asarray(ll) - h["LL"]) / np.abs(h["LL"]))))
    print("30-iteration run: margin", h["margin"], "errors x, rho1, rho2, LL", errs)
    assert t == 30 and abs(sbm - 2.0 ** -3) < 1e-15
    assert h["margin"] > 1e-4
    assert errs[0] < TOL["fp32"] and errs[1] < TOL["fp32"] and errs[2] < TOL["fp32"]
    assert errs[3] < 1e-6


def test_checkpoint_resume_is_bitwise(S):
    p = synth.make_problem(32, 2, 600, 0.3, seed=77, n_blobs=10)
    a = make_solver(S, p)
    a.solve(6, 2)
    xa, r1a, r2a, sa, ta = a.state()
    b = make_solver(S, p)
    b.solve(3, 2)
    st = b.state()
    b.close()
    c = make_solver(S, p)
    c.set_state(*st)
    c.solve(3, 2, sigma_bm1=0.0)
    xc, r1c, r2c, sc, tc = c.state()
    assert xa.tobytes() == xc.tobytes() and r1a.tobytes() == r1c.tobytes()
    assert r2a.tobytes() == r2c.tobytes() and sa == sc and ta == tc == 6
    a.close()
    c.close()


def test_determinism(S):
    p = synth.make_problem(32, 2, 700, 0.3, seed=78)
    outs = []
    for _ in range(2):
        s = make_solver(S, p)
        s.solve(3, 1)
        outs.append(s.state())
        s.close()
    assert outs[0][0].tobytes() == outs[1][0].tobytes()


def test_user_denoiser_callback(S):
    """Pluggable denoiser: a callback that leaves x alone gives plain EM; a failing
    callback surfaces as EINVAL."""
    p = synth.make_problem(16, 2, 100, 0.3, seed=79)
    calls = []

    def identity(xptr, L, sbm, stream, user):
        calls.append((L, sbm))
        return 0

    a = make_solver(S, p)
    a.solve(4, 2, denoiser=identity)
    b = make_solver(S, p)
    b.em_iter(4)
    assert a.state()[0].tobytes() == b.state()[0].tobytes()
    assert [c[0] for c in calls] == [16, 16]
    assert abs(calls[1][1] - 2 ** -0.1) < 1e-15

    def failing(xptr, L, sbm, stream, user):
        return 3

    with pytest.raises(S.SrmraError) as e:
        a.project(0.5, denoiser=failing)
    assert e.value.status == S.SRMRA_EINVAL
    a.close()
    b.close()


def test_device_resident_input_and_default_init(S):
    torch = pytest.importorskip("torch")
    p = synth.make_problem(16, 2, 300, 0.2, seed=80)
    yd = torch.from_numpy(p.y).cuda()
    s = S.Solver(p.L, p.K, p.sigma, yd, stream=torch.cuda.current_stream().cuda_stream)
    x0 = s.state()[0]
    np.testing.assert_allclose(x0, p.x0, rtol=0, atol=2e-7)
    s.em_iter(2)
    s.close()


def test_allocation_failure_is_enomem(S, monkeypatch):
    p = synth.make_problem(16, 2, 50, 0.2, seed=81)
    monkeypatch.setenv("SRMRA_ALLOC_LIMIT_BYTES", "4096")
    with pytest.raises(S.SrmraError) as e:
        make_solver(S, p)
    assert e.value.status == S.SRMRA_ENOMEM


def test_builtin_denoiser_needs_multiple_of_8(S):
    p = synth.make_problem(12, 2, 50, 0.2, seed=82)
    s = make_solver(S, p)
    with pytest.raises(S.SrmraError) as e:
        s.project(0.5)
    assert e.value.status == S.SRMRA_EINVAL
    s.close()


def test_launch_count_is_reported(S):
    p = synth.make_problem(16, 2, 50, 0.2, seed=83)
    s = make_solver(S, p)
    n0 = s.launches
    s.em_iter(2, loglik=False)
    s.sync()
    assert s.launches - n0 >= 2 * 5
    s.close()


@pytest.mark.parametrize("mode,spin", [("soft", False), ("hard", True), ("soft", True)])
def test_denoiser_variants_against_oracle(S, mode, spin):
    """Soft threshold (the l1 prox) and cycle spinning on the GPU against the oracle's
    denoiser applied to the same image."""
    p = synth.make_problem(32, 2, 500, 0.3, seed=synth.seed_for(2, 77), n_blobs=12, n_rects=3)
    s = make_solver(S, p)
    s.set_denoiser(mode, 2.7, spin)
    s.em_iter(1)
    x_pre = s.state()[0]
    s.project(0.2)
    x_gpu = s.state()[0]
    x_ref, margin = O.dct_denoise(x_pre, 0.2, mode=mode, spin=spin)
    if mode == "hard":
        assert margin > 1e-6
    assert rel(x_gpu, x_ref) < 1e-6
    # the same variant drives Algorithm 2 (single-context path and a batch)
    a = make_solver(S, p)
    a.set_denoiser(mode, 2.7, spin)
    a.solve(3, 1)
    b = make_solver(S, p)
    b.set_denoiser(mode, 2.7, spin)
    bt = S.Batch([b])
    bt.solve(3, 1)
    assert a.state()[0].tobytes() == b.state()[0].tobytes()
    bt.close()
    for z in (s, a, b):
        z.close()
