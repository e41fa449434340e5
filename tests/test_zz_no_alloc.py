"""The allocation-free entry point srmra_loglik_noalloc, called through the C ABI.

It serves callers that cannot call cudaMalloc (services that size device memory once
at start-up, host code that must not block on the allocator, embedders that own all
device memory), so the first test calls it before any other library call, on two
problems in a row that share its fixed scratch array, and only then checks both
results element by element against the FP64 oracle (Eq. likelihood_EM) and against
the context-based entry point (srmra_create / srmra_em_iter / srmra_get_estep).  This
file is collected last on purpose."""
import ctypes
from ctypes import c_double, c_int32, c_int64, c_void_p

import numpy as np
import pytest

from oracle import srmra_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the float32-form tolerance used by the other parity tests


def _fn():
    from paper_2204_04754_gb300 import srmra
    if not __import__("os").path.exists(srmra.LIB_PATH):
        from paper_2204_04754_gb300 import build
        build.build()
    lib = srmra.lib()
    f = lib.srmra_loglik_noalloc
    f.restype = c_int32
    f.argtypes = [c_void_p, c_int64, c_int32, c_int32, c_double, c_void_p, c_void_p, c_void_p,
                  c_void_p, c_void_p, c_void_p]
    lib.srmra_noalloc_last_error.restype = ctypes.c_char_p
    lib.srmra_noalloc_scratch_bytes.restype = c_int64
    return lib, f


def _context_path(p):
    """lse_i and LL of theta_0 from the context-based path."""
    from paper_2204_04754_gb300 import srmra
    s = srmra.Solver(p.L, p.K, p.sigma, p.y, prec="fp32", x0=p.x0, rho1=p.rho1_true,
                     rho2=p.rho2_true)
    ll = s.em_iter(1)[0]
    lse, _ = s.estep()
    s.close()
    return lse, ll


def _errors(p, lse, ll, lse_ref, ll_ref):
    yscale = (p.y.astype(np.float64) ** 2).sum(axis=(1, 2)) / (2 * p.sigma ** 2)
    err_lse = float(np.max(np.abs(lse - lse_ref) / (1.0 + np.abs(lse_ref) + yscale)))
    err_ll = abs(ll - ll_ref) / (abs(ll_ref) + yscale.sum())
    rel_ll = abs(ll - ll_ref) / abs(ll_ref)
    return err_lse, err_ll, rel_ll


def test_noalloc_first_call_then_oracle_and_context_path():
    torch = pytest.importorskip("torch")
    from paper_2204_04754_gb300 import synth
    lib, f = _fn()
    probs = [synth.make_problem(16, 2, 500, 0.1, seed=synth.seed_for(1, 501)),
             synth.make_problem(24, 3, 777, 0.4, seed=synth.seed_for(1, 502))]
    stream = torch.cuda.current_stream().cuda_stream
    got = []
    for p in probs:  # two calls in a row, different sizes, sharing the scratch array
        y = torch.from_numpy(p.y).cuda()
        x = torch.from_numpy(p.x0).cuda()
        r1 = torch.from_numpy(p.rho1_true).cuda()
        r2 = torch.from_numpy(p.rho2_true).cuda()
        lse = torch.full((p.N,), float("nan"), dtype=torch.float64, device="cuda")
        ll = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = f(y.data_ptr(), p.N, p.L, p.K, p.sigma, x.data_ptr(), r1.data_ptr(), r2.data_ptr(),
               lse.data_ptr(), ll.data_ptr(), stream)
        assert st == 0, lib.srmra_noalloc_last_error()
        torch.cuda.synchronize()
        got.append((lse.cpu().numpy(), float(ll.cpu().item())))
    for p, (lse_g, ll_g) in zip(probs, got):
        assert np.all(np.isfinite(lse_g))
        _, lse_o, ll_o = O.estep(p.y, p.x0, p.rho1_true, p.rho2_true, p.sigma, p.K)
        e_lse, e_ll, r_ll = _errors(p, lse_g, ll_g, lse_o, ll_o)
        print("noalloc vs oracle", p.L, p.K, p.N, e_lse, e_ll, r_ll)
        assert e_lse < TOL and e_ll < TOL and r_ll < 1e-4, (e_lse, e_ll, r_ll)
        lse_c, ll_c = _context_path(p)
        e_lse, e_ll, _ = _errors(p, lse_g, ll_g, lse_c, ll_c)
        assert e_lse < TOL and e_ll < TOL, (e_lse, e_ll)


def test_noalloc_rejects_problems_beyond_the_scratch_size():
    torch = pytest.importorskip("torch")
    lib, f = _fn()
    assert lib.srmra_noalloc_scratch_bytes() == 64 << 20
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = f(t.data_ptr(), 1_000_000, 64, 2, 0.3, t.data_ptr(), t.data_ptr(), t.data_ptr(),
           t.data_ptr(), t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 1  # SRMRA_EINVAL
    assert b"scratch" in lib.srmra_noalloc_last_error()
