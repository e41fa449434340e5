"""The allocation-free entry point srmra_loglik_noalloc, called through the C ABI,
against the context-based entry point (srmra_create / srmra_em_iter / srmra_get_estep)
on the same inputs.  This file is collected last on purpose."""
import ctypes
from ctypes import c_double, c_int32, c_int64, c_void_p

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the float32-form tolerance used by the other parity tests


def _fn():
    from paper_2204_04754_gb300 import srmra
    lib = srmra.lib()
    f = lib.srmra_loglik_noalloc
    f.restype = c_int32
    f.argtypes = [c_void_p, c_int64, c_int32, c_int32, c_double, c_void_p, c_void_p, c_void_p,
                  c_void_p, c_void_p, c_void_p]
    lib.srmra_noalloc_last_error.restype = ctypes.c_char_p
    lib.srmra_noalloc_scratch_bytes.restype = c_int64
    return lib, f


def _reference(p):
    """lse_i and LL of theta_0 from the context-based path."""
    from paper_2204_04754_gb300 import srmra
    s = srmra.Solver(p.L, p.K, p.sigma, p.y, prec="fp32", x0=p.x0, rho1=p.rho1_true,
                     rho2=p.rho2_true)
    ll = s.em_iter(1)[0]
    lse, _ = s.estep()
    s.close()
    return lse, ll


def test_noalloc_matches_context_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2204_04754_gb300 import synth
    lib, f = _fn()
    probs = [synth.make_problem(16, 2, 500, 0.1, seed=synth.seed_for(1, 501)),
             synth.make_problem(24, 3, 777, 0.4, seed=synth.seed_for(1, 502))]
    stream = torch.cuda.current_stream().cuda_stream
    for p in probs:  # two calls in a row, different sizes, sharing the scratch array
        lse_ref, ll_ref = _reference(p)
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
        lse_g = lse.cpu().numpy()
        ll_g = float(ll.cpu().item())
        yscale = (p.y.astype(np.float64) ** 2).sum(axis=(1, 2)) / (2 * p.sigma ** 2)
        err_lse = np.max(np.abs(lse_g - lse_ref) / (1.0 + np.abs(lse_ref) + yscale))
        err_ll = abs(ll_g - ll_ref) / (abs(ll_ref) + yscale.sum())
        assert np.all(np.isfinite(lse_g))
        assert err_lse < TOL and err_ll < TOL, (err_lse, err_ll)


def test_noalloc_rejects_problems_beyond_the_scratch_size():
    torch = pytest.importorskip("torch")
    lib, f = _fn()
    assert lib.srmra_noalloc_scratch_bytes() == 64 << 20
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = f(t.data_ptr(), 1_000_000, 64, 2, 0.3, t.data_ptr(), t.data_ptr(), t.data_ptr(),
           t.data_ptr(), t.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 1  # SRMRA_EINVAL
    assert b"scratch" in lib.srmra_noalloc_last_error()
