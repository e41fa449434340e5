"""CPU-side checks of the C ABI: the library loads, exports every entry point that
include/srmra.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "srmra.h")


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:srmra_status|void|const char\*|int64_t)\s+(srmra_\w+)\s*\(",
                                 txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_04754_gb300 import srmra
    if not os.path.exists(srmra.LIB_PATH):
        from paper_2204_04754_gb300 import build
        build.build()
    return srmra.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["srmra_create", "srmra_em_iter", "srmra_project", "srmra_solve",
              "srmra_get_state", "srmra_set_state", "srmra_destroy", "srmra_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    from paper_2204_04754_gb300 import srmra as S
    y = np.zeros((4, 2, 2), np.float32)
    bad = [S.srmra_params(6, 4, 4, 0.5, 0, 0),     # K does not divide L
           S.srmra_params(4, 2, 0, 0.5, 0, 0),     # N < 1
           S.srmra_params(4, 2, 4, 0.0, 0, 0),     # sigma <= 0
           S.srmra_params(4, 2, 4, -1.0, 0, 0),
           S.srmra_params(1, 1, 4, 0.5, 0, 0),     # L < 2
           S.srmra_params(4, 2, 4, 0.5, 7, 0)]     # unknown precision
    for p in bad:
        with pytest.raises(S.SrmraError) as e:
            S.srmra_create(p, y, False)
        assert e.value.status == S.SRMRA_EINVAL
    p = S.srmra_params(4, 2, 4, 0.5, 0, 0)
    with pytest.raises(S.SrmraError) as e:
        S.srmra_create(p, y, False, rho1_0=np.array([0.5, 0.5, 0.5, 0.5]))
    assert e.value.status == S.SRMRA_EINVAL
    with pytest.raises(S.SrmraError) as e:
        S.srmra_create(p, y, False, rho1_0=np.array([1.2, -0.2, 0.0, 0.0]))
    assert e.value.status == S.SRMRA_EINVAL
    # NULL context is an error, not a crash
    assert lib.srmra_em_iter(None, 1, None) == S.SRMRA_EINVAL
    lib.srmra_destroy(None)
    out = ctypes.c_void_p()
    assert lib.srmra_mom_create(None, ctypes.byref(out)) == S.SRMRA_EINVAL and not out.value
    assert lib.srmra_mom_run(None, 1, 0, 0.1, 0.1, 1.0, 0.9, None, None, None) == S.SRMRA_EINVAL
    assert lib.srmra_mom_eval(None, None, None, None, None) == S.SRMRA_EINVAL
    lib.srmra_mom_destroy(None)
    n = ctypes.c_int64()
    assert lib.srmra_stats_length(None, ctypes.byref(n)) == S.SRMRA_EINVAL
    assert lib.srmra_estep_stats(None, None, 0) == S.SRMRA_EINVAL
    assert lib.srmra_mstep_stats(None, None, 0, None) == S.SRMRA_EINVAL


def test_no_cpu_fallback(lib):
    """Valid arguments on a machine without a usable GB300 fail loudly (ECUDA)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2204_04754_gb300 import srmra as S
    y = np.zeros((4, 2, 2), np.float32)
    with pytest.raises(S.SrmraError) as e:
        S.srmra_create(S.srmra_params(4, 2, 4, 0.5, 0, 0), y, False)
    assert e.value.status == S.SRMRA_ECUDA


def test_version_string(lib):
    assert lib.srmra_version().startswith(b"srmra")


def test_binding_constants_match_the_header():
    """The flag values and pass-2 form codes of include/srmra.h and of the Python
    binding agree, and the binding names every form the header defines."""
    from paper_2204_04754_gb300 import srmra
    txt = open(HEADER).read()
    flags = dict(re.findall(r"^#define (SRMRA_FLAG_\w+) (\d+)u", txt, flags=re.M))
    assert len(flags) >= 6
    for name, v in flags.items():
        assert getattr(srmra, name) == int(v), name
    forms = {int(v): n for n, v in re.findall(r"^#define SRMRA_P2_(\w+) (\d+)", txt, flags=re.M)}
    assert sorted(forms) == sorted(srmra.P2_FORMS), (forms, srmra.P2_FORMS)
    for code, name in forms.items():
        assert srmra.P2_FORMS[code] == name.lower(), (code, name)
