"""The oracle's pins catch plausible mistakes: each test plants one mistake in the
oracle (on the CPU, through monkeypatching) and checks that a pin from test_oracle.py
then fails."""
import math

import numpy as np
import pytest

import tests.test_oracle as T
from oracle import fft_oracle as FO
from oracle import srmra_oracle as O


def fails(check) -> bool:
    try:
        check()
    except AssertionError:
        return True
    return False


def pin_templates():
    T.test_templates_and_adjoint_match_explicit_matrices(6, 2)


def pin_estep():
    T.test_estep_matches_brute_force(6, 2, 4, 0.9)


def pin_mstep():
    T.test_mstep_matches_dense_linear_solve(6, 2)


def pin_fft():
    T.test_fft_oracle_matches_dense(12, 3, 200, 0.5)


def pin_dct():
    T.test_dct_matrix_is_orthonormal_and_matches_scipy()
    T.test_dct_denoise_rules()


def pin_worked():
    T.test_worked_example_closed_form()


def test_wrong_shift_sign_is_caught(monkeypatch):
    monkeypatch.setattr(O, "shift", lambda x, s1, s2: np.roll(x, shift=(-s1, -s2), axis=(0, 1)))
    assert fails(pin_templates)


def test_dropped_prior_term_is_caught(monkeypatch):
    orig = O.log_prior
    monkeypatch.setattr(O, "log_prior", lambda r1, r2: orig(r1, np.full(len(r2), 1.0 / len(r2))))
    assert fails(pin_estep) and fails(pin_worked)


def test_sigma_instead_of_sigma_squared_is_caught(monkeypatch):
    orig = O.estep

    def bad(Y, x, rho1, rho2, sigma, K, literal=False):
        return orig(Y, x, rho1, rho2, math.sqrt(sigma), K, literal)

    monkeypatch.setattr(O, "estep", bad)
    assert fails(pin_estep) and fails(pin_worked)


def test_wrong_adjoint_is_caught(monkeypatch):
    monkeypatch.setattr(O, "template_adjoint",
                        lambda v, K, s1, s2: O.shift(O.sample_adjoint(v, K), s1, s2))
    assert fails(pin_templates) and fails(pin_mstep)


def test_transposed_dct_is_caught(monkeypatch):
    orig = O.dct_matrix
    monkeypatch.setattr(O, "dct_matrix", lambda B=8: orig(B).T)
    assert fails(pin_dct)


def test_fft_conjugate_on_wrong_operand_is_caught(monkeypatch):
    orig_fft2, orig_ifft2 = np.fft.fft2, np.fft.ifft2

    class FakeFFT:
        @staticmethod
        def fft2(a, *args, **kw):
            return orig_fft2(a, *args, **kw)

        @staticmethod
        def ifft2(a, *args, **kw):
            return orig_ifft2(np.conj(a), *args, **kw)

    monkeypatch.setattr(FO.np, "fft", FakeFFT)
    assert fails(pin_fft)


def test_rho_without_normalisation_is_caught(monkeypatch):
    orig = O.mstep_from_sums

    def bad(Z, c, x_prev, K):
        x, r1, r2, b, A = orig(Z, c, x_prev, K)
        return x, r1 * 1.01, r2, b, A

    monkeypatch.setattr(O, "mstep_from_sums", bad)
    assert fails(pin_mstep) and fails(pin_worked)


def test_x_update_without_coverage_division_is_caught(monkeypatch):
    orig = O.mstep_from_sums

    def bad(Z, c, x_prev, K):
        x, r1, r2, b, A = orig(Z, c, x_prev, K)
        return b / A.max(), r1, r2, b, A

    monkeypatch.setattr(O, "mstep_from_sums", bad)
    assert fails(pin_mstep) and fails(pin_worked)


def test_unweighted_online_update_is_caught(monkeypatch):
    monkeypatch.setattr(O, "sa_update",
                        lambda S, Sb, g: Sb if S is None else tuple(a + g * b for a, b in zip(S, Sb)))
    assert fails(T.test_online_statistics_average_to_the_full_data_ones)


def test_loglik_chunk_overlap_is_caught(monkeypatch):
    """A chunked log-likelihood whose chunks overlap by one observation."""
    orig = O.loglik

    def overlapping(Y, x, rho1, rho2, sigma, K, chunk=None):
        if chunk is None or chunk >= len(Y):
            return orig(Y, x, rho1, rho2, sigma, K, chunk=chunk)
        total = 0.0
        for a in range(0, len(Y), chunk):
            total += orig(Y[max(0, a - 1):a + chunk], x, rho1, rho2, sigma, K)
        return total
    monkeypatch.setattr(O, "loglik", overlapping)
    assert fails(lambda: T.test_chunked_loglik_matches_brute_force(3))
