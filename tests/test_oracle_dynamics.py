"""Pins of the oracle's App. C estimators (C(k, omega), chi(k, omega), the FDT
deviation) against facts that do not come from the oracle itself.

* A hand-computed case: one mode sampled as e^{-2 pi i m / M} has all of its
  time transform (+ sign, App. C) at b = 1, |phi_b|^2 = M^2, so C = norm T at
  b = 1 and 0 elsewhere; with K = c phi, chi = norm T / M^2 / (2D) M^2
  (i omega - c) at that frequency.  Pins the normalisation, the transform sign
  and the sign of omega.
* The linear-model identity (Sec. V.A): for K = c phi with real c, every sample
  gives phi conj(-i omega phi - c phi) = (i omega - c) |phi|^2, so
  2 Im chi = (omega / D) C holds exactly for ANY series; the deviation vanishes
  to rounding.  A non-zero nonlinear term breaks it.
* Parseval in time: sum_b |phi_b|^2 = M sum_m |phi_m|^2, so sum_b C_{a,b} equals
  T times App. C's equal-time estimator norm (1/M) sum_m |phi_{a,m}|^2 (averaged
  over the ensemble).
"""
import numpy as np
import pytest


def test_hand_computed_single_frequency(oracle_mod):
    M, T, norm, c, D = 4, 2.0, 0.5, -1.0, 0.5
    m = np.arange(M)
    phi = np.exp(-2j * np.pi * m / M)[None, None, :]
    F = np.zeros_like(phi)
    C, chi, dbar = oracle_mod.dyn_estimators(phi, F, [c], [D], T, norm)
    want_C = np.zeros(M)
    want_C[1] = norm * T  # norm T / M^2 * M^2
    assert np.allclose(C[0], want_C, rtol=0, atol=1e-14)
    om1 = 2 * np.pi * 1 / T
    want_chi = np.zeros(M, complex)
    want_chi[1] = norm * T / (2 * D) * (1j * om1 - c)  # = 1 + i pi
    assert np.allclose(chi[0], want_chi, rtol=0, atol=1e-13)
    assert abs(want_chi[1] - (1 + 1j * np.pi)) < 1e-14
    assert dbar < 1e-13


def test_linear_model_identity_for_any_series(oracle_mod):
    rng = np.random.default_rng(7)
    S, n, M, T, norm = 5, 6, 16, 3.0, 0.25
    phi = rng.standard_normal((S, n, M)) + 1j * rng.standard_normal((S, n, M))
    c = -rng.uniform(0.1, 2.0, n)
    D = rng.uniform(0.2, 1.0, n)
    C, chi, dbar = oracle_mod.dyn_estimators(phi, np.zeros_like(phi), c, D, T, norm)
    b = np.fft.fftfreq(M, 1.0 / M)
    om = 2 * np.pi * b / T
    rhs = om[None, :] / D[:, None] * C
    assert np.max(np.abs(2 * chi.imag - rhs)) <= 1e-12 * np.max(np.abs(rhs))
    assert dbar <= 1e-12 * np.mean(np.abs(rhs))
    # a nonlinear term breaks the identity
    F = 0.3 * (rng.standard_normal((S, n, M)) + 1j * rng.standard_normal((S, n, M)))
    _, _, dbar_nl = oracle_mod.dyn_estimators(phi, F, c, D, T, norm)
    assert dbar_nl > 1e-3 * np.mean(np.abs(rhs))


def test_parseval_links_dynamic_and_equal_time_estimators(oracle_mod):
    rng = np.random.default_rng(11)
    S, n, M, T, norm = 3, 4, 12, 1.5, 0.125
    phi = rng.standard_normal((S, n, M)) + 1j * rng.standard_normal((S, n, M))
    F = rng.standard_normal((S, n, M)) + 1j * rng.standard_normal((S, n, M))
    C, _, _ = oracle_mod.dyn_estimators(phi, F, -np.ones(n), np.ones(n), T, norm)
    c_et = norm * np.mean(np.sum(np.abs(phi) ** 2, axis=2) / M, axis=0)  # App. C equal-time estimator
    assert np.allclose(C.sum(axis=1), T * c_et, rtol=1e-12, atol=0)


def test_modes_without_noise_are_left_out(oracle_mod):
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((2, 3, 8)) + 1j * rng.standard_normal((2, 3, 8))
    C, chi, dbar = oracle_mod.dyn_estimators(phi, 0.5 * phi, [-1.0, -1.0, -1.0], [1.0, 0.0, 1.0], 1.0, 1.0)
    assert np.all(chi[1] == 0)
    C2, chi2, dbar2 = oracle_mod.dyn_estimators(phi[:, [0, 2]], 0.5 * phi[:, [0, 2]], [-1.0, -1.0], [1.0, 1.0],
                                                1.0, 1.0)
    assert abs(dbar - dbar2) <= 1e-14 * dbar2


@pytest.mark.parametrize("bad", [dict(T=0.0), dict(T=-1.0)])
def test_rejects_bad_arguments(oracle_mod, bad):
    phi = np.ones((1, 1, 4), complex)
    with pytest.raises(ValueError):
        oracle_mod.dyn_estimators(phi, phi, [-1.0], [1.0], bad["T"], 1.0)
