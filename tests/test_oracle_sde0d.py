"""Pins of the oracle's 0-d SDE ensembles (Sec. III) against what the paper and
the mathematics fix: the exact GBM solution on the same Wiener path (strong
orders 1/2 for EM and SETD-EM, 1 for Milstein and SETD-Milstein), the one-step
mean-square factors E[S(h)^2] of the stability table, the exact Ornstein-
Uhlenbeck moments (SETD1 exact at any h; SETD-EM and EM with their closed-form
stationary variances) and the Boltzmann moments of the SAO."""
import numpy as np
import pytest
from scipy import integrate


def gbm_exact(u0, lam, mu, t, W):
    return u0 * np.exp((lam - 0.5 * mu * mu) * t + mu * W)


def fit_order(hs, errs):
    return float(np.polyfit(np.log(hs), np.log(errs), 1)[0])


@pytest.mark.parametrize("scheme,order", [(0, 0.5), (1, 1.0), (2, 0.5), (3, 1.0)],
                         ids=["EM", "Milstein", "SETD-EM", "SETD-Milstein"])
def test_gbm_strong_order(oracle_mod, scheme, order):
    lam, mu, delta = 2.0, 1.0, 1.0  # delta = 1: the SETD schemes carry a deterministic term too
    S, kmax = 4000, 7
    hs, errs = [], []
    for k in range(3, kmax + 1):
        h = 2.0 ** -k
        sub = 2 ** (kmax - k)  # every run sums the same 2^-7 increments
        u, W = oracle_mod.sde0d(oracle_mod.SDE_GBM, [lam, mu, delta], scheme, h, 2 ** k, np.ones(S), seed=11,
                                substeps=sub)
        errs.append(np.mean(np.abs(u - gbm_exact(1.0, lam, mu, 1.0, W))))
        hs.append(h)
    assert abs(fit_order(hs, errs) - order) < 0.15, (scheme, fit_order(hs, errs), errs)


def test_stability_table_second_moments(oracle_mod):
    """One step from U0 = 1: E[U1^2] = E[S(h)^2], the left sides of the stability
    conditions of the table in Sec. III."""
    lam, mu, delta, h = -1.5, 1.2, 0.5, 0.3
    c = lam - delta
    f1, f2 = np.exp(c * h), np.expm1(c * h) / c
    f3, f4 = np.exp(0.5 * c * h), np.sqrt(np.expm1(2 * c * h) / (2 * c))
    want = {0: (1 + lam * h) ** 2 + h * mu ** 2,
            1: (1 + lam * h) ** 2 + h * mu ** 2 + 0.5 * h * h * mu ** 4,
            2: (f1 + f2 * delta) ** 2 + h * (f3 * mu) ** 2,
            3: (f1 + f2 * delta) ** 2 + h * (f3 * mu) ** 2 + 0.5 * h * h * (f3 * mu * mu) ** 2,
            4: (f1 + f2 * delta) ** 2 + (f4 * mu) ** 2}
    S = 200000
    for scheme, m2 in want.items():
        # EM and Milstein have no exponential part: their drift is lambda u, i.e. c + delta
        u, _ = oracle_mod.sde0d(oracle_mod.SDE_GBM, [lam, mu, delta], scheme, h, 1, np.ones(S), seed=5)
        x = u * u
        assert abs(x.mean() - m2) < 4 * x.std() / np.sqrt(S), (scheme, x.mean(), m2)


def test_ou_moments(oracle_mod):
    """b = 0: Ornstein-Uhlenbeck.  SETD1 is exact in distribution at any h; the
    stationary variances of SETD-EM and EM are T Gamma h / sinh(Gamma h) and
    T / (1 - Gamma h / 2)."""
    G, T, h, n = 5.0, 6.0, 0.2, 40
    S = 40000
    t = n * h
    u0 = np.full(S, 2.0)
    u, _ = oracle_mod.sde0d(oracle_mod.SDE_SAO, [G, T, 0.0], 4, h, n, u0, seed=21)
    m, v = 2.0 * np.exp(-G * t), T * (1 - np.exp(-2 * G * t))
    assert abs(u.mean() - m) < 4 * np.sqrt(v / S)
    assert abs(u.var() - v) < 4 * v * np.sqrt(2.0 / S)
    for scheme, vs in ((2, T * G * h / np.sinh(G * h)), (0, T / (1 - G * h / 2))):
        u, _ = oracle_mod.sde0d(oracle_mod.SDE_SAO, [G, T, 0.0], scheme, h, 200, np.zeros(S), seed=22)
        assert abs(u.var() - vs) < 4 * vs * np.sqrt(2.0 / S), (scheme, u.var(), vs)


def test_sao_boltzmann_moments(oracle_mod):
    """Steady state of the SAO with SETD1 at h = 0.01 (the parameters of the SAO
    figure of Sec. III: Gamma = 5, T = 6, b = 0.01): <u^2> and <u^4> of
    P(u) ~ exp(-V(u)/T), V = u^2/2 + b u^4/4, within 4 sigma plus O(h)."""
    G, T, b, h = 5.0, 6.0, 0.01, 0.01
    S = 20000
    u, _ = oracle_mod.sde0d(oracle_mod.SDE_SAO, [G, T, b], 4, h, 400, np.zeros(S), seed=31)
    w = lambda x: np.exp(-(0.5 * x * x + 0.25 * b * x ** 4) / T)
    Z = integrate.quad(w, -np.inf, np.inf)[0]
    for k in (2, 4):
        mk = integrate.quad(lambda x: x ** k * w(x), -np.inf, np.inf)[0] / Z
        x = u ** k
        assert abs(x.mean() - mk) < 4 * x.std() / np.sqrt(S) + 0.02 * mk, (k, x.mean(), mk)
