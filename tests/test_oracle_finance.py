"""Pins of the BlackScholes oracle (Fig. 6): the risk-neutral expectation
the closed form must equal (numerical quadrature), put-call parity, limits,
the at-the-money-forward closed form, and monotonicity."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import finance

CASES = [(42.0, 40.0, 0.10, 0.20, 0.5), (20.0, 20.0, 0.02, 0.30, 1.0), (5.0, 20.0, 0.02, 0.30, 1.0),
         (30.0, 20.0, 0.05, 0.60, 2.5), (100.0, 80.0, 0.0, 0.15, 0.25)]


def expectation(S, K, r, sigma, T, put=False):
    """e^{-rT} E[payoff(S_T)], S_T = S exp((r - sigma^2/2) T + sigma sqrt(T) Z),
    Z standard normal, by adaptive quadrature split at the exercise point."""
    st = lambda z: S * math.exp((r - 0.5 * sigma * sigma) * T + sigma * math.sqrt(T) * z)  # noqa: E731
    phi = lambda z: math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)  # noqa: E731
    pay = (lambda z: max(K - st(z), 0.0)) if put else (lambda z: max(st(z) - K, 0.0))
    zk = (math.log(K / S) - (r - 0.5 * sigma * sigma) * T) / (sigma * math.sqrt(T))
    f = lambda z: pay(z) * phi(z)  # noqa: E731
    a, _ = integrate.quad(f, -40.0, zk, epsabs=1e-13, epsrel=1e-12, limit=200)
    b, _ = integrate.quad(f, zk, 40.0, epsabs=1e-13, epsrel=1e-12, limit=200)
    return math.exp(-r * T) * (a + b)


@pytest.mark.parametrize("S,K,r,sigma,T", CASES)
def test_closed_form_equals_the_risk_neutral_expectation(S, K, r, sigma, T):
    c, p = finance.black_scholes(np.array([S]), K, r, sigma, T)
    assert abs(c[0] - expectation(S, K, r, sigma, T)) <= 1e-9 * (S + K)
    assert abs(p[0] - expectation(S, K, r, sigma, T, put=True)) <= 1e-9 * (S + K)


def test_put_call_parity_and_bounds():
    rng = np.random.default_rng(0)
    S = rng.uniform(1, 200, 10000)
    K, r, sigma, T = 50.0, 0.03, 0.4, 1.7
    c, p = finance.black_scholes(S, K, r, sigma, T)
    ke = K * math.exp(-r * T)
    assert np.all(np.abs((c - p) - (S - ke)) <= 1e-12 * (S + ke))
    assert np.all(c >= np.maximum(S - ke, 0) - 1e-12 * S) and np.all(c <= S)
    assert np.all(p >= np.maximum(ke - S, 0) - 1e-12 * ke) and np.all(p <= ke)
    order = np.argsort(S)
    assert np.all(np.diff(c[order]) >= 0) and np.all(np.diff(p[order]) <= 0)


def test_limits():
    K, r, T = 20.0, 0.02, 1.0
    ke = K * math.exp(-r * T)
    S = np.array([10.0, 19.0, 25.0, 40.0])
    c, p = finance.black_scholes(S, K, r, 1e-9, T)          # no volatility: forward payoff
    assert np.allclose(c, np.maximum(S - ke, 0), rtol=0, atol=1e-12)
    assert np.allclose(p, np.maximum(ke - S, 0), rtol=0, atol=1e-12)
    c, p = finance.black_scholes(np.array([0.0]), K, r, 0.3, T)   # worthless stock
    assert c[0] == 0.0 and p[0] == ke


def test_at_the_money_forward():
    # S = K e^{-rT}: d1 = sigma sqrt(T)/2 = -d2, so call = put = S (2 N(sigma sqrt(T)/2) - 1)
    K, r, sigma, T = 20.0, 0.02, 0.3, 1.0
    S = K * math.exp(-r * T)
    c, p = finance.black_scholes(np.array([S]), K, r, sigma, T)
    h = 0.5 * sigma * math.sqrt(T)
    exact = S * math.erf(h / math.sqrt(2.0))      # 2 N(h) - 1 = erf(h / sqrt 2)
    assert abs(c[0] - exact) <= 1e-14 * S and abs(p[0] - exact) <= 1e-14 * S


def test_tolerance_formula():
    t = finance.tolerance(np.array([10.0]), 20.0, 0.0, 1.0)
    assert t[0] == 16 * 2.0 ** -24 * 30.0
