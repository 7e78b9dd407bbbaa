"""BlackScholes (arXiv 1502.02389, Sec. 7 "Mathematical Finance
Application", Fig. 6) in FP64.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Fig. 6 maps BSComputation over the stock prices s: d1 = compD1(s),
d2 = compD2(d1, s), and the pair {compCall(d1, d2, s), compPut(d1, d2, s)}.
The paper does not print the four functions ("purely sequential code
implementing the BlackScholes model"); they are written here from the
Black-Scholes model of a European option with strike K, riskless rate r,
volatility sigma and maturity T (years):

    d1   = (ln(s/K) + (r + sigma^2/2) T) / (sigma sqrt(T))
    d2   = d1 - sigma sqrt(T)
    call = s N(d1) - K e^{-rT} N(d2)
    put  = K e^{-rT} N(-d2) - s N(-d1)

N is the standard normal distribution function, N(x) = erfc(-x/sqrt(2))/2
(scipy's FP64 erfc).  The put is computed from its own formula, not from
put-call parity, so that parity is a check of the pair.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def normal_cdf(x):
    return 0.5 * erfc(-np.asarray(x, np.float64) / math.sqrt(2.0))


def comp_d1(s, K, r, sigma, T):
    return (np.log(np.asarray(s, np.float64) / K) + (r + 0.5 * sigma * sigma) * T) / \
        (sigma * math.sqrt(T))


def comp_d2(d1, s, K, r, sigma, T):
    return d1 - sigma * math.sqrt(T)


def comp_call(d1, d2, s, K, r, sigma, T):
    return np.asarray(s, np.float64) * normal_cdf(d1) - K * math.exp(-r * T) * normal_cdf(d2)


def comp_put(d1, d2, s, K, r, sigma, T):
    return K * math.exp(-r * T) * normal_cdf(-d2) - np.asarray(s, np.float64) * normal_cdf(-d1)


def bs_computation(s, K, r, sigma, T):
    """One {call, put} pair per price (vectorised over s: the map)."""
    with np.errstate(divide="ignore"):
        d1 = comp_d1(s, K, r, sigma, T)
    d2 = comp_d2(d1, s, K, r, sigma, T)
    return comp_call(d1, d2, s, K, r, sigma, T), comp_put(d1, d2, s, K, r, sigma, T)


def black_scholes(s, K, r, sigma, T):
    """blackScholes(s) = map(BSComputation, s): (call[], put[])."""
    return bs_computation(np.asarray(s, np.float64), K, r, sigma, T)


U_FP32 = 2.0 ** -24


def tolerance(s, K, r, T):
    """Per-option bound for an fp32 evaluation: 16 u (s + K e^{-rT}).  Both
    terms of the call are at most s and K e^{-rT} in size and each is formed
    with a few units of relative error (logf 1 ulp, erfcf 4 ulp, the
    roundings of the arguments and products); an error in d1 moves the call
    by s phi(d1) - K e^{-rT} phi(d2) = 0 to first order, because d2 is
    formed from the same d1; the rounding of d2 adds at most
    K e^{-rT} max|x phi(x)| u < 0.25 K e^{-rT} u; put-call parity adds two
    roundings of size s + K e^{-rT}."""
    return 16.0 * U_FP32 * (np.asarray(s, np.float64) + K * math.exp(-r * T))
