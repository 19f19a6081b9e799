"""Cumulative table for the discrete Gaussian error distribution.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

The error polynomials of key generation and encryption have coefficients
drawn from the discrete Gaussian D_sigma, rho(k) = exp(-k^2 / (2 sigma^2)),
cut at |k| <= floor(6 sigma) (sigma = 3.2 gives 19).  Sampling draws the
magnitude by comparing 63 random bits with the cumulative table

    cdt[k] = floor(2^63 * Pr[|X| <= k]),  k = 0 .. tail-1,

with Pr[|X| = 0] = rho(0)/Z, Pr[|X| = k] = 2 rho(k)/Z and
Z = rho(0) + 2 sum_{k=1..tail} rho(k).  sigma is the exact value of the IEEE
double passed in (3.2 is 3.2000000000000001776...).  The table is computed
here in 60-digit decimal arithmetic, exactly enough for 63-bit thresholds.
"""
import decimal
import math

import numpy as np


def tail_cut(sigma: float) -> int:
    return int(math.floor(6 * sigma))


def cdt_table(sigma: float = 3.2) -> np.ndarray:
    tail = tail_cut(sigma)
    ctx = decimal.Context(prec=60)
    s = decimal.Decimal(float(sigma))  # exact binary value of the double
    two_s2 = ctx.multiply(2, ctx.multiply(s, s))
    rho = [ctx.exp(ctx.divide(-decimal.Decimal(k * k), two_s2)) for k in range(tail + 1)]
    z = rho[0]
    for k in range(1, tail + 1):
        z = ctx.add(z, ctx.multiply(2, rho[k]))
    out = []
    cum = decimal.Decimal(0)
    scale = decimal.Decimal(2) ** 63
    for k in range(tail):
        p = rho[0] if k == 0 else ctx.multiply(2, rho[k])
        cum = ctx.add(cum, ctx.divide(p, z))
        out.append(int(ctx.multiply(cum, scale).to_integral_value(rounding=decimal.ROUND_FLOOR)))
    return np.array(out, dtype=np.uint64)
