"""CPU replay of the basis-conversion and key-product arithmetic (no GPU):
the steps of k_modup_bconv_h / k_moddown_bconv_h and k_key_product_t
restated with 64-bit wrap -- inputs straight from an inverse transform
without its N^{-1} (folded into the (D/q_i)^{-1} constants), constants and
keys in Montgomery form split into 30-bit halves, lazy 64-bit half sums,
one Montgomery reduction per output -- against the integer definitions
(fast basis conversion; sum of products modulo q)."""
import random

import pytest

from test_modular_bounds_host import M64, acc30_sum, is_prime, redc, shoup_lazy, shoup_of

N = 1 << 12


def primes(bits_list, two_n=2 * N):
    """Distinct primes 1 mod 2N, the largest below 2^bits for each size in turn."""
    out = []
    for b in bits_list:
        q = ((1 << b) - 1) // two_n * two_n + 1
        while not is_prime(q) or q in out:
            q -= two_n
        out.append(q)
    return out


def shoup(a, w, q):
    r = shoup_lazy(a, w, shoup_of(w, q), q)
    return r - q if r >= q else r


def conversion_replay(xs_unscaled, src, dst):
    """One coefficient: inputs N x_i mod q_i (an unscaled inverse transform),
    outputs y_t mod t, as the halves kernels compute them."""
    D = 1
    for q in src:
        D *= q
    v = []
    for x, qi in zip(xs_unscaled, src):
        hinv = pow((D // qi) % qi, -1, qi) * pow(N, -1, qi) % qi  # N^{-1} folded in
        v.append(shoup(x, hinv, qi))
    out = []
    for t in dst:
        hm = [((D // qi) % t) * (1 << 64) % t for qi in src]  # Montgomery form, staged as halves
        s = acc30_sum(v, hm)
        assert (s >> 64) < t
        out.append(redc(s & M64, s >> 64, t))
    return out


def fast_bconv_definition(xs, src, dst):
    D = 1
    for q in src:
        D *= q
    y = sum((x * pow((D // qi) % qi, -1, qi) % qi) * (D // qi) for x, qi in zip(xs, src))  # no reduction mod D
    return [y % t for t in dst]


@pytest.mark.parametrize("ns,bits", [(1, 60), (3, 50), (7, 50), (7, 60), (8, 59)])
def test_conversion_halves_form_equals_fast_basis_conversion(ns, bits):
    src = primes([bits] * ns)
    dst = primes([60, 50, 40, 30] + [bits] * 3)
    dst = [t for t in dst if t not in src][:5]
    rng = random.Random(ns * 100 + bits)
    for trial in range(200):
        xs = [rng.randrange(q) for q in src]
        if trial == 0:
            xs = [q - 1 for q in src]
        unscaled = [x * N % q for x, q in zip(xs, src)]
        assert conversion_replay(unscaled, src, dst) == fast_bconv_definition(xs, src, dst)


@pytest.mark.parametrize("dnum,bits", [(1, 60), (3, 50), (3, 60), (8, 59)])
def test_key_product_halves_form_equals_the_sum(dnum, bits):
    """acc_t = sum_j y_j key_j mod t with keys stored as key 2^64 (times
    P^{-1} on the limbs of Q): the Montgomery reduction of the halves sum
    returns the plain sum (times P^{-1})."""
    t = primes([bits])[0]
    P_inv = random.Random(1).randrange(1, t)  # any stored factor rides through unchanged
    rng = random.Random(dnum * 10 + bits)
    for trial in range(300):
        ys = [rng.randrange(t) for _ in range(dnum)]
        ks = [rng.randrange(t) for _ in range(dnum)]
        if trial == 0:
            ys, ks = [t - 1] * dnum, [t - 1] * dnum
        stored = [k * P_inv % t * (1 << 64) % t for k in ks]
        s = acc30_sum(ys, stored)
        assert (s >> 64) < t
        assert redc(s & M64, s >> 64, t) == sum(y * k for y, k in zip(ys, ks)) * P_inv % t


def tensor_replay(xs, ws, q, chunk):
    """k_tensor_acc for one coefficient: 128-bit sums a0 = sum x0 w0,
    s = sum (x0 + x1)(w0 + w1), a2 = sum x1 w1, folded to residues every
    `chunk` terms with s carrying r0 + r1 + r2; the middle output is
    s - a0 - a2 (k_tensor_pair is the one-term case)."""
    from test_modular_bounds_host import reduce128_est

    def red(v):
        assert 0 <= v < 1 << 128
        return reduce128_est(v & M64, v >> 64, q)

    a0 = s = a2 = 0
    for cnt, ((x0, x1), (w0, w1)) in enumerate(zip(xs, ws), 1):
        a0 += x0 * w0
        s += (x0 + x1) * (w0 + w1)
        a2 += x1 * w1
        assert s < 1 << 128
        if cnt % chunk == 0:
            r1 = red(s - a0 - a2)
            r0, r2 = red(a0), red(a2)
            a0, a2, s = r0, r2, r0 + r1 + r2
    return red(a0), red(s - a0 - a2), red(a2)


@pytest.mark.parametrize("terms,bits", [(1, 61), (25, 40), (25, 60), (150, 60), (1800, 61)])
def test_tensor_accumulation_equals_the_products(terms, bits):
    q = primes([bits])[0]
    lim = (1 << 128) - 1 - (1 << 64)
    per = lim // (4 * q * q)
    chunk = 1024 if per > 1024 else per - 1
    rng = random.Random(terms + bits)
    for trial in range(20 if terms > 100 else 100):
        if trial == 0:
            xs = [(q - 1, q - 1)] * terms
            ws = [(q - 1, q - 1)] * terms
        else:
            xs = [(rng.randrange(q), rng.randrange(q)) for _ in range(terms)]
            ws = [(rng.randrange(q), rng.randrange(q)) for _ in range(terms)]
        d0 = sum(x0 * w0 for (x0, _), (w0, _) in zip(xs, ws)) % q
        d1 = sum(x0 * w1 + x1 * w0 for (x0, x1), (w0, w1) in zip(xs, ws)) % q
        d2 = sum(x1 * w1 for (_, x1), (_, w1) in zip(xs, ws)) % q
        assert tensor_replay(xs, ws, q, chunk) == (d0, d1, d2)
