"""Pins of the oracle's arithmetic layer against things other than itself:
numpy's Philox, sympy's primality test, big-integer brute force, polynomial
evaluation at the roots of X^N + 1, exact CRT, mpmath."""
import math
import random

import numpy as np
import pytest

import oracle
from oracle import ckks, gaussian
from oracle._lib import lib

sympy = pytest.importorskip("sympy")


# ---------------------------------------------------------------- Philox ---
def numpy_philox_block(ctr, key):
    """Philox4x64-10 block for counter `ctr` via numpy's generator, which
    increments its 256-bit counter before each block."""
    c = list(ctr)
    # subtract one from the little-endian 256-bit counter
    for i in range(4):
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = (1 << 64) - 1  # borrow (all-zero wraps to all-ones)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (1, 2)),
    ((0, 0, 0, 0), (0, 0)),
    ((12345, 7, 0, 0), (0xDEADBEEF, 0x101)),
    ((0, 3, 0, 0), (2**64 - 1, 2**63 | 17)),
    ((2**64 - 1, 2**64 - 1, 5, 9), (3, 4)),
])
def test_philox_kat_numpy(ctr, key):
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(np.array(ctr, dtype=np.uint64), np.array(key, dtype=np.uint64), out)
    assert [int(v) for v in out] == numpy_philox_block(ctr, key)


def stream_words(seed, tag, lane, count):
    """Words of stream (seed, tag, lane) from numpy's Philox, counter (b, lane, 0, 0)."""
    words = []
    b = 0
    while len(words) < count:
        words += numpy_philox_block((b, lane, 0, 0), (seed, tag))
        b += 1
    return words[:count]


def test_sampler_stream_layout():
    p = ckks.Params(6, [30, 30], [30], 20)
    seed, tag = 0x1234, ckks.tag_enc(5, 0)
    w = stream_words(seed, tag, 0, p.N)
    assert list(ckks.sample_ternary(p, seed, tag)) == [int(x % 3) - 1 for x in w]
    g = ckks.sample_gauss(p, seed, tag)
    cdt = [int(v) for v in p.cdt]
    exp = []
    for x in w:
        mag = sum(1 for t in cdt if (x >> 1) >= t)
        exp.append(-mag if x & 1 else mag)
    assert list(g) == exp
    lane = 2
    wu = stream_words(seed, tag, lane, 2 * p.N)
    u = ckks.sample_uniform(p, seed, tag, [lane])[0]
    q = p.chain[lane]
    assert [int(v) for v in u] == [((wu[2 * i + 1] << 64) | wu[2 * i]) % q for i in range(p.N)]


def test_sampler_statistics():
    p = ckks.Params(14, [40], [40], 20)
    t = ckks.sample_ternary(p, 7, 1)
    counts = np.bincount(t + 1, minlength=3) / p.N
    assert np.all(np.abs(counts - 1 / 3) < 0.02)
    g = np.concatenate([ckks.sample_gauss(p, 7, tag) for tag in range(3, 8)])
    assert abs(np.mean(g)) < 0.05
    assert abs(np.std(g) - 3.2) < 0.05
    assert np.max(np.abs(g)) <= gaussian.tail_cut(3.2)
    u = ckks.sample_uniform(p, 7, 2, [0])[0].astype(np.float64) / p.q[0]
    assert abs(np.mean(u) - 0.5) < 0.01


# ------------------------------------------------------------------- CDT ---
def test_cdt_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 100
    sigma = mpmath.mpf(3.2)  # the double nearest 3.2, exactly
    tail = 19
    rho = [mpmath.e ** (-(k * k) / (2 * sigma * sigma)) for k in range(tail + 1)]
    z = rho[0] + 2 * sum(rho[1:])
    cum = mpmath.mpf(0)
    exp = []
    for k in range(tail):
        cum += (rho[0] if k == 0 else 2 * rho[k]) / z
        exp.append(int(mpmath.floor(cum * mpmath.mpf(2) ** 63)))
    assert [int(v) for v in gaussian.cdt_table(3.2)] == exp


# ---------------------------------------------------------------- primes ---
def test_is_prime_matches_sympy():
    rng = random.Random(5)
    cands = [rng.getrandbits(64) | 1 for _ in range(300)]
    cands += [561, 1105, 1729, 2465, 3215031751, 3825123056546413051, 2**61 - 1, 2**64 - 59, 1, 2, 3, 4]
    for c in cands:
        assert bool(lib().or_is_prime(c)) == sympy.isprime(c), c


@pytest.mark.parametrize("log_n,bits", [(10, [30, 30, 25, 30]), (12, [50, 30, 30, 50]), (16, [60, 50, 50, 60])])
def test_prime_chain_is_largest_unused(log_n, bits):
    out = np.zeros(len(bits), dtype=np.uint64)
    assert lib().or_gen_primes(log_n, np.array(bits, dtype=np.int32), len(bits), out) == 0
    primes = [int(v) for v in out]
    two_n = 2 << log_n
    assert len(set(primes)) == len(primes)
    for i, (q, b) in enumerate(zip(primes, bits)):
        assert sympy.isprime(q) and q % two_n == 1 and q.bit_length() == b
        # every larger candidate of that size is composite or already taken
        c = q + two_n
        while c < (1 << b):
            assert (not sympy.isprime(c)) or c in primes[:i], (i, c)
            c += two_n


# ------------------------------------------------------ negacyclic product ---
def eval_poly(coeffs, x, q):
    acc = 0
    for c in reversed([int(v) for v in coeffs]):
        acc = (acc * x + c) % q
    return acc


def roots_of_xn_plus_1(n, q, count):
    """Some roots of X^N + 1 mod q: odd powers of a primitive 2N-th root."""
    for g in range(2, 1000):
        psi = pow(g, (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            break
    return [pow(psi, 2 * k + 1, q) for k in range(count)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("log_n", [4, 6, 8, 10])
def test_negacyclic_product_at_roots(mode, log_n):
    """c = a b mod (X^N + 1, q) iff c(r) = a(r) b(r) at every root r of X^N + 1."""
    n = 1 << log_n
    primes = np.zeros(2, dtype=np.uint64)
    lib().or_gen_primes(log_n, np.array([60, 40], dtype=np.int32), 2, primes)
    rng = np.random.default_rng(log_n)
    a = np.stack([rng.integers(0, int(q), n, dtype=np.uint64) for q in primes])
    b = np.stack([rng.integers(0, int(q), n, dtype=np.uint64) for q in primes])
    lib().or_set_mode(mode)
    try:
        c = ckks.pmul(a, b, primes)
    finally:
        lib().or_set_mode(-1)
    for l, q in enumerate(int(v) for v in primes):
        for r in roots_of_xn_plus_1(n, q, 3):
            assert eval_poly(c[l], r, q) == eval_poly(a[l], r, q) * eval_poly(b[l], r, q) % q


@pytest.mark.parametrize("log_n", [4, 7, 10, 12])
def test_ntt_mode_equals_schoolbook(log_n):
    n = 1 << log_n
    primes = np.zeros(3, dtype=np.uint64)
    lib().or_gen_primes(log_n, np.array([60, 50, 30], dtype=np.int32), 3, primes)
    rng = np.random.default_rng(100 + log_n)
    a = np.stack([rng.integers(0, int(q), n, dtype=np.uint64) for q in primes])
    b = np.stack([rng.integers(0, int(q), n, dtype=np.uint64) for q in primes])
    lib().or_set_mode(0)
    c0 = ckks.pmul(a, b, primes)
    lib().or_set_mode(1)
    c1 = ckks.pmul(a, b, primes)
    lib().or_set_mode(-1)
    assert np.array_equal(c0, c1)


def test_negacyclic_small_integer_bruteforce():
    """Against an integer convolution folded by X^N = -1 (no modular step)."""
    n = 32
    rng = np.random.default_rng(3)
    a = rng.integers(-50, 50, n)
    b = rng.integers(-50, 50, n)
    full = np.convolve(a, b)
    exp = full[:n].copy()
    exp[: n - 1] -= full[n:]
    primes = np.array([1 << 40], dtype=np.uint64)
    lib().or_gen_primes(5, np.array([40], dtype=np.int32), 1, primes)
    q = int(primes[0])
    c = ckks.pmul(ckks.reduce_signed(a, primes), ckks.reduce_signed(b, primes), primes)
    assert [int(v) for v in c[0]] == [int(v) % q for v in exp]


# ------------------------------------------------------------ automorphism ---
@pytest.mark.parametrize("g", [5, 25, 3, 2 * 64 - 1])
def test_automorphism_is_substitution(g):
    """kappa_g(a)(r) = a(r^g) at roots r of X^N + 1."""
    n = 64
    primes = np.zeros(1, dtype=np.uint64)
    lib().or_gen_primes(6, np.array([50], dtype=np.int32), 1, primes)
    q = int(primes[0])
    a = np.random.default_rng(g).integers(0, q, (1, n), dtype=np.uint64)
    c = ckks.automorph(a, g, primes)
    for r in roots_of_xn_plus_1(n, q, 4):
        assert eval_poly(c[0], r, q) == eval_poly(a[0], pow(r, g, q), q)


# -------------------------------------------------------- basis conversion ---
def test_fast_bconv_bigint_definition():
    primes = np.zeros(6, dtype=np.uint64)
    lib().or_gen_primes(5, np.array([50, 45, 40, 60, 55, 30], dtype=np.int32), 6, primes)
    src, dst = primes[:3], primes[3:]
    rng = np.random.default_rng(11)
    n = 32
    x = np.stack([rng.integers(0, int(q), n, dtype=np.uint64) for q in src])
    y = ckks.fast_bconv(x, src, dst)
    D = math.prod(int(q) for q in src)
    for c in range(n):
        yy = 0
        for i, qi in enumerate(int(q) for q in src):
            hat = D // qi
            yy += (int(x[i, c]) * pow(hat, -1, qi) % qi) * hat
        # invariants of the fast conversion
        assert 0 <= yy < len(src) * D
        for i, qi in enumerate(int(q) for q in src):
            assert yy % qi == int(x[i, c])
        for k, t in enumerate(int(q) for q in dst):
            assert int(y[k, c]) == yy % t


# ----------------------------------------------------------------- rescale ---
def test_rescale_closed_form():
    """rescale(c) = round(C / q_l) for the centred CRT integer C of c."""
    primes = np.zeros(4, dtype=np.uint64)
    lib().or_gen_primes(5, np.array([60, 40, 40, 40], dtype=np.int32), 4, primes)
    n = 32
    rng = np.random.default_rng(21)
    c = np.stack([rng.integers(0, int(q), n, dtype=np.uint64) for q in primes])
    out = np.empty((3, n), dtype=np.uint64)
    lib().or_rescale(c, out, primes, 4, n)
    Q = math.prod(int(q) for q in primes)
    ql = int(primes[3])
    for k in range(n):
        C = 0
        for l, q in enumerate(int(v) for v in primes):
            hat = Q // q
            C += (int(c[l, k]) * pow(hat, -1, q) % q) * hat
        C %= Q
        if C > Q // 2:
            C -= Q
        num, den = 2 * C + ql, 2 * ql          # round(C/ql) = floor((2C + ql) / (2 ql))
        R = num // den
        for l in range(3):
            assert int(out[l, k]) == R % int(primes[l])


def test_llround_half_away_from_zero():
    assert ckks.llround(2.5) == 3 and ckks.llround(-2.5) == -3
    assert ckks.llround(0.49999999999999994) == 0
    assert ckks.llround(-0.5) == -1 and ckks.llround(1e18 + 0.0) == 10**18
