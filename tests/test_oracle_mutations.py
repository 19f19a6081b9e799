"""The oracle's pins catch plausible mistakes: each test plants one mistake in
a CPU copy of an oracle step and shows that the check which the real oracle
passes rejects the mutant."""
import math

import numpy as np

from oracle import ckks
from oracle._lib import lib



def _primes(log_n, bits):
    out = np.zeros(len(bits), dtype=np.uint64)
    lib().or_gen_primes(log_n, np.array(bits, dtype=np.int32), len(bits), out)
    return [int(v) for v in out]


def _eval(coeffs, x, q):
    acc = 0
    for c in reversed([int(v) for v in coeffs]):
        acc = (acc * x + c) % q
    return acc


def _root(n, q):
    for g in range(2, 1000):
        psi = pow(g, (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            return psi


def product_ok(mul, n=32, q=None):
    """c = a b in Z_q[X]/(X^N+1) iff c(r) = a(r) b(r) at the roots of X^N+1."""
    q = q or _primes(5, [50])[0]
    rng = np.random.default_rng(1)
    a, b = rng.integers(0, q, n, dtype=np.uint64), rng.integers(0, q, n, dtype=np.uint64)
    c = mul(a, b, q)
    psi = _root(n, q)
    return all(_eval(c, pow(psi, 2 * k + 1, q), q) == _eval(a, pow(psi, 2 * k + 1, q), q) *
               _eval(b, pow(psi, 2 * k + 1, q), q) % q for k in range(4))


def test_product_pin_rejects_cyclic_convolution():
    def oracle_mul(a, b, q):
        return ckks.pmul(a[None], b[None], np.array([q], dtype=np.uint64))[0]

    def cyclic(a, b, q):
        n = len(a)
        return np.array([sum(int(a[i]) * int(b[(k - i) % n]) for i in range(n)) % q for k in range(n)],
                        dtype=np.uint64)

    assert product_ok(oracle_mul)
    assert not product_ok(cyclic)


def rescale_ok(rescale):
    primes = _primes(5, [60, 40, 40])
    n = 16
    rng = np.random.default_rng(2)
    c = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in primes])
    out = rescale(c, primes)
    Qv = math.prod(primes)
    for k in range(n):
        C = sum((int(c[l, k]) * pow(Qv // q, -1, q) % q) * (Qv // q) for l, q in enumerate(primes)) % Qv
        if C > Qv // 2:
            C -= Qv
        R = (2 * C + primes[-1]) // (2 * primes[-1])
        if any(int(out[l, k]) != R % primes[l] for l in range(2)):
            return False
    return True


def test_rescale_pin_rejects_floor_division():
    def oracle(c, primes):
        out = np.empty((2, c.shape[1]), dtype=np.uint64)
        lib().or_rescale(c, out, np.array(primes, dtype=np.uint64), 3, c.shape[1])
        return out

    def floor_mutant(c, primes):  # subtracts the unsigned residue (no centring)
        ql = primes[-1]
        return np.array([[(int(c[i, k]) - int(c[2, k])) * pow(ql, -1, primes[i]) % primes[i]
                          for k in range(c.shape[1])] for i in range(2)], dtype=np.uint64)

    assert rescale_ok(oracle)
    assert not rescale_ok(floor_mutant)


def bconv_ok(conv):
    src, dst = _primes(5, [50, 45, 40]), _primes(5, [60, 55])
    rng = np.random.default_rng(3)
    x = np.stack([rng.integers(0, q, 16, dtype=np.uint64) for q in src])
    y = conv(x, src, dst)
    D = math.prod(src)
    for c in range(16):
        yy = sum((int(x[i, c]) * pow(D // qi, -1, qi) % qi) * (D // qi) for i, qi in enumerate(src))
        if any(int(y[k, c]) != yy % t for k, t in enumerate(dst)):
            return False
    return True


def test_bconv_pin_rejects_reduction_mod_D():
    def oracle(x, src, dst):
        return ckks.fast_bconv(x, np.array(src, dtype=np.uint64), np.array(dst, dtype=np.uint64))

    def exact_crt(x, src, dst):  # the exact CRT lift (reduced mod D), not the fast conversion
        D = math.prod(src)
        out = np.zeros((len(dst), x.shape[1]), dtype=np.uint64)
        for c in range(x.shape[1]):
            yy = sum((int(x[i, c]) * pow(D // qi, -1, qi) % qi) * (D // qi) for i, qi in enumerate(src)) % D
            for k, t in enumerate(dst):
                out[k, c] = yy % t
        return out

    assert bconv_ok(oracle)
    assert not bconv_ok(exact_crt)


def automorph_ok(aut, g=5):
    n, q = 32, _primes(5, [50])[0]
    a = np.random.default_rng(4).integers(0, q, n, dtype=np.uint64)
    c = aut(a, g, q)
    psi = _root(n, q)
    return all(_eval(c, pow(psi, 2 * k + 1, q), q) == _eval(a, pow(pow(psi, 2 * k + 1, q), g, q), q) for k in range(4))


def test_automorphism_pin_rejects_missing_sign_flip():
    def oracle(a, g, q):
        return ckks.automorph(a[None], g, np.array([q], dtype=np.uint64))[0]

    def no_sign(a, g, q):
        n = len(a)
        out = np.zeros(n, dtype=np.uint64)
        for i in range(n):
            out[(i * g) % (2 * n) % n] = a[i]
        return out

    assert automorph_ok(oracle)
    assert not automorph_ok(no_sign)


def _philox(ctr, key, rounds):
    M0, M1 = 0xD2E7470EE14C6C93, 0xCA5A826395121157
    W0, W1 = 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B
    c, k = list(ctr), list(key)
    mask = (1 << 64) - 1
    for r in range(rounds):
        if r:
            k = [(k[0] + W0) & mask, (k[1] + W1) & mask]
        p0, p1 = M0 * c[0], M1 * c[2]
        c = [(p1 >> 64) ^ c[1] ^ k[0], p1 & mask, (p0 >> 64) ^ c[3] ^ k[1], p0 & mask]
    return c


def test_philox_pin_rejects_nine_rounds():
    ctr, key = (7, 1, 0, 0), (11, 13)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array((6, 1, 0, 0), dtype=np.uint64))
    kat = [int(v) for v in bg.random_raw(4)]
    assert _philox(ctr, key, 10) == kat
    assert _philox(ctr, key, 9) != kat


def test_public_key_pin_rejects_sign_error():
    p = ckks.Params(5, [40], [40], 20)
    s = ckks.sample_ternary(p, 9, ckks.TAG_S)
    a = ckks.sample_uniform(p, 9, ckks.TAG_PK_A, [0])
    e = ckks.reduce_signed(ckks.sample_gauss(p, 9, ckks.TAG_PK_E), p.q)
    s_q = ckks.reduce_signed(s, p.q)
    good = ckks.psub(e, ckks.pmul(a, s_q, p.q), p.q)   # b = -a s + e
    bad = ckks.padd(e, ckks.pmul(a, s_q, p.q), p.q)    # b = a s + e

    def identity_small(b):
        r = ckks.padd(b, ckks.pmul(a, s_q, p.q), p.q)[0]
        q = p.q[0]
        return all(min(int(v), q - int(v)) <= 19 for v in r)

    assert identity_small(good)
    assert not identity_small(bad)


def _automorph_int(m, g):
    """kappa_g on an integer polynomial: X^i -> X^{i g} in Z[X]/(X^N + 1)."""
    n = len(m)
    out = np.zeros(n, dtype=np.float64)
    for i, c in enumerate(m):
        e = (i * g) % (2 * n)
        if e < n:
            out[e] += c
        else:
            out[e - n] -= c
    return out


def rotation_ok(encode_real, decode_real, n=64):
    """Slot rotation pin: kappa_5 of an encoded vector decodes to the vector
    shifted left by one slot."""
    z = np.random.default_rng(9).uniform(-1, 1, n // 2)
    m = encode_real(z, n)
    back = decode_real(_automorph_int(m, 5), n)
    return np.max(np.abs(back - np.roll(z, -1))) < 1e-9


def test_rotation_pin_rejects_slot_order_by_generator_3(monkeypatch):
    from oracle import encoding

    def enc(z, n):
        return encoding.encode_real_coeffs(z, n, 1.0)

    def dec(m, n):
        return encoding.decode_coeffs(m, n, 1.0).real

    assert rotation_ok(enc, dec)

    def group_of_3(n):  # slots ordered by powers of 3 instead of 5
        out = np.empty(n // 2, dtype=np.int64)
        g = 1
        for j in range(n // 2):
            out[j] = g
            g = (g * 3) % (2 * n)
        return out

    monkeypatch.setattr(encoding, "_rot_group", group_of_3)
    assert not rotation_ok(enc, dec)
