"""CPU check of the lazy modular arithmetic the kernels rely on (no GPU):
the device helpers of csrc/hc_device.cuh and the 30-bit-halves sums of
csrc/hc_kernels.cu, restated with explicit 64-bit wrap-around, against exact
integer arithmetic at edge and random operands for the widest primes the
library accepts (below 2^61), and the tensor accumulation's fold interval
against its 128-bit bound."""
import random

import pytest

M64 = (1 << 64) - 1


def umulhi(a, b):
    return (a * b) >> 64


def shoup_of(w, q):
    return (w << 64) // q


def shoup_lazy(a, w, wsh, q):
    return (a * w - umulhi(a, wsh) * q) & M64


def mulhi_est(y, wsh):
    y0, y1 = y & 0xFFFFFFFF, y >> 32
    w0, w1 = wsh & 0xFFFFFFFF, wsh >> 32
    return (y1 * w1 + ((y1 * w0) >> 32) + ((y0 * w1) >> 32)) & M64


def shoup_lazy4(a, w, wsh, q):
    return (a * w - mulhi_est(a, wsh) * q) & M64


def csub(x, q):
    return x - q if x >= q else x


def reduce128(lo, hi, q):
    r64 = (1 << 64) % q
    t = shoup_lazy(hi, r64, shoup_of(r64, q), q)
    r = (lo - umulhi(lo, shoup_of(1, q)) * q) & M64
    s = t + r
    assert s < 4 * q
    return csub(csub(s, 2 * q), q)


def reduce128_est(lo, hi, q):
    r64 = (1 << 64) % q
    t = shoup_lazy4(hi, r64, shoup_of(r64, q), q)
    r = (lo - mulhi_est(lo, shoup_of(1, q)) * q) & M64
    s = t + r
    assert s < 8 * q and s <= M64
    return csub(csub(csub(s, 4 * q), 2 * q), q)


def redc(lo, hi, q):
    qinv = pow(q, -1, 1 << 64)
    mh = umulhi((lo * qinv) & M64, q)
    return hi - mh if hi >= mh else hi - mh + q


def is_prime(n):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d, s = d // 2, s + 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def largest_prime(bits, two_n=1 << 17):
    q = ((1 << bits) - 1) // two_n * two_n + 1
    while not is_prime(q):
        q -= two_n
    return q


PRIMES = [largest_prime(b) for b in (30, 40, 50, 60, 61)]


def operands(q, rng, count=300):
    edge = [0, 1, 2, q - 2, q - 1, q, 2 * q - 1, 4 * q - 1, (1 << 63) - 1, M64]
    return edge + [rng.randrange(1 << 64) for _ in range(count)]


@pytest.mark.parametrize("q", PRIMES)
def test_shoup_products(q):
    """a w - floor(a w' / 2^64) q is in [0, 2q) and congruent to a w for every
    64-bit a (w < q); with the estimated quotient it is in [0, 4q)."""
    rng = random.Random(q)
    for w in (0, 1, q - 1, rng.randrange(q), rng.randrange(q)):
        wsh = shoup_of(w, q)
        for a in operands(q, rng):
            r = shoup_lazy(a, w, wsh, q)
            assert r < 2 * q and r % q == a * w % q
            r4 = shoup_lazy4(a, w, wsh, q)
            assert r4 < 4 * q and r4 % q == a * w % q
            assert 0 <= umulhi(a, wsh) - mulhi_est(a, wsh) <= 2


@pytest.mark.parametrize("q", PRIMES)
def test_128_bit_reductions(q):
    rng = random.Random(q + 1)
    values = [0, 1, q - 1, q, (q - 1) * (q - 1), (1 << 128) - 1, ((q - 1) << 64) | M64]
    values += [rng.randrange(1 << 128) for _ in range(500)]
    for v in values:
        lo, hi = v & M64, v >> 64
        assert reduce128(lo, hi, q) == v % q
        assert reduce128_est(lo, hi, q) == v % q
        if hi < q:  # Montgomery: s 2^-64 mod q, fully reduced
            assert redc(lo, hi, q) == v * pow(1 << 64, -1, q) % q


def acc30_sum(vs, hs):
    """The halves sums of k_modup_bconv_h / k_key_product_t: lo, hi and the
    Karatsuba sum accumulated modulo 2^64, then assembled into 128 bits."""
    lo = hi = sm = 0
    for v, h in zip(vs, hs):
        vl, vh = v & ((1 << 30) - 1), v >> 30
        hl, hh = h & ((1 << 30) - 1), h >> 30
        assert vl + vh < (1 << 32) and hl + hh < (1 << 32)
        lo = (lo + vl * hl) & M64
        hi = (hi + vh * hh) & M64
        sm = (sm + (vl + vh) * (hl + hh)) & M64
    mid = (sm - lo - hi) & M64
    x = (lo + (mid << 30)) & M64
    c1 = 1 if x < lo else 0
    y = (x + (hi << 60)) & M64
    c2 = 1 if y < x else 0
    return ((mid >> 34) + (hi >> 4) + c1 + c2) << 64 | y


@pytest.mark.parametrize("terms", [1, 2, 7, 8])
def test_halves_sums_are_exact_up_to_eight_terms(terms):
    """Operands below 2^60, at most eight terms: the wrapped Karatsuba sum
    still yields the exact 128-bit value (its cross sum stays below 2^64)."""
    rng = random.Random(terms)
    top = (1 << 60) - 1
    cases = [([top] * terms, [top] * terms), ([0] * terms, [top] * terms)]
    cases += [([rng.randrange(1 << 60) for _ in range(terms)], [rng.randrange(1 << 60) for _ in range(terms)])
              for _ in range(300)]
    for vs, hs in cases:
        assert acc30_sum(vs, hs) == sum(v * h for v, h in zip(vs, hs))


def test_halves_sum_breaks_beyond_its_bound():
    """The bound is real: sixteen terms of operands near 2^60 wrap the cross
    sum, so the sums must not be used past eight terms."""
    top = (1 << 60) - 1
    assert acc30_sum([top] * 16, [top] * 16) != 16 * top * top


@pytest.mark.parametrize("q", PRIMES)
def test_conversion_sum_fits_montgomery_reduction(q):
    """A conversion output sums at most 8 products of a residue below 2^60
    and a constant below q_t, so its high word stays below q_t (REDC's
    precondition)."""
    v = (1 << 60) - 1
    assert (8 * v * (q - 1)) >> 64 < q


@pytest.mark.parametrize("q", PRIMES)
def test_tensor_accumulation_fold_interval(q):
    """k_tensor_acc folds its 128-bit sums every `chunk` terms, chunk chosen
    from the largest prime as in launch_tensor_acc: the Karatsuba sum gains
    (x0 + x1)(w0 + w1) < 4 q^2 per term on top of a folded value below 3 q,
    and must stay below 2^128."""
    lim = (1 << 128) - 1 - (1 << 64)
    per = lim // (4 * q * q)
    chunk = 1024 if per > 1024 else per - 1
    assert chunk >= 1
    worst = 3 * q + chunk * (2 * (q - 1)) ** 2
    assert worst < (1 << 128)
