"""Exact noise identity of the oracle's hybrid key switch (relinearisation
and Galois keys), checked in integers on tiny rings.

For a coefficient-form x over Q_l, digit j keeps the primes D_j of its
block and raises y_j = sum_{i in D_j} [x_i (D_j/q_i)^{-1}]_{q_i} (D_j/q_i),
an integer with y_j = x mod D_j and 0 <= y_j < |D_j| D_j (fast basis
conversion).  The key of digit j satisfies b_j + a_j s = e_j + P g_j s' over
Q_L P, with g_j = 1 on the primes of block j and 0 elsewhere, so the key
product u_k = sum_j y_j (b_j, a_j) gives u_0 + u_1 s = E + P x s' mod Q_l P
with E = sum_j y_j e_j.  ModDown subtracts z_k = FastBConv_{P->Q}([u_k]_P),
an integer with z_k = u_k mod P and 0 <= z_k < alpha P, and divides by P.
Hence, exactly over the integers,

    KS(x)_0 + KS(x)_1 s = x s' + R  (mod Q_l),   R = (E - z_0 - z_1 s) / P,

where P divides E - z_0 - z_1 s exactly, and |R| <= |E|_inf / P +
alpha (1 + |s|_1).  Every quantity on the right is recomputed here from its
definition with Python integers (the e_j from the key-generation streams),
not with the oracle's key-switch code.  A wrong gadget, a missing P^{-1}, a
wrong ModDown sign or a conversion from the wrong digit breaks the identity
(the mutation tests below).
"""
import math

import numpy as np
import pytest

from oracle import ckks


def negamul(a, b):
    """Integer product in Z[X]/(X^N + 1) (Python ints)."""
    n = len(a)
    out = [0] * n
    for i, ai in enumerate(a):
        if ai == 0:
            continue
        for j, bj in enumerate(b):
            k = i + j
            if k < n:
                out[k] += ai * bj
            else:
                out[k - n] -= ai * bj
    return out


def fbconv_int(residues, moduli):
    """The integer sum_i [r_i (M/m_i)^{-1}]_{m_i} (M/m_i), per coefficient."""
    M = math.prod(moduli)
    n = len(residues[0])
    out = [0] * n
    for r, m in zip(residues, moduli):
        h = M // m
        hinv = pow(h % m, -1, m)
        for c in range(n):
            out[c] += (int(r[c]) * hinv % m) * h
    return out


def identity_holds(p, sk, swk, seed, g, s_prime, x, level, out0, out1):
    """True iff KS output (out0, out1) of x at `level` satisfies the exact
    identity of the module docstring for the switch s_prime -> s."""
    n = p.N
    chain = [int(v) for v in p.chain]
    qs = chain[: level + 1]
    ps = chain[p.L + 1: p.L + 1 + p.alpha]
    P = math.prod(ps)
    s = [int(v) for v in sk.s]
    ys = []
    for j in range(p.dnum_at(level)):
        block = p.digit(j, level)
        D = [chain[t] for t in block]
        y = fbconv_int([x[t] for t in block], D)
        # the raised digit is x modulo each of its primes, and below |D_j| D_j
        if any(y[c] % q != int(x[t][c]) for t, q in zip(block, D) for c in range(n)):
            return False
        if any(not (0 <= v < len(D) * math.prod(D)) for v in y):
            return False
        ys.append(y)
    E = [0] * n
    for j, y in enumerate(ys):
        e = [int(v) for v in ckks.sample_gauss(p, seed, ckks.tag_swk_e(j, g))]
        E = [a + b for a, b in zip(E, negamul(y, e))]
    # key product on the special primes, then ModDown's conversion integers
    z = []
    for k, key in enumerate((swk.b, swk.a)):
        u_p = []
        for r, pr in enumerate(ps):
            t = p.L + 1 + r
            acc = [0] * n
            for j, y in enumerate(ys):
                prod = negamul([v % pr for v in y], [int(v) for v in key[j][t]])
                acc = [(a + b) % pr for a, b in zip(acc, prod)]
            u_p.append(acc)
        z.append(fbconv_int(u_p, ps))
    num = [e - z0 - z1s for e, z0, z1s in zip(E, z[0], negamul(z[1], s))]
    if any(v % P for v in num):
        return False
    R = [v // P for v in num]
    bound = max(abs(v) for v in E) / P + p.alpha * (1 + sum(abs(v) for v in s))
    if max(abs(v) for v in R) > bound:
        return False
    xs = [[int(x[i][c]) for c in range(n)] for i in range(level + 1)]
    sp = [int(v) for v in s_prime]
    for i, q in enumerate(qs):
        lhs = [(a + b) % q for a, b in zip((int(v) for v in out0[i]), negamul([int(v) for v in out1[i]], s))]
        rhs = [(a + b) % q for a, b in zip(negamul(xs[i], sp), R)]
        if lhs != rhs:
            return False
    return True


def s_squared(sk):
    return negamul([int(v) for v in sk.s], [int(v) for v in sk.s])


def s_galois(p, sk, g):
    """kappa_g(s): coefficient i goes to i g mod 2N, negated past N."""
    n = p.N
    out = [0] * n
    for i, v in enumerate(int(t) for t in sk.s):
        k = (i * g) % (2 * n)
        if k < n:
            out[k] += v
        else:
            out[k - n] -= v
    return out


PARAMS = [
    # (log_n, q bits, p bits, log2 scale): dnum = 2 with a truncated digit at
    # level 2; dnum = 3 at the top level with a one-prime last digit; alpha = 1
    (5, [60, 40, 40, 40], [60, 60], 40),
    (5, [60, 50, 50, 50, 50, 50, 50], [60, 60, 60], 50),
    (5, [60, 40, 40], [60], 40),
]


@pytest.fixture(scope="module", params=PARAMS, ids=["dnum2", "dnum3", "alpha1"])
def keyed(request):
    log_n, qb, pb, ls = request.param
    p = ckks.Params(log_n, qb, pb, ls)
    seed = 77
    sk, pk, evk = ckks.keygen(p, seed, [1, 3])
    return p, sk, evk, seed


def _random_x(p, level, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, int(q), p.N, dtype=np.uint64) for q in p.chain[: level + 1]])


def test_relin_key_switch_identity_at_every_level(keyed):
    p, sk, evk, seed = keyed
    s2 = s_squared(sk)
    for level in range(p.L, -1, -1):
        x = _random_x(p, level, 10 + level)
        o0, o1 = ckks.keyswitch(p, x, evk.relin, level)
        assert identity_holds(p, sk, evk.relin, seed, 0, s2, x, level, o0, o1), level


def test_galois_key_switch_identity(keyed):
    p, sk, evk, seed = keyed
    for r in (1, 3):
        g = p.galois_elt(r)
        x = _random_x(p, p.L, 20 + r)
        o0, o1 = ckks.keyswitch(p, x, evk.galois[g], p.L)
        assert identity_holds(p, sk, evk.galois[g], seed, g, s_galois(p, sk, g), x, p.L, o0, o1), r


def test_relin_of_a_product_obeys_the_identity(keyed):
    """relin(d) - d keeps d0 + d1 s + d2 s^2 up to exactly R."""
    p, sk, evk, seed = keyed
    level = p.L
    rng = np.random.default_rng(3)
    cts = []
    for k in range(2):
        m = rng.integers(-2 ** 20, 2 ** 20, p.N)
        cts.append(ckks.encrypt(p, ckks.keygen(p, seed)[1], ckks.plaintext_from_ints(p, m, level, p.scale), 5, k))
    d = ckks.mul(p, cts[0], cts[1])
    r = ckks.relin(p, evk, d)
    qs = ckks.primes_of(p, range(level + 1))
    o0, o1 = ckks.psub(r.c[0], d.c[0], qs), ckks.psub(r.c[1], d.c[1], qs)
    assert identity_holds(p, sk, evk.relin, seed, 0, s_squared(sk), d.c[2], level, o0, o1)


# ------------------------------------------------------------ mutations
def _with_key(p, swk, fn):
    """A switching key whose digit limbs are fn(j, t, b, a) -> (b', a')."""
    bs, as_ = [], []
    for j in range(len(swk.b)):
        b, a = swk.b[j].copy(), swk.a[j].copy()
        for t in range(b.shape[0]):
            b[t], a[t] = fn(j, t, b[t], a[t])
        bs.append(b)
        as_.append(a)
    return ckks.SwitchKey(bs, as_)


def test_identity_rejects_a_gadget_of_one_instead_of_p():
    p = ckks.Params(*PARAMS[0])
    seed = 77
    sk, pk, evk = ckks.keygen(p, seed)
    s2 = s_squared(sk)
    chain = [int(v) for v in p.chain]
    P = math.prod(chain[p.L + 1:])
    s2_res = [[v % q for v in s2] for q in chain]

    def gadget_one(j, t, b, a):  # b_j carries s' instead of P s' on its block
        if t not in p.digit(j, p.L):
            return b, a
        q = chain[t]
        return np.array([(int(bv) - (P - 1) * s2_res[t][c]) % q for c, bv in enumerate(b)], dtype=np.uint64), a

    bad = _with_key(p, evk.relin, gadget_one)
    x = _random_x(p, p.L, 1)
    o0, o1 = ckks.keyswitch(p, x, bad, p.L)
    assert not identity_holds(p, sk, bad, seed, 0, s2, x, p.L, o0, o1)
    o0, o1 = ckks.keyswitch(p, x, evk.relin, p.L)
    assert identity_holds(p, sk, evk.relin, seed, 0, s2, x, p.L, o0, o1)


def test_identity_rejects_moddown_mutants(monkeypatch):
    p = ckks.Params(*PARAMS[0])
    seed = 77
    sk, pk, evk = ckks.keygen(p, seed)
    s2 = s_squared(sk)
    x = _random_x(p, p.L, 2)
    real = ckks.moddown

    def no_pinv(params, u, level):  # forgets the division by P
        nq = level + 1
        qp = ckks.primes_of(params, range(nq))
        pp = ckks.primes_of(params, range(params.L + 1, params.L + 1 + params.alpha))
        return ckks.psub(u[:nq], ckks.fast_bconv(u[nq:], pp, qp), qp)

    def plus_z(params, u, level):  # adds the conversion instead of subtracting it
        nq = level + 1
        qp = ckks.primes_of(params, range(nq))
        pp = ckks.primes_of(params, range(params.L + 1, params.L + 1 + params.alpha))
        P = params.P()
        pinv = np.array([pow(P % int(q), -1, int(q)) for q in qp], dtype=np.uint64)
        return ckks.pscalar(ckks.padd(u[:nq], ckks.fast_bconv(u[nq:], pp, qp), qp), pinv, qp)

    for mutant in (no_pinv, plus_z):
        monkeypatch.setattr(ckks, "moddown", mutant)
        o0, o1 = ckks.keyswitch(p, x, evk.relin, p.L)
        assert not identity_holds(p, sk, evk.relin, seed, 0, s2, x, p.L, o0, o1), mutant.__name__
    monkeypatch.setattr(ckks, "moddown", real)
    o0, o1 = ckks.keyswitch(p, x, evk.relin, p.L)
    assert identity_holds(p, sk, evk.relin, seed, 0, s2, x, p.L, o0, o1)


def test_identity_rejects_a_conversion_from_the_wrong_digit(monkeypatch):
    p = ckks.Params(*PARAMS[0])
    seed = 77
    sk, pk, evk = ckks.keygen(p, seed)
    s2 = s_squared(sk)
    x = _random_x(p, p.L, 3)
    real = ckks.modup

    def swapped(params, xx, level):  # digits raised in the opposite order
        return list(reversed(real(params, xx, level)))

    monkeypatch.setattr(ckks, "modup", swapped)
    o0, o1 = ckks.keyswitch(p, x, evk.relin, p.L)
    assert not identity_holds(p, sk, evk.relin, seed, 0, s2, x, p.L, o0, o1)


def test_identity_rejects_a_single_unit_change():
    p = ckks.Params(*PARAMS[2])
    seed = 77
    sk, pk, evk = ckks.keygen(p, seed)
    x = _random_x(p, p.L, 4)
    o0, o1 = ckks.keyswitch(p, x, evk.relin, p.L)
    assert identity_holds(p, sk, evk.relin, seed, 0, s_squared(sk), x, p.L, o0, o1)
    o0 = o0.copy()
    o0[1][5] = (int(o0[1][5]) + 1) % int(p.chain[1])
    assert not identity_holds(p, sk, evk.relin, seed, 0, s_squared(sk), x, p.L, o0, o1)
