"""RNS-CKKS scheme, written step by step from its definitions (CPU oracle).

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares nothing with the GPU
library except the interface conventions listed below, which both sides
implement independently.

What the paper fixes and what is read into it
---------------------------------------------
The paper (Jain et al., arXiv 2102.00319) evaluates its CNN with the CKKS
scheme (Sec. "Proposed Approach", CKKS slots and SIMD packing; Sec.
"Impact of FHE parameters": ring from the cyclotomic polynomial, K = phi(m)/2
slots, modulus size L and precision r).  It uses HElib and does not spell out
the scheme's internals.  This module takes the standard full-RNS reading:

* Ring R_Q = Z_Q[X]/(X^N + 1), Q = q_0 q_1 ... q_L, primes q = 1 mod 2N,
  special modulus P = p_0 ... p_{alpha-1} for key switching.  Polynomials are
  kept in COEFFICIENT form, one limb of N residues per prime.
* Ciphertext at level l: polynomials over q_0..q_l; decryption
  m = c_0 + c_1 s (+ c_2 s^2 for the degree-2 tensor) mod Q_l.
* Key switching is hybrid (digit) key switching: digits are consecutive
  blocks of alpha primes from q_0; digit j at level l keeps the primes of the
  block that are <= l.  ModUp is the fast basis conversion of Cheon et al.
  (SAC 2018), the key for digit j carries P * s' on the limbs of its block
  only, ModDown subtracts the fast conversion of the P-part and multiplies by
  P^{-1}.
* Rescale divides by the last prime with centred (round-to-nearest)
  rounding; the scale, a double, is divided by that prime.
* Randomness: Philox4x64-10 counter streams, keyed by (seed, domain tag);
  the conventions (tags, word use, samplers) are in `_tags` and the C core.

Interface conventions shared (by definition, not by code) with the library:
prime chain selection, Philox stream layout and domain tags, sampler
definitions, digit blocks, the Galois element 5^r mod 2N for a left rotation
by r, constant encoding by round-half-away-from-zero, the scale tolerance of
additions and the canonical layer circuits in `oracle.cnn`.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from . import gaussian
from ._lib import as_u64, lib

# ---------------------------------------------------------------------------
# Domain tags of the Philox streams (key = (seed, tag)).
# ---------------------------------------------------------------------------
TAG_S = 1
TAG_PK_A = 2
TAG_PK_E = 3


def tag_swk_a(j: int, g: int = 0) -> int:
    """Uniform part of digit j of a switching key (g = 0: relinearisation)."""
    return (g << 16) | (0x100 + 2 * j)


def tag_swk_e(j: int, g: int = 0) -> int:
    return (g << 16) | (0x101 + 2 * j)


def tag_enc(nonce: int, which: int) -> int:
    """which = 0: v, 1: e0, 2: e1."""
    return (1 << 63) | (nonce << 2) | which


SCALE_RTOL = 2.0 ** -40  # additions accept scales equal up to this relative gap


def llround(x: float) -> int:
    """Round half away from zero, exactly (as C's llround on a double)."""
    f = Fraction(x)
    a = abs(f)
    n = math.floor(a + Fraction(1, 2))
    return n if f >= 0 else -n


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------
@dataclass
class Params:
    log_n: int
    q_bits: list
    p_bits: list
    log2_scale: float
    sigma: float = 3.2
    q: list = field(init=False)
    p: list = field(init=False)
    cdt: np.ndarray = field(init=False)

    def __post_init__(self):
        bits = np.array(list(self.q_bits) + list(self.p_bits), dtype=np.int32)
        out = np.zeros(len(bits), dtype=np.uint64)
        if lib().or_gen_primes(self.log_n, bits, len(bits), out) != 0:
            raise ValueError("no prime chain for these bit sizes")
        primes = [int(v) for v in out]
        self.q = primes[: len(self.q_bits)]
        self.p = primes[len(self.q_bits):]
        self.cdt = gaussian.cdt_table(self.sigma)

    @property
    def N(self) -> int:
        return 1 << self.log_n

    @property
    def K(self) -> int:
        return self.N // 2

    @property
    def L(self) -> int:
        return len(self.q) - 1

    @property
    def alpha(self) -> int:
        return len(self.p)

    @property
    def dnum(self) -> int:
        return -(-(self.L + 1) // self.alpha)

    @property
    def scale(self) -> float:
        return 2.0 ** self.log2_scale

    @property
    def chain(self) -> list:
        """All primes by chain index: q_0..q_L, then p_0..p_{alpha-1}."""
        return self.q + self.p

    def P(self) -> int:
        return math.prod(self.p)

    def digit(self, j: int, level: int) -> list:
        """Chain indices of digit j at level `level`."""
        lo = j * self.alpha
        return list(range(lo, min(lo + self.alpha, level + 1)))

    def dnum_at(self, level: int) -> int:
        return -(-(level + 1) // self.alpha)

    def ext_indices(self, level: int) -> list:
        """Chain indices of Q_level and P."""
        return list(range(level + 1)) + list(range(self.L + 1, self.L + 1 + self.alpha))

    def galois_elt(self, r: int) -> int:
        """Galois element of a left rotation by r slots: 5^r mod 2N."""
        return pow(5, r % self.K, 2 * self.N)


def primes_of(params: Params, idx) -> np.ndarray:
    ch = params.chain
    return np.array([ch[i] for i in idx], dtype=np.uint64)


# ---------------------------------------------------------------------------
# Polynomial helpers (all [limbs][N] uint64 arrays in coefficient form)
# ---------------------------------------------------------------------------
def pmul(a, b, primes):
    c = np.empty_like(a)
    lib().or_poly_mul(as_u64(a), as_u64(b), c, as_u64(primes), len(primes), a.shape[-1])
    return c


def padd(a, b, primes):
    c = np.empty_like(a)
    lib().or_poly_add(as_u64(a), as_u64(b), c, as_u64(primes), len(primes), a.shape[-1])
    return c


def psub(a, b, primes):
    c = np.empty_like(a)
    lib().or_poly_sub(as_u64(a), as_u64(b), c, as_u64(primes), len(primes), a.shape[-1])
    return c


def pneg(a, primes):
    c = np.empty_like(a)
    lib().or_poly_neg(as_u64(a), c, as_u64(primes), len(primes), a.shape[-1])
    return c


def pscalar(a, scalars, primes):
    c = np.empty_like(a)
    lib().or_poly_scalar_mul(as_u64(a), as_u64(scalars), c, as_u64(primes), len(primes), a.shape[-1])
    return c


def padd_const(a, scalars, primes):
    c = np.empty_like(a)
    lib().or_poly_add_const(as_u64(a), as_u64(scalars), c, as_u64(primes), len(primes), a.shape[-1])
    return c


def reduce_signed(v, primes):
    v = np.ascontiguousarray(v, dtype=np.int64)
    out = np.empty((len(primes), v.shape[0]), dtype=np.uint64)
    lib().or_reduce_signed(v, v.shape[0], as_u64(primes), len(primes), out)
    return out


def residues_of_int(x: int, primes) -> np.ndarray:
    return np.array([x % int(q) for q in primes], dtype=np.uint64)


def automorph(a, g, primes):
    c = np.empty_like(a)
    lib().or_automorph(as_u64(a), c, as_u64(primes), len(primes), a.shape[-1], g)
    return c


def fast_bconv(x, src, dst):
    n = x.shape[-1]
    y = np.empty((len(dst), n), dtype=np.uint64)
    lib().or_fast_bconv(as_u64(x), as_u64(src), len(src), y, as_u64(dst), len(dst), n)
    return y


# ---------------------------------------------------------------------------
# Samplers
# ---------------------------------------------------------------------------
def sample_ternary(params, seed, tag):
    out = np.empty(params.N, dtype=np.int64)
    lib().or_sample_ternary(seed, tag, params.N, out)
    return out


def sample_gauss(params, seed, tag):
    out = np.empty(params.N, dtype=np.int64)
    lib().or_sample_gauss(seed, tag, params.N, params.cdt, len(params.cdt), out)
    return out


def sample_uniform(params, seed, tag, chain_idx):
    """Uniform limbs for the given chain indices (lane = chain index)."""
    out = np.empty((len(chain_idx), params.N), dtype=np.uint64)
    for r, t in enumerate(chain_idx):
        row = np.empty(params.N, dtype=np.uint64)
        lib().or_sample_uniform(seed, tag, t, params.chain[t], params.N, row)
        out[r] = row
    return out


# ---------------------------------------------------------------------------
# Keys and ciphertexts
# ---------------------------------------------------------------------------
@dataclass
class SecretKey:
    s: np.ndarray  # int64 [N], ternary


@dataclass
class PublicKey:
    b: np.ndarray  # [L+1][N]
    a: np.ndarray


@dataclass
class SwitchKey:
    """Digit j: (b_j, a_j), each [L+1+alpha][N] over the whole chain."""
    b: list
    a: list


@dataclass
class EvalKeys:
    relin: SwitchKey
    galois: dict  # Galois element -> SwitchKey


@dataclass
class Plaintext:
    m: np.ndarray  # [level+1][N] residues
    level: int
    scale: float


@dataclass
class Ciphertext:
    c: np.ndarray  # [deg+1][level+1][N]
    level: int
    scale: float

    @property
    def degree(self) -> int:
        return self.c.shape[0] - 1


def _switch_key(params, sk, s_prime, seed, g):
    """Digit keys for switching s_prime -> s (Han-Ki hybrid, per-limb gadget).

    b_j = -a_j s + e_j + P [t in block j] s_prime   on every chain limb t.
    """
    chain_idx = list(range(params.L + 1 + params.alpha))
    primes = primes_of(params, chain_idx)
    s_res = reduce_signed(sk.s, primes)
    sp_res = s_prime if s_prime.dtype == np.uint64 else reduce_signed(s_prime, primes)
    P = params.P()
    bs, as_ = [], []
    for j in range(params.dnum):
        a = sample_uniform(params, seed, tag_swk_a(j, g), chain_idx)
        e = reduce_signed(sample_gauss(params, seed, tag_swk_e(j, g)), primes)
        b = psub(e, pmul(a, s_res, primes), primes)
        block = params.digit(j, params.L)
        gadget = np.array([P % int(primes[t]) if t in block else 0 for t in chain_idx], dtype=np.uint64)
        b = padd(b, pscalar(sp_res, gadget, primes), primes)
        bs.append(b)
        as_.append(a)
    return SwitchKey(bs, as_)


def keygen(params: Params, seed: int, rot_steps=()):
    """Secret, public and evaluation keys from one seed."""
    s = sample_ternary(params, seed, TAG_S)
    sk = SecretKey(s)
    q_idx = list(range(params.L + 1))
    qp = primes_of(params, q_idx)
    a = sample_uniform(params, seed, TAG_PK_A, q_idx)
    e = reduce_signed(sample_gauss(params, seed, TAG_PK_E), qp)
    s_q = reduce_signed(s, qp)
    b = psub(e, pmul(a, s_q, qp), qp)
    pk = PublicKey(b, a)
    all_idx = list(range(params.L + 1 + params.alpha))
    allp = primes_of(params, all_idx)
    s_all = reduce_signed(s, allp)
    s2 = pmul(s_all, s_all, allp)
    relin = _switch_key(params, sk, s2, seed, 0)
    galois = {}
    for r in rot_steps:
        g = params.galois_elt(r)
        if g == 1 or g in galois:
            continue
        sg = automorph(s_all, g, allp)
        galois[g] = _switch_key(params, sk, sg, seed, g)
    return sk, pk, EvalKeys(relin, galois)


def plaintext_from_ints(params, coeffs, level, scale) -> Plaintext:
    primes = primes_of(params, range(level + 1))
    return Plaintext(reduce_signed(np.asarray(coeffs, dtype=np.int64), primes), level, scale)


def encrypt(params, pk: PublicKey, pt: Plaintext, seed: int, nonce: int) -> Ciphertext:
    """Public-key encryption: (v b + e0 + m, v a + e1) on the limbs 0..level."""
    lv = pt.level
    primes = primes_of(params, range(lv + 1))
    v = reduce_signed(sample_ternary(params, seed, tag_enc(nonce, 0)), primes)
    e0 = reduce_signed(sample_gauss(params, seed, tag_enc(nonce, 1)), primes)
    e1 = reduce_signed(sample_gauss(params, seed, tag_enc(nonce, 2)), primes)
    c0 = padd(padd(pmul(v, pk.b[: lv + 1], primes), e0, primes), pt.m, primes)
    c1 = padd(pmul(v, pk.a[: lv + 1], primes), e1, primes)
    return Ciphertext(np.stack([c0, c1]), lv, pt.scale)


def decrypt(params, sk: SecretKey, ct: Ciphertext) -> Plaintext:
    """m = sum_k c_k s^k mod Q_level (residues)."""
    primes = primes_of(params, range(ct.level + 1))
    s = reduce_signed(sk.s, primes)
    m = ct.c[0].copy()
    sp = s
    for k in range(1, ct.degree + 1):
        m = padd(m, pmul(ct.c[k], sp, primes), primes)
        if k < ct.degree:
            sp = pmul(sp, s, primes)
    return Plaintext(m, ct.level, ct.scale)


# ---------------------------------------------------------------------------
# Homomorphic operations
# ---------------------------------------------------------------------------
def _check_scales(a: float, b: float):
    if abs(a - b) > SCALE_RTOL * max(abs(a), abs(b)):
        raise ValueError("scale mismatch")


def add(params, x: Ciphertext, y: Ciphertext) -> Ciphertext:
    if x.level != y.level or x.degree != y.degree:
        raise ValueError("level/degree mismatch")
    _check_scales(x.scale, y.scale)
    primes = primes_of(params, range(x.level + 1))
    return Ciphertext(np.stack([padd(x.c[k], y.c[k], primes) for k in range(x.degree + 1)]), x.level, x.scale)


def sub(params, x: Ciphertext, y: Ciphertext) -> Ciphertext:
    if x.level != y.level or x.degree != y.degree:
        raise ValueError("level/degree mismatch")
    _check_scales(x.scale, y.scale)
    primes = primes_of(params, range(x.level + 1))
    return Ciphertext(np.stack([psub(x.c[k], y.c[k], primes) for k in range(x.degree + 1)]), x.level, x.scale)


def add_const(params, x: Ciphertext, c: float) -> Ciphertext:
    """Adds the slot-constant c, encoded at the ciphertext's scale: the
    constant polynomial round(c * scale) (a CT-PT add)."""
    primes = primes_of(params, range(x.level + 1))
    m = residues_of_int(llround(c * x.scale), primes)
    out = x.c.copy()
    out[0] = padd_const(x.c[0], m, primes)
    return Ciphertext(out, x.level, x.scale)


def mul_const(params, x: Ciphertext, c: float, const_scale: float) -> Ciphertext:
    """Multiplies by the slot-constant c encoded at const_scale: every limb is
    multiplied by round(c * const_scale); the scale multiplies (a CT-PT mult,
    no rescale)."""
    primes = primes_of(params, range(x.level + 1))
    m = residues_of_int(llround(c * const_scale), primes)
    out = np.stack([pscalar(x.c[k], m, primes) for k in range(x.degree + 1)])
    return Ciphertext(out, x.level, x.scale * const_scale)


def mul(params, x: Ciphertext, y: Ciphertext) -> Ciphertext:
    """Tensor product (CT-CT mult before relinearisation):
    (a0 b0, a0 b1 + a1 b0, a1 b1); the scale multiplies."""
    if x.level != y.level or x.degree != 1 or y.degree != 1:
        raise ValueError("mul needs two degree-1 ciphertexts at one level")
    primes = primes_of(params, range(x.level + 1))
    a0, a1 = x.c
    b0, b1 = y.c
    d0 = pmul(a0, b0, primes)
    d1 = padd(pmul(a0, b1, primes), pmul(a1, b0, primes), primes)
    d2 = pmul(a1, b1, primes)
    return Ciphertext(np.stack([d0, d1, d2]), x.level, x.scale * y.scale)


def tensor_sum(params, xs, ys) -> Ciphertext:
    """Sum of tensor products sum_k xs[k] (x) ys[k] (one level, degree 2)."""
    acc = None
    for x, y in zip(xs, ys):
        t = mul(params, x, y)
        acc = t if acc is None else Ciphertext(
            np.stack([padd(acc.c[k], t.c[k], primes_of(params, range(t.level + 1))) for k in range(3)]),
            t.level, acc.scale)
    return acc


def modup(params, x, level):
    """ModUp of a coefficient-form polynomial over Q_level: for each digit j,
    the limbs over Q_level u P of the integer y_j = FastBConv([x]_{D_j}),
    y_j = x on the digit's own limbs.  Returns a list over digits of
    [len(ext)][N] arrays in `ext_indices(level)` order."""
    ext = params.ext_indices(level)
    out = []
    for j in range(params.dnum_at(level)):
        block = params.digit(j, level)
        others = [t for t in ext if t not in block]
        y = fast_bconv(x[block], primes_of(params, block), primes_of(params, others))
        full = np.empty((len(ext), params.N), dtype=np.uint64)
        for r, t in enumerate(ext):
            full[r] = x[t] if t in block else y[others.index(t)]
        out.append(full)
    return out


def key_product(params, ys, swk: SwitchKey, level):
    """(sum_j y_j b_j, sum_j y_j a_j) over Q_level u P."""
    ext = params.ext_indices(level)
    primes = primes_of(params, ext)
    u0 = np.zeros((len(ext), params.N), dtype=np.uint64)
    u1 = np.zeros_like(u0)
    for j, y in enumerate(ys):
        u0 = padd(u0, pmul(y, swk.b[j][ext], primes), primes)
        u1 = padd(u1, pmul(y, swk.a[j][ext], primes), primes)
    return u0, u1


def moddown(params, u, level):
    """(u - FastBConv_{P->Q}([u]_P)) * P^{-1} mod q_i for q_i in Q_level."""
    nq = level + 1
    q_idx = list(range(nq))
    p_idx = list(range(params.L + 1, params.L + 1 + params.alpha))
    qp = primes_of(params, q_idx)
    z = fast_bconv(u[nq:], primes_of(params, p_idx), qp)
    P = params.P()
    pinv = np.array([pow(P % int(q), -1, int(q)) for q in qp], dtype=np.uint64)
    return pscalar(psub(u[:nq], z, qp), pinv, qp)


def keyswitch(params, x, swk: SwitchKey, level):
    """Key switch of a single polynomial: returns (u0', u1') over Q_level."""
    ys = modup(params, x, level)
    u0, u1 = key_product(params, ys, swk, level)
    return moddown(params, u0, level), moddown(params, u1, level)


def relin(params, evk: EvalKeys, d: Ciphertext) -> Ciphertext:
    if d.degree != 2:
        raise ValueError("relin needs a degree-2 ciphertext")
    primes = primes_of(params, range(d.level + 1))
    u0, u1 = keyswitch(params, d.c[2], evk.relin, d.level)
    return Ciphertext(np.stack([padd(d.c[0], u0, primes), padd(d.c[1], u1, primes)]), d.level, d.scale)


def rescale(params, x: Ciphertext) -> Ciphertext:
    if x.level < 1:
        raise ValueError("no level left to rescale")
    primes = primes_of(params, range(x.level + 1))
    out = np.empty((x.degree + 1, x.level, params.N), dtype=np.uint64)
    for k in range(x.degree + 1):
        lib().or_rescale(as_u64(x.c[k]), out[k], primes, x.level + 1, params.N)
    return Ciphertext(out, x.level - 1, x.scale / float(params.q[x.level]))


def drop_to_level(params, x: Ciphertext, level: int) -> Ciphertext:
    if level > x.level or level < 0:
        raise ValueError("bad level")
    return Ciphertext(x.c[:, : level + 1].copy(), level, x.scale)


def rotate(params, evk: EvalKeys, x: Ciphertext, r: int) -> Ciphertext:
    """Left rotation of the slots by r: kappa_g with g = 5^r mod 2N, then a
    key switch from kappa_g(s) back to s."""
    g = params.galois_elt(r)
    if g == 1:
        return Ciphertext(x.c.copy(), x.level, x.scale)
    if g not in evk.galois:
        raise KeyError("no Galois key for rotation %d" % r)
    primes = primes_of(params, range(x.level + 1))
    c0 = automorph(x.c[0], g, primes)
    c1 = automorph(x.c[1], g, primes)
    u0, u1 = keyswitch(params, c1, evk.galois[g], x.level)
    return Ciphertext(np.stack([padd(c0, u0, primes), u1]), x.level, x.scale)


def rotate_hoisted(params, evk: EvalKeys, x: Ciphertext, steps):
    """Several rotations sharing one ModUp of c1: the automorphism is applied
    to each extended digit (limb by limb) before the key product.  Not
    bit-identical to `rotate` (ModUp does not commute with the sign flips of
    kappa_g), but decrypts to the same slots."""
    lv = x.level
    primes = primes_of(params, range(lv + 1))
    ext = params.ext_indices(lv)
    eprimes = primes_of(params, ext)
    ys = modup(params, x.c[1], lv)
    outs = []
    for r in steps:
        g = params.galois_elt(r)
        if g == 1:
            outs.append(Ciphertext(x.c.copy(), lv, x.scale))
            continue
        if g not in evk.galois:
            raise KeyError("no Galois key for rotation %d" % r)
        ysg = [automorph(y, g, eprimes) for y in ys]
        u0, u1 = key_product(params, ysg, evk.galois[g], lv)
        u0, u1 = moddown(params, u0, lv), moddown(params, u1, lv)
        c0 = automorph(x.c[0], g, primes)
        outs.append(Ciphertext(np.stack([padd(c0, u0, primes), u1]), lv, x.scale))
    return outs
