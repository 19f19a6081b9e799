"""Pins of the oracle's scheme layer: exact noise identities of key generation
and encryption (integer convolutions, no modular reduction), closed forms of
the canonical embedding, sympy's CRT, and decryption against the FP64
network."""
import math

import numpy as np
import pytest

from oracle import ckks, cnn, encoding

sympy = pytest.importorskip("sympy")


def centred(residues, primes):
    return encoding.crt_centred(residues, primes)


def int_negacyclic(a, b):
    """Exact integer product in Z[X]/(X^N + 1) through np.convolve."""
    n = len(a)
    full = np.convolve(np.asarray(a, dtype=object), np.asarray(b, dtype=object))
    out = list(full[:n])
    for k in range(n - 1):
        out[k] -= full[n + k]
    return out


@pytest.fixture(scope="module")
def small():
    p = ckks.Params(6, [40, 30, 30], [40], 25)
    sk, pk, evk = ckks.keygen(p, 77, [1, 3])
    return p, sk, pk, evk


def test_crt_matches_sympy(small):
    p = small[0]
    rng = np.random.default_rng(1)
    res = np.stack([rng.integers(0, q, 8, dtype=np.uint64) for q in p.q])
    got = centred(res, p.q)
    Q = math.prod(p.q)
    for i in range(8):
        x = int(sympy.ntheory.modular.crt(p.q, [int(r[i]) for r in res])[0])
        if x > Q // 2:
            x -= Q
        assert got[i] == x


def test_public_key_identity(small):
    """b + a s = e exactly, with e the Gaussian error (|e| <= 19)."""
    p, sk, pk, _ = small
    e = ckks.sample_gauss(p, 77, ckks.TAG_PK_E)
    s_q = ckks.reduce_signed(sk.s, p.q)
    lhs = ckks.padd(pk.b, ckks.pmul(pk.a, s_q, p.q), p.q)
    assert centred(lhs, p.q) == [int(v) for v in e]


def test_switch_key_identity(small):
    """b_j + a_j s - P [t in block j] s' = e_j on every chain limb."""
    p, sk, _, evk = small
    chain = p.chain
    s_int = [int(v) for v in sk.s]
    s2 = int_negacyclic(s_int, s_int)
    P = p.P()
    for j in range(p.dnum):
        e = [int(v) for v in ckks.sample_gauss(p, 77, ckks.tag_swk_e(j))]
        block = p.digit(j, p.L)
        for t, qt in enumerate(chain):
            st = ckks.reduce_signed(sk.s, [qt])
            lhs = ckks.padd(evk.relin.b[j][t:t + 1], ckks.pmul(evk.relin.a[j][t:t + 1], st, [qt]), [qt])
            exp = [(e[i] + (P * s2[i] if t in block else 0)) % qt for i in range(p.N)]
            assert [int(v) for v in lhs[0]] == exp
    for g, swk in evk.galois.items():
        sg = [0] * p.N
        for i, v in enumerate(s_int):  # kappa_g(s) by index arithmetic on integers
            k = i * g % (2 * p.N)
            if k < p.N:
                sg[k] += v
            else:
                sg[k - p.N] -= v
        for j in range(p.dnum):
            e = [int(v) for v in ckks.sample_gauss(p, 77, ckks.tag_swk_e(j, g))]
            block = p.digit(j, p.L)
            for t, qt in enumerate(chain):
                st = ckks.reduce_signed(sk.s, [qt])
                lhs = ckks.padd(swk.b[j][t:t + 1], ckks.pmul(swk.a[j][t:t + 1], st, [qt]), [qt])
                exp = [(e[i] + (P * sg[i] if t in block else 0)) % qt for i in range(p.N)]
                assert [int(v) for v in lhs[0]] == exp


def test_encrypt_identity(small):
    """c0 + c1 s - m = v e + e0 + e1 s exactly (integer polynomial products)."""
    p, sk, pk, _ = small
    rng = np.random.default_rng(2)
    m = rng.integers(-10**6, 10**6, p.N)
    pt = ckks.plaintext_from_ints(p, m, p.L, p.scale)
    ct = ckks.encrypt(p, pk, pt, 5, 9)
    dec = ckks.decrypt(p, sk, ct)
    got = centred(ckks.psub(dec.m, pt.m, p.q), p.q)
    v = [int(x) for x in ckks.sample_ternary(p, 5, ckks.tag_enc(9, 0))]
    e0 = [int(x) for x in ckks.sample_gauss(p, 5, ckks.tag_enc(9, 1))]
    e1 = [int(x) for x in ckks.sample_gauss(p, 5, ckks.tag_enc(9, 2))]
    e = [int(x) for x in ckks.sample_gauss(p, 77, ckks.TAG_PK_E)]
    s = [int(x) for x in sk.s]
    ve = int_negacyclic(v, e)
    e1s = int_negacyclic(e1, s)
    assert got == [ve[i] + e0[i] + e1s[i] for i in range(p.N)]


# ------------------------------------------------------------- encoding ---
def test_encode_slot_constant_is_constant_polynomial():
    n, scale = 256, 2.0 ** 30
    for c in (0.3, -1.75, 1.0):
        m = encoding.encode(np.full(n // 2, c), n, scale)
        assert m[0] == ckks.llround(c * scale)
        assert np.all(m[1:] == 0)


def test_encode_evaluates_to_slots():
    """The integer polynomial evaluated at zeta^{5^j} (Horner in complex128)
    gives scale z_j up to the rounding of the coefficients."""
    n, scale = 128, 2.0 ** 30
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, n // 2) + 1j * rng.uniform(-1, 1, n // 2)
    m = encoding.encode(z, n, scale)
    for j in range(0, n // 2, 7):
        root = np.exp(1j * np.pi * pow(5, j, 2 * n) / n)
        val = np.polyval(m[::-1].astype(np.float64), root)
        assert abs(val / scale - z[j]) <= n / (2 * scale) + 1e-9


def test_decode_closed_forms():
    n, scale = 64, 2.0 ** 20
    q = [int(x) for x in ckks.Params(6, [50], [50], 20).q]
    # monomial X^k decodes to zeta^{5^j k} / scale
    k = 5
    m = np.zeros(n, dtype=np.int64)
    m[k] = 1
    z = encoding.decode(ckks.reduce_signed(m, q), q, n, 1.0)
    exp = np.array([np.exp(1j * np.pi * (pow(5, j, 2 * n) * k % (2 * n)) / n) for j in range(n // 2)])
    assert np.max(np.abs(z - exp)) < 1e-12
    # negative constant survives the centred lift
    m = np.zeros(n, dtype=np.int64)
    m[0] = -3 * 2**20
    z = encoding.decode(ckks.reduce_signed(m, q), q, n, scale)
    assert np.max(np.abs(z + 3)) < 1e-12


def test_encode_round_trip_and_homomorphism():
    n, scale = 256, 2.0 ** 30
    rng = np.random.default_rng(5)
    a = rng.uniform(-1, 1, n // 2)
    b = rng.uniform(-1, 1, n // 2)
    ma = encoding.encode(a, n, scale)
    mb = encoding.encode(b, n, scale)
    q = ckks.Params(8, [60, 60], [60], 30).q
    za = encoding.decode(ckks.reduce_signed(ma, q), q, n, scale)
    assert np.max(np.abs(za - a)) <= n / (2 * scale) + 1e-9
    prod = int_negacyclic([int(x) for x in ma], [int(x) for x in mb])
    zab = encoding.decode_coeffs([float(x) for x in prod], n, scale * scale)
    assert np.max(np.abs(zab - a * b)) < 1e-6


# --------------------------------------------------------- ciphertext ops ---
@pytest.fixture(scope="module")
def mid():
    p = ckks.Params(8, [60, 40, 40, 40], [60, 60], 40)
    sk, pk, evk = ckks.keygen(p, 99, [1, 2, 5, -1])
    return p, sk, pk, evk


def enc(p, pk, z, level=None, nonce=0):
    lv = p.L if level is None else level
    m = encoding.encode(z, p.N, p.scale)
    return ckks.encrypt(p, pk, ckks.plaintext_from_ints(p, m, lv, p.scale), 1234, nonce)


def dec(p, sk, ct):
    d = ckks.decrypt(p, sk, ct)
    return encoding.decode(d.m, p.q[: ct.level + 1], p.N, ct.scale)


def test_mul_relin_rescale_decrypts_to_product(mid):
    p, sk, pk, evk = mid
    rng = np.random.default_rng(6)
    a, b = rng.uniform(-1, 1, p.K), rng.uniform(-1, 1, p.K)
    ca, cb = enc(p, pk, a, nonce=1), enc(p, pk, b, nonce=2)
    d = ckks.mul(p, ca, cb)
    # degree-2 decryption of the tensor already gives a*b
    assert np.max(np.abs(dec(p, sk, d) - a * b)) < 1e-7
    r = ckks.relin(p, evk, d)
    # relinearisation changes the decryption only by the key-switch noise
    diff = ckks.psub(ckks.decrypt(p, sk, r).m, ckks.decrypt(p, sk, d).m, p.q[: d.level + 1])
    assert max(abs(v) for v in centred(diff, p.q[: d.level + 1])) < 2 ** 12
    out = ckks.rescale(p, r)
    assert out.level == p.L - 1
    assert out.scale == d.scale / p.q[p.L]
    assert np.max(np.abs(dec(p, sk, out) - a * b)) < 1e-7


def test_mul_with_two_digit_key_switch():
    """alpha = 2 digits of two primes (the truncated last digit at level 2)."""
    p = ckks.Params(7, [60, 40, 40, 40], [60, 60], 40)
    assert p.dnum == 2
    sk, pk, evk = ckks.keygen(p, 5, [])
    rng = np.random.default_rng(7)
    a, b = rng.uniform(-1, 1, p.K), rng.uniform(-1, 1, p.K)
    for lv in (3, 2):
        ca, cb = enc(p, pk, a, lv, 1), enc(p, pk, b, lv, 2)
        out = ckks.rescale(p, ckks.relin(p, evk, ckks.mul(p, ca, cb)))
        assert np.max(np.abs(dec(p, sk, out) - a * b)) < 1e-7


def test_rotation_is_cyclic_shift(mid):
    p, sk, pk, evk = mid
    z = np.random.default_rng(8).uniform(-1, 1, p.K)
    ct = enc(p, pk, z)
    for r in (1, 2, 5, -1, 0):
        out = ckks.rotate(p, evk, ct, r)
        assert np.max(np.abs(dec(p, sk, out) - np.roll(z, -r))) < 1e-7
    hs = ckks.rotate_hoisted(p, evk, ct, [1, 5, -1])
    for r, h in zip([1, 5, -1], hs):
        assert np.max(np.abs(dec(p, sk, h) - np.roll(z, -r))) < 1e-7
    with pytest.raises(KeyError):
        ckks.rotate(p, evk, ct, 3)


def test_constants_and_levels(mid):
    p, sk, pk, evk = mid
    z = np.random.default_rng(9).uniform(-1, 1, p.K)
    ct = enc(p, pk, z)
    assert np.max(np.abs(dec(p, sk, ckks.add_const(p, ct, 0.47)) - (z + 0.47))) < 1e-8
    mc = ckks.mul_const(p, ct, -0.25, float(p.q[p.L]))
    assert np.max(np.abs(dec(p, sk, ckks.rescale(p, mc)) + 0.25 * z)) < 1e-8
    dropped = ckks.drop_to_level(p, ct, 1)
    assert np.max(np.abs(dec(p, sk, dropped) - z)) < 1e-8
    assert np.max(np.abs(dec(p, sk, ckks.add(p, ct, ct)) - 2 * z)) < 1e-8
    assert np.max(np.abs(dec(p, sk, ckks.sub(p, ct, ct)))) < 1e-8
    with pytest.raises(ValueError):
        ckks.add(p, ct, mc)
    with pytest.raises(ValueError):
        ckks.rescale(p, ckks.drop_to_level(p, ct, 0))


# ---------------------------------------------------------------- network ---
def test_fp64_network_against_scipy():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(10)
    x = rng.uniform(0, 1, (3, 9, 9, 1))
    w = rng.normal(0, 0.3, (2, 3, 3, 1))
    y = cnn.conv2d(x, w, stride=2)
    for b in range(3):
        for co in range(2):
            full = scipy_signal.correlate2d(x[b, :, :, 0], w[co, :, :, 0], mode="valid")
            assert np.allclose(y[b, :, :, co], full[::2, ::2])
    z = cnn.mean_pool2(y)
    assert z.shape == (3, 2, 2, 2)
    assert np.isclose(z[1, 1, 0, 1], y[1, 2:4, 0:2, 1].mean())


def test_encrypted_layers_match_fp64():
    p = ckks.Params(8, [60, 40, 40, 40, 40, 40], [60], 40)
    sk, pk, evk = ckks.keygen(p, 3, [])
    rng = np.random.default_rng(11)
    B, H, W, Cout, k, s = p.K, 6, 6, 2, 3, 1
    x = rng.uniform(0, 1, (B, H, W, 1))
    w = rng.normal(0, 0.3, (Cout, k, k, 1))
    Ho = (H - k) // s + 1
    n_in = (Ho // 2) * (Ho // 2) * Cout
    fw = rng.normal(0, 0.3, (3, n_in))
    x_cts = [enc(p, pk, x[:, h, ww, 0], nonce=h * W + ww) for h in range(H) for ww in range(W)]
    w_cts = [enc(p, pk, np.full(p.K, w[co, a, b, 0]), nonce=100 + (co * k + a) * k + b)
             for co in range(Cout) for a in range(k) for b in range(k)]
    fw_cts = [enc(p, pk, np.full(p.K, fw[r, i]), nonce=200 + r * n_in + i) for r in range(3) for i in range(n_in)]
    y = cnn.enc_conv2d_batch(p, evk, x_cts, H, W, 1, w_cts, Cout, k, k, s)
    a = [cnn.enc_poly_act(p, evk, c, (0.0, 0.0, 1.0)) for c in y]
    pool = cnn.enc_pool_batch(p, a, Cout, Ho, Ho)
    logits = cnn.enc_fc(p, evk, pool, fw_cts, 3)
    ref = cnn.network(x, w, s, (0.0, 0.0, 1.0), fw)
    got = np.stack([dec(p, sk, z).real for z in logits], axis=1)
    assert np.max(np.abs(got - ref)) < 2.0 ** -15
    # the paper's activation g (two levels) on one conv output
    g = cnn.enc_poly_act(p, evk, y[0], (0.47, 0.50, 0.09))
    yref = cnn.conv2d(x, w, s)[:, 0, 0, 0]
    assert np.max(np.abs(dec(p, sk, g).real - cnn.poly_act(yref, (0.47, 0.50, 0.09)))) < 2.0 ** -15


def test_single_packing_conv_matches_fp64():
    p = ckks.Params(8, [50, 30, 30], [50], 30)
    rots = cnn.conv_rotations(8, 3, 3)
    sk, pk, evk = ckks.keygen(p, 4, rots)
    rng = np.random.default_rng(12)
    img = rng.uniform(0, 1, (8, 8))
    w = rng.normal(0, 0.3, (3, 3))
    z = np.zeros(p.K)
    z[:64] = img.reshape(-1)
    x_ct = enc(p, pk, z)
    w_cts = [enc(p, pk, np.full(p.K, w[a, b]), nonce=10 + a * 3 + b) for a in range(3) for b in range(3)]
    y = cnn.enc_conv2d_single(p, evk, x_ct, 8, w_cts, 3, 3)
    y2 = cnn.enc_poly_act(p, evk, y, (0.0, 0.0, 1.0))
    ref = cnn.conv2d(img[None, :, :, None], w[None, :, :, None])[0, :, :, 0] ** 2
    got = dec(p, sk, y2).real
    for m in range(6):
        for n in range(6):
            assert abs(got[m * 8 + n] - ref[m, n]) < 1e-3
