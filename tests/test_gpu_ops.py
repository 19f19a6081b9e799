"""GPU parity of the scheme operations against the CPU oracle, through the C
ABI.  Integer results are compared bit for bit in coefficient form."""
import numpy as np
import pytest

from oracle import ckks, encoding
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    from hc_pair import Pair
    # N = 2^10, five q primes and two special primes: dnum = 3 with a
    # truncated last digit; several NTT tiles per limb.
    return Pair(10, [60, 40, 40, 40, 40], [60, 60], 40, seed=11, rot_steps=[1, 3, -1, 5, 17])


@pytest.fixture(scope="module")
def pair12():
    from hc_pair import Pair
    return Pair(12, [50, 30, 30], [50], 30, seed=12, rot_steps=[1, 8])


def test_keys_bit_exact(pair):
    ctx = pair.ctx
    s = H.hc_sk_export(ctx, pair.g_sk)
    assert np.array_equal(s.astype(np.int64), pair.o_sk.s)
    pk = H.hc_pk_export(ctx, pair.g_pk)
    assert np.array_equal(pk[0], pair.o_pk.b) and np.array_equal(pk[1], pair.o_pk.a)
    rk = H.hc_evk_export(ctx, pair.g_evk, 1)
    for j in range(pair.op.dnum):
        assert np.array_equal(rk[j, 0], pair.o_evk.relin.b[j]), j
        assert np.array_equal(rk[j, 1], pair.o_evk.relin.a[j]), j
    for g, swk in pair.o_evk.galois.items():
        gk = H.hc_evk_export(ctx, pair.g_evk, g)
        for j in range(pair.op.dnum):
            assert np.array_equal(gk[j, 0], swk.b[j]) and np.array_equal(gk[j, 1], swk.a[j]), (g, j)


def test_encrypt_bit_exact_all_levels(pair):
    for lv in range(pair.op.L + 1):
        m = W.int_plaintext(100 + lv, pair.op.N, 2 ** 45)
        g, o = pair.encrypt(m, level=lv, nonce=lv)
        pair.assert_same(g, o, "encrypt level %d" % lv)


def test_import_export_roundtrip(pair):
    rng = W.rng(5)
    q = pair.op.q
    data = np.stack([np.stack([rng.integers(0, qi, pair.op.N, dtype=np.uint64) for qi in q[:4]]) for _ in range(2)])
    ct = H.hc_ct_import(pair.ctx, data, 3, 1, 2.0 ** 40)
    back, meta = H.hc_ct_export(pair.ctx, ct)
    assert np.array_equal(back, data) and meta.level == 3


def test_batch_import_export_match_single(pair):
    """The batched import/export calls give the single calls' results (mixed
    levels and degrees in one batch) and reject an out-of-range residue."""
    r = np.random.Generator(np.random.PCG64(77))
    n, q = pair.op.N, pair.op.q
    arrays, metas = [], []
    for lv, dg in [(3, 1), (1, 2), (3, 1), (0, 1)]:
        a = np.stack([np.stack([r.integers(0, q[j], n, dtype=np.uint64) for j in range(lv + 1)])
                      for _ in range(dg + 1)])
        arrays.append(np.ascontiguousarray(a))
        metas.append((lv, dg, 2.0 ** 40))
    cts = H.hc_ct_import_batch(pair.ctx, arrays, metas)
    singles = [H.hc_ct_import(pair.ctx, a, lv, dg, sc) for a, (lv, dg, sc) in zip(arrays, metas)]
    outs = [np.zeros_like(a) for a in arrays]
    H.hc_ct_export_batch(pair.ctx, cts, outs)
    for c, s1, a, o in zip(cts, singles, arrays, outs):
        np.testing.assert_array_equal(o, a)
        np.testing.assert_array_equal(H.hc_ct_export(pair.ctx, s1)[0], a)
        m = c.meta()
        assert (m.level, m.degree) == (s1.meta().level, s1.meta().degree)
    bad = [a.copy() for a in arrays]
    bad[2][1, 0, 5] = np.uint64(q[0])
    with pytest.raises(H.HcError):
        H.hc_ct_import_batch(pair.ctx, bad, metas)


def test_host_pipeline_matches_device_batch(pair):
    """The host-to-host pipelined call gives, word for word, the exported
    results of the device-resident batch call, for a ragged last chunk and
    for the automatic chunking (12 pairs: six chunks of 2); an
    out-of-range input residue and a negative chunk are rejected."""
    op = pair.op
    lv, n = 3, 12
    ga = [pair.encrypt_values(W.slot_values(60 + i, op.K), level=lv, nonce=600 + i)[0] for i in range(n)]
    gb = [pair.encrypt_values(W.slot_values(70 + i, op.K), level=lv, nonce=700 + i)[0] for i in range(n)]
    want = [H.hc_ct_export(pair.ctx, c)[0] for c in H.hc_mul_relin_rescale_batch(pair.ctx, pair.g_evk, ga, gb)]
    a_arr = [H.hc_ct_export(pair.ctx, c)[0] for c in ga]
    b_arr = [H.hc_ct_export(pair.ctx, c)[0] for c in gb]
    a_m = [(lv, 1, c.meta().scale) for c in ga]
    b_m = [(lv, 1, c.meta().scale) for c in gb]
    default_streams = H.hc_tune_get(pair.ctx, H.HC_TUNE_HOST_STREAMS)
    assert default_streams == 2
    try:
        for streams in (1, 2, 3, 4):  # chunks' kernels round-robin over this many streams
            H.hc_tune_set(pair.ctx, H.HC_TUNE_HOST_STREAMS, streams)
            for chunk in (2, 0, 7):
                outs = [np.zeros((2, lv, op.N), dtype=np.uint64) for _ in range(n)]
                metas = H.hc_mul_relin_rescale_host(pair.ctx, pair.g_evk, a_arr, a_m, b_arr, b_m, outs, chunk=chunk)
                for o, w, m in zip(outs, want, metas):
                    np.testing.assert_array_equal(o, w)
                    assert (m.level, m.degree) == (lv - 1, 1)
                tl = H.hc_profile_host_timeline(pair.ctx)
                assert len(tl) == (6 if chunk == 0 else -(-n // chunk))
                assert all(c[0] <= c[1] <= c[2] <= c[3] <= c[4] <= c[5] for c in tl)
        with pytest.raises(H.HcError):
            H.hc_tune_set(pair.ctx, H.HC_TUNE_HOST_STREAMS, 5)
    finally:
        H.hc_tune_set(pair.ctx, H.HC_TUNE_HOST_STREAMS, default_streams)
    bad = [a.copy() for a in a_arr]
    bad[4][0, 1, 3] = np.uint64(op.q[1])
    outs = [np.zeros((2, lv, op.N), dtype=np.uint64) for _ in range(n)]
    with pytest.raises(H.HcError):
        H.hc_mul_relin_rescale_host(pair.ctx, pair.g_evk, bad, a_m, b_arr, b_m, outs, chunk=2)
    with pytest.raises(H.HcError):
        H.hc_mul_relin_rescale_host(pair.ctx, pair.g_evk, a_arr, a_m, b_arr, b_m, outs, chunk=-1)


def test_evaluation_form_host_call_and_export(pair):
    """Evaluation-form export/import round-trips the device words; the
    evaluation-form host-to-host call equals the device batch exported in
    that form, and its outputs, imported back and exported in coefficient
    form, equal the coefficient-form host call's words (which the oracle
    pins elsewhere), for chunk sizes 2, automatic and a ragged 5, also with
    three asynchronous calls in flight; an out-of-range residue is rejected
    by the import, by the call and by an asynchronous call's wait."""
    op = pair.op
    lv, n = 3, 12
    ga = [pair.encrypt_values(W.slot_values(160 + i, op.K), level=lv, nonce=1600 + i)[0] for i in range(n)]
    gb = [pair.encrypt_values(W.slot_values(170 + i, op.K), level=lv, nonce=1700 + i)[0] for i in range(n)]
    ea = [H.hc_ct_export_eval(pair.ctx, c)[0] for c in ga]
    eb = [H.hc_ct_export_eval(pair.ctx, c)[0] for c in gb]
    back = H.hc_ct_import_eval(pair.ctx, ea[0], lv, 1, ga[0].meta().scale)
    np.testing.assert_array_equal(H.hc_ct_export(pair.ctx, back)[0], H.hc_ct_export(pair.ctx, ga[0])[0])
    np.testing.assert_array_equal(H.hc_ct_export_eval(pair.ctx, back)[0], ea[0])
    want = [H.hc_ct_export_eval(pair.ctx, c)[0] for c in H.hc_mul_relin_rescale_batch(pair.ctx, pair.g_evk, ga, gb)]
    coeff, _ = _host_products(pair, ga, gb, lv)
    a_m = [(lv, 1, c.meta().scale) for c in ga]
    b_m = [(lv, 1, c.meta().scale) for c in gb]
    for chunk in (2, 0, 5):
        outs = [np.zeros((2, lv, op.N), dtype=np.uint64) for _ in range(n)]
        metas = H.hc_mul_relin_rescale_host(pair.ctx, pair.g_evk, ea, a_m, eb, b_m, outs, chunk=chunk, eval_form=True)
        for o, w, c, m in zip(outs, want, coeff, metas):
            np.testing.assert_array_equal(o, w)
            assert (m.level, m.degree) == (lv - 1, 1)
            ct = H.hc_ct_import_eval(pair.ctx, o, m.level, m.degree, m.scale)
            np.testing.assert_array_equal(H.hc_ct_export(pair.ctx, ct)[0], c)
    # three calls in flight at once (each with its own outputs), waited for in turn
    sets = [[np.zeros((2, lv, op.N), dtype=np.uint64) for _ in range(n)] for _ in range(3)]
    ops = [H.hc_mul_relin_rescale_host_async(pair.ctx, pair.g_evk, ea, a_m, eb, b_m, outs, chunk=chunk)
           for outs, chunk in zip(sets, (2, 0, 5))]
    for hop, outs in zip(ops, sets):
        metas = hop.wait()
        assert len(H.hc_profile_host_timeline(pair.ctx)) >= 1
        for o, w, m in zip(outs, want, metas):
            np.testing.assert_array_equal(o, w)
            assert (m.level, m.degree) == (lv - 1, 1)
    bad = ea[4].copy()
    bad[1, 2, 7] = np.uint64(op.q[2])
    with pytest.raises(H.HcError):
        H.hc_ct_import_eval(pair.ctx, bad, lv, 1, 1.0)
    hop = H.hc_mul_relin_rescale_host_async(pair.ctx, pair.g_evk, ea[:4] + [bad] + ea[5:], a_m, eb, b_m, sets[0],
                                            chunk=2)
    with pytest.raises(H.HcError):
        hop.wait()
    outs = [np.zeros((2, lv, op.N), dtype=np.uint64) for _ in range(n)]
    with pytest.raises(H.HcError):
        H.hc_mul_relin_rescale_host(pair.ctx, pair.g_evk, ea[:4] + [bad] + ea[5:], a_m, eb, b_m, outs, chunk=2,
                                    eval_form=True)


def _host_products(p, ga, gb, lv):
    """The host-to-host call on exported inputs: coefficient-form outputs."""
    a_arr = [H.hc_ct_export(p.ctx, c)[0] for c in ga]
    b_arr = [H.hc_ct_export(p.ctx, c)[0] for c in gb]
    a_m = [(lv, 1, c.meta().scale) for c in ga]
    b_m = [(lv, 1, c.meta().scale) for c in gb]
    outs = [np.zeros((2, lv, p.op.N), dtype=np.uint64) for _ in ga]
    metas = H.hc_mul_relin_rescale_host(p.ctx, p.g_evk, a_arr, a_m, b_arr, b_m, outs)
    return outs, metas


def _assert_host_same(out, meta, octx, what):
    assert (meta.level, meta.degree, meta.scale) == (octx.level, octx.degree, octx.scale), what
    if not np.array_equal(out, octx.c):
        bad = np.argwhere(out != octx.c)
        raise AssertionError("%s: %d of %d words differ, first at %s" % (what, len(bad), out.size, bad[:3].tolist()))


def test_batch_mul_relin_rescale_every_level_and_edges(pair):
    """The fused batch at every level down to 1 (truncated last digit at low
    levels, a one-limb fused tail at level 1) equals the oracle, in NTT form
    (device batch) and in coefficient form (host call, whose tail is carried
    by the inverse transform); an empty batch, an aliased pair (a is b) and
    level 0 behave."""
    op = pair.op
    for lv in range(op.L, 0, -1):
        ga, oa = pair.encrypt_values(W.slot_values(80 + lv, op.K), level=lv, nonce=800 + lv)
        gb, ob = pair.encrypt_values(W.slot_values(90 + lv, op.K), level=lv, nonce=900 + lv)
        r = H.hc_mul_relin_rescale_batch(pair.ctx, pair.g_evk, [ga, ga], [gb, ga])
        want_ab = ckks.rescale(op, ckks.relin(op, pair.o_evk, ckks.mul(op, oa, ob)))
        want_aa = ckks.rescale(op, ckks.relin(op, pair.o_evk, ckks.mul(op, oa, oa)))
        pair.assert_same(r[0], want_ab, "l=%d" % lv)
        pair.assert_same(r[1], want_aa, "a*a l=%d" % lv)
        outs, metas = _host_products(pair, [ga, ga], [gb, ga], lv)
        _assert_host_same(outs[0], metas[0], want_ab, "host l=%d" % lv)
        _assert_host_same(outs[1], metas[1], want_aa, "host a*a l=%d" % lv)
    assert H.hc_mul_relin_rescale_batch(pair.ctx, pair.g_evk, [], []) == []
    assert H.hc_ct_import_batch(pair.ctx, [], []) == []
    H.hc_ct_export_batch(pair.ctx, [], [])
    assert H.hc_mul_relin_rescale_host(pair.ctx, pair.g_evk, [], [], [], [], []) == []
    g0, _ = pair.encrypt_values(W.slot_values(99, op.K), level=0, nonce=999)
    with pytest.raises(H.HcError) as e:
        H.hc_mul_relin_rescale_batch(pair.ctx, pair.g_evk, [g0], [g0])
    assert e.value.code == -5  # HC_ERR_DEPTH


def test_autotune_and_every_tuning_choice_bit_identical(pair):
    """hc_autotune picks a value for every knob; every candidate value of every
    knob gives the same words (tiles and launch shapes only)."""
    op = pair.op
    ga, _ = pair.encrypt_values(W.slot_values(41, op.K), nonce=4100)
    gb, _ = pair.encrypt_values(W.slot_values(42, op.K), nonce=4200)
    report = H.hc_autotune(pair.ctx, pair.g_evk, 4)
    lines = dict(l.split(" ", 1) for l in report.strip().splitlines())
    assert set(lines) == {"ntt_variant", "key_product_z", "modup_split"}
    assert int(lines["ntt_variant"].split()[0]) == H.hc_tune_get(pair.ctx, H.HC_TUNE_NTT)
    want = None
    for ntt in (0, 1):
        for kz in (1, 4):
            for sp in (1, 3):
                H.hc_tune_set(pair.ctx, H.HC_TUNE_NTT, ntt)
                H.hc_tune_set(pair.ctx, H.HC_TUNE_KEY_PRODUCT_Z, kz)
                H.hc_tune_set(pair.ctx, H.HC_TUNE_MODUP_SPLIT, sp)
                r = H.hc_mul_relin_rescale_batch(pair.ctx, pair.g_evk, [ga, gb], [gb, gb])
                got = [H.hc_ct_export(pair.ctx, c)[0] for c in r]
                rot = H.hc_rotate_hoisted(pair.ctx, pair.g_evk, ga, [1, 3])
                got += [H.hc_ct_export(pair.ctx, c)[0] for c in rot]
                if want is None:
                    want = got
                for x, y in zip(got, want):
                    np.testing.assert_array_equal(x, y)
    for knob, bad in ((H.HC_TUNE_NTT, 2), (H.HC_TUNE_KEY_PRODUCT_Z, 0), (H.HC_TUNE_MODUP_SPLIT, 65), (7, 1)):  # N = 2^10: no variant 2
        with pytest.raises(H.HcError):
            H.hc_tune_set(pair.ctx, knob, bad)
    H.hc_tune_set(pair.ctx, H.HC_TUNE_NTT, 1)
    H.hc_tune_set(pair.ctx, H.HC_TUNE_KEY_PRODUCT_Z, 1)
    H.hc_tune_set(pair.ctx, H.HC_TUNE_MODUP_SPLIT, 1)


@pytest.mark.parametrize("log_n", [13, 14, 15, 16])
def test_ntt_tile_variants_match_oracle(log_n):
    """Every NTT form the tuner can pick at N = 2^13..2^16 (two-pass block
    sizes including the 64-thread tiles that exist only there, the
    single-pass transforms on one CTA (2^13, 2^14) or a cluster of two or
    four (2^15, 2^16), and the pipelined two-pass form) gives the oracle's words for a multiply + relinearise
    + rescale, a rotation and the host-to-host call."""
    from hc_pair import Pair
    p = Pair(log_n, [50, 30, 30], [50], 30, seed=70 + log_n, rot_steps=[5])
    op = p.op
    ga, oa = p.encrypt_values(W.slot_values(71, op.K), nonce=1)
    gb, ob = p.encrypt_values(W.slot_values(72, op.K), nonce=2)
    want_m = ckks.rescale(op, ckks.relin(op, p.o_evk, ckks.mul(op, oa, ob)))
    want_r = ckks.rotate(op, p.o_evk, oa, 5)
    for v in (0, 1, 2, 3, 4, 5):
        H.hc_tune_set(p.ctx, H.HC_TUNE_NTT, v)
        p.assert_same(H.hc_mul_relin_rescale_batch(p.ctx, p.g_evk, [ga], [gb])[0], want_m, "mul v=%d" % v)
        p.assert_same(H.hc_rotate(p.ctx, p.g_evk, ga, 5), want_r, "rot v=%d" % v)
        outs, metas = _host_products(p, [ga], [gb], op.L)
        _assert_host_same(outs[0], metas[0], want_m, "host v=%d" % v)
    with pytest.raises(H.HcError):
        H.hc_tune_set(p.ctx, H.HC_TUNE_NTT, 6)


def test_batch_larger_than_workspace_chunk(pair):
    """300 pairs at N = 2^10: the key switch works in chunks of at most 256
    items, so the batch runs as 256 + a ragged 44.  Items on both sides of the
    chunk boundary match the oracle; all 300 match the unfused three-call
    form (relinearise, then rescale)."""
    op = pair.op
    lv = 2
    A = [pair.encrypt_values(W.slot_values(1000 + i, op.K), level=lv, nonce=10000 + i) for i in range(300)]
    B = [pair.encrypt_values(W.slot_values(2000 + i, op.K), level=lv, nonce=20000 + i) for i in range(300)]
    r = H.hc_mul_relin_rescale_batch(pair.ctx, pair.g_evk, [g for g, _ in A], [g for g, _ in B])
    for i in (0, 255, 256, 299):
        (_, oa), (_, ob) = A[i], B[i]
        pair.assert_same(r[i], ckks.rescale(op, ckks.relin(op, pair.o_evk, ckks.mul(op, oa, ob))), "item %d" % i)
    for i in range(300):
        g = H.hc_rescale(pair.ctx, H.hc_relin(pair.ctx, pair.g_evk, H.hc_mul(pair.ctx, A[i][0], B[i][0])))
        np.testing.assert_array_equal(H.hc_ct_export(pair.ctx, r[i])[0], H.hc_ct_export(pair.ctx, g)[0])


def test_import_rejects_out_of_range(pair):
    data = np.zeros((2, 1, pair.op.N), dtype=np.uint64)
    data[1, 0, 7] = pair.op.q[0]
    with pytest.raises(H.HcError) as e:
        H.hc_ct_import(pair.ctx, data, 0, 1, 1.0)
    assert e.value.code == -1


def test_mul_relin_rescale_bit_exact(pair):
    op = pair.op
    za, zb = W.slot_values(1, op.K), W.slot_values(2, op.K)
    for lv in (op.L, 3, 2, 1):
        ga, oa = pair.encrypt(pair.encode_int(za), level=lv, nonce=10 + lv)
        gb, ob = pair.encrypt(pair.encode_int(zb), level=lv, nonce=20 + lv)
        gd = H.hc_mul(pair.ctx, ga, gb)
        od = ckks.mul(op, oa, ob)
        pair.assert_same(gd, od, "tensor l=%d" % lv)
        gr = H.hc_relin(pair.ctx, pair.g_evk, gd)
        orl = ckks.relin(op, pair.o_evk, od)
        pair.assert_same(gr, orl, "relin l=%d" % lv)
        gs = H.hc_rescale(pair.ctx, gr)
        os_ = ckks.rescale(op, orl)
        pair.assert_same(gs, os_, "rescale l=%d" % lv)
        got = pair.decrypt_gpu(gs)
        assert np.max(np.abs(got - za * zb)) < 2.0 ** -15


def test_mul_relin_rescale_61bit_primes():
    """61-bit primes leave the 30-bit-halves basis conversions and key
    product for their 128-bit carry-chained form: both stay bit-exact."""
    from hc_pair import Pair
    p = Pair(10, [61, 61, 61, 61], [61, 61], 40, seed=13)
    op = p.op
    za, zb = W.slot_values(11, op.K), W.slot_values(12, op.K)
    ga, oa = p.encrypt(p.encode_int(za), nonce=1)
    gb, ob = p.encrypt(p.encode_int(zb), nonce=2)
    gs = H.hc_mul_relin_rescale_batch(p.ctx, p.g_evk, [ga], [gb])[0]
    os_ = ckks.rescale(op, ckks.relin(op, p.o_evk, ckks.mul(op, oa, ob)))
    p.assert_same(gs, os_, "61-bit mul+relin+rescale")
    gr = H.hc_relin(p.ctx, p.g_evk, H.hc_mul(p.ctx, ga, gb))
    p.assert_same(gr, ckks.relin(op, p.o_evk, ckks.mul(op, oa, ob)), "61-bit relin")


def test_mul_relin_rescale_base_prime_below_half_the_last():
    """A chain whose q_0 (30 bits) is below half of the rescaled prime (45
    bits): the centred last limb then needs reducing modulo q_0 in the fused
    tail (every other chain here skips that reduction).  Device batch and
    host call both give the oracle's words."""
    from hc_pair import Pair
    p = Pair(10, [30, 45, 45], [50], 25, seed=15)
    op = p.op
    za, zb = W.slot_values(13, op.K), W.slot_values(14, op.K)
    ga, oa = p.encrypt(p.encode_int(za), nonce=1)
    gb, ob = p.encrypt(p.encode_int(zb), nonce=2)
    want = ckks.rescale(op, ckks.relin(op, p.o_evk, ckks.mul(op, oa, ob)))
    p.assert_same(H.hc_mul_relin_rescale_batch(p.ctx, p.g_evk, [ga], [gb])[0], want, "small q_0")
    outs, metas = _host_products(p, [ga], [gb], op.L)
    _assert_host_same(outs[0], metas[0], want, "host small q_0")


def test_rescale_degree2_and_level_errors(pair):
    op = pair.op
    ga, oa = pair.encrypt_values(W.slot_values(3, op.K), level=2, nonce=40)
    gd, od = H.hc_mul(pair.ctx, ga, ga), ckks.mul(op, oa, oa)
    pair.assert_same(H.hc_rescale(pair.ctx, gd), ckks.rescale(op, od), "rescale degree 2")
    g0, _ = pair.encrypt_values(W.slot_values(3, op.K), level=0, nonce=41)
    with pytest.raises(H.HcError) as e:
        H.hc_rescale(pair.ctx, g0)
    assert e.value.code == -5
    with pytest.raises(H.HcError) as e:
        H.hc_add(pair.ctx, ga, g0)
    assert e.value.code == -2


def test_missing_key_and_scale_mismatch_are_error_codes(pair):
    """A rotation without its Galois key gives HC_ERR_NO_KEY and an addition
    of operands whose scales differ gives HC_ERR_SCALE_MISMATCH, both before
    any device work; the context keeps working."""
    op = pair.op
    ga, oa = pair.encrypt_values(W.slot_values(5, op.K), level=2, nonce=50)
    with pytest.raises(H.HcError) as e:
        H.hc_rotate(pair.ctx, pair.g_evk, ga, 2)  # keys exist for 1, 3, -1, 5, 17 only
    assert e.value.code == -4
    sq = H.hc_rescale(pair.ctx, H.hc_relin(pair.ctx, pair.g_evk, H.hc_mul(pair.ctx, ga, ga)))  # level 1, scale s^2 / q_2
    g1 = H.hc_drop_to_level(pair.ctx, ga, 1)  # level 1, scale s
    with pytest.raises(H.HcError) as e:
        H.hc_add(pair.ctx, sq, g1)
    assert e.value.code == -3
    pair.assert_same(H.hc_rotate(pair.ctx, pair.g_evk, ga, 1), ckks.rotate(op, pair.o_evk, oa, 1), "after errors")


def test_rotations_bit_exact(pair):
    op = pair.op
    z = W.slot_values(4, op.K)
    g, o = pair.encrypt_values(z, level=3, nonce=50)
    for r in (1, 3, -1, 5, 0, op.K):
        pair.assert_same(H.hc_rotate(pair.ctx, pair.g_evk, g, r), ckks.rotate(op, pair.o_evk, o, r), "rot %d" % r)
    steps = [1, 5, 17, 0]
    gh = H.hc_rotate_hoisted(pair.ctx, pair.g_evk, g, steps)
    oh = ckks.rotate_hoisted(op, pair.o_evk, o, steps)
    for r, a, b in zip(steps, gh, oh):
        pair.assert_same(a, b, "hoisted %d" % r)
        assert np.max(np.abs(pair.decrypt_gpu(a) - np.roll(z, -r))) < 2.0 ** -15
    with pytest.raises(H.HcError) as e:
        H.hc_rotate(pair.ctx, pair.g_evk, g, 2)
    assert e.value.code == -4


def test_add_sub_constants(pair):
    op = pair.op
    ga, oa = pair.encrypt_values(W.slot_values(6, op.K), level=4, nonce=60)
    gb, ob = pair.encrypt_values(W.slot_values(7, op.K), level=4, nonce=61)
    pair.assert_same(H.hc_add(pair.ctx, ga, gb), ckks.add(op, oa, ob), "add")
    pair.assert_same(H.hc_sub(pair.ctx, ga, gb), ckks.sub(op, oa, ob), "sub")
    pair.assert_same(H.hc_add_const(pair.ctx, ga, -0.47), ckks.add_const(op, oa, -0.47), "add_const")
    cs = float(op.q[4])
    pair.assert_same(H.hc_mul_const(pair.ctx, ga, 0.25, cs), ckks.mul_const(op, oa, 0.25, cs), "mul_const")
    pair.assert_same(H.hc_drop_to_level(pair.ctx, ga, 1), ckks.drop_to_level(op, oa, 1), "drop")
    gm = H.hc_mul_const(pair.ctx, ga, 0.5, 2.0 ** 20)
    with pytest.raises(H.HcError) as e:
        H.hc_add(pair.ctx, ga, gm)
    assert e.value.code == -3


def test_decrypt_matches_oracle(pair):
    op = pair.op
    z = W.slot_values(8, op.K)
    g, o = pair.encrypt_values(z, level=2, nonce=70)
    gpt = H.hc_decrypt(pair.ctx, pair.g_sk, g)
    assert np.array_equal(H.hc_pt_export(pair.ctx, gpt), ckks.decrypt(op, pair.o_sk, o).m)
    got = H.hc_decode(pair.ctx, gpt)
    exp = pair.decrypt_oracle(o)
    assert np.max(np.abs(got - exp)) < 1e-9
    assert np.max(np.abs(got - z)) < 2.0 ** -20


def test_encode_within_one_of_oracle(pair12):
    op = pair12.op
    z = W.slot_values(9, op.K) + 1j * W.slot_values(10, op.K)
    gpt = H.hc_encode(pair12.ctx, z, op.scale, 2)
    got = H.hc_pt_export(pair12.ctx, gpt)
    m = encoding.encode(z, op.N, op.scale)
    exp = ckks.reduce_signed(m, op.q[:3])
    # FP64 rounding may move a coefficient by one: |GPU - oracle| <= 1
    for l in range(3):
        q = op.q[l]
        d = (got[l].astype(object) - exp[l].astype(object)) % q
        assert all(x in (0, 1, q - 1) for x in d), l
    back = H.hc_decode(pair12.ctx, gpt)
    assert np.max(np.abs(back - z)) < 2.0 ** -18


def test_batch_mul_relin_rescale(pair12):
    op = pair12.op
    gs, os_ = [], []
    for i in range(5):
        ga, oa = pair12.encrypt_values(W.slot_values(200 + i, op.K), nonce=100 + i)
        gb, ob = pair12.encrypt_values(W.slot_values(300 + i, op.K), nonce=200 + i)
        gs.append((ga, gb))
        os_.append((oa, ob))
    outs = H.hc_mul_relin_rescale_batch(pair12.ctx, pair12.g_evk, [a for a, _ in gs], [b for _, b in gs])
    for i, (oa, ob) in enumerate(os_):
        exp = ckks.rescale(op, ckks.relin(op, pair12.o_evk, ckks.mul(op, oa, ob)))
        pair12.assert_same(outs[i], exp, "batch %d" % i)
    assert H.hc_mul_relin_rescale_batch(pair12.ctx, pair12.g_evk, [], []) == []
