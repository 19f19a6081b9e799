"""Full-size checks in the benchmark's launch configurations.

The oracle cannot run whole full-size workloads in seconds, so these compare
sampled outputs bit for bit (the oracle recomputes just the sampled output
from the same inputs) and check properties that hold at any size (decrypted
results against plain arithmetic / the FP64 network) everywhere."""
import numpy as np
import pytest

from oracle import ckks, cnn
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 2.0 ** -15


def test_deep_n16_batch_sampled_bit_exact():
    """hc_mul_relin_rescale_batch at N = 2^16, L = 20, dnum = 3, batch 64 (the
    benchmark's step, eager and captured into a CUDA graph as the benchmark
    times it, and through the host-to-host pipelined call); pairs 5 and 63
    are recomputed by the oracle, every other pair is checked equal across
    the three forms."""
    import torch
    from hc_pair import Pair
    ps = W.DEEP_N16
    stream = torch.cuda.Stream()  # a stream of its own: capturable
    p = Pair(ps.log_n, ps.q_bits, ps.p_bits, ps.log2_scale, seed=W.MASTER_SEED + 4, stream=stream.cuda_stream)
    B, ks = 64, (5, 63)
    A, Bc, oracle_in = [], [], {}
    for i in range(B):
        ma, mb = W.int_plaintext(10 + i, p.op.N, 2 ** 50), W.int_plaintext(100 + i, p.op.N, 2 ** 50)
        if i in ks:
            ga, oa = p.encrypt(ma, nonce=2 * i)
            gb, ob = p.encrypt(mb, nonce=2 * i + 1)
            oracle_in[i] = (oa, ob)
        else:
            ga = H.hc_encrypt(p.ctx, p.g_pk, H.hc_pt_from_coeffs(p.ctx, ma, p.op.L, p.op.scale), p.seed + 1, 2 * i)
            gb = H.hc_encrypt(p.ctx, p.g_pk, H.hc_pt_from_coeffs(p.ctx, mb, p.op.L, p.op.scale), p.seed + 1, 2 * i + 1)
        A.append(ga)
        Bc.append(gb)
    outs = H.hc_mul_relin_rescale_batch(p.ctx, p.g_evk, A, Bc)
    for k in ks:
        oa, ob = oracle_in[k]
        exp = ckks.rescale(p.op, ckks.relin(p.op, p.o_evk, ckks.mul(p.op, oa, ob)))
        p.assert_same(outs[k], exp, "batch item %d" % k)
    eager = [H.hc_ct_export(p.ctx, c)[0] for c in outs]
    # the captured step, replayed twice
    H.hc_graph_begin([p.ctx], int(4 + 0.2 * B + 1) << 30)
    g_outs = H.hc_mul_relin_rescale_batch(p.ctx, p.g_evk, A, Bc)
    graph = H.hc_graph_end([p.ctx])
    H.hc_graph_launch(graph)
    H.hc_graph_launch(graph)
    for i in range(B):
        np.testing.assert_array_equal(H.hc_ct_export(p.ctx, g_outs[i])[0], eager[i])
    del g_outs
    del graph
    # host buffers in, host buffers out
    a_arr = [H.hc_ct_export(p.ctx, c)[0] for c in A]
    b_arr = [H.hc_ct_export(p.ctx, c)[0] for c in Bc]
    metas = [(p.op.L, 1, c.meta().scale) for c in A]
    host = [np.zeros((2, p.op.L, p.op.N), dtype=np.uint64) for _ in range(B)]
    H.hc_mul_relin_rescale_host(p.ctx, p.g_evk, a_arr, metas, b_arr, metas, host)
    for i in range(B):
        np.testing.assert_array_equal(host[i], eager[i])
    # the evaluation-form host call: the device batch's words, exported in that form
    ea = [H.hc_ct_export_eval(p.ctx, c)[0] for c in A]
    eb = [H.hc_ct_export_eval(p.ctx, c)[0] for c in Bc]
    host_e = [np.zeros((2, p.op.L, p.op.N), dtype=np.uint64) for _ in range(B)]
    H.hc_mul_relin_rescale_host(p.ctx, p.g_evk, ea, metas, eb, metas, host_e, eval_form=True)
    for i in ks:
        ct = H.hc_ct_import_eval(p.ctx, host_e[i], p.op.L - 1, 1, 1.0)
        np.testing.assert_array_equal(H.hc_ct_export(p.ctx, ct)[0], eager[i])
    del ea, eb, host_e
    # the other NTT tile shapes at N = 2^16 (autotuning choices) give the same words
    default = H.hc_tune_get(p.ctx, H.HC_TUNE_NTT)
    for v in (0, 1, 2, 3, 4, 5):
        H.hc_tune_set(p.ctx, H.HC_TUNE_NTT, v)
        r = H.hc_mul_relin_rescale_batch(p.ctx, p.g_evk, [A[k] for k in ks], [Bc[k] for k in ks])
        for k, c in zip(ks, r):
            np.testing.assert_array_equal(H.hc_ct_export(p.ctx, c)[0], eager[k])
        hk = [np.zeros((2, p.op.L, p.op.N), dtype=np.uint64) for _ in ks]
        H.hc_mul_relin_rescale_host(p.ctx, p.g_evk, [a_arr[k] for k in ks], [metas[k] for k in ks],
                                    [b_arr[k] for k in ks], [metas[k] for k in ks], hk)
        for k, h in zip(ks, hk):
            np.testing.assert_array_equal(h, eager[k])
    H.hc_tune_set(p.ctx, H.HC_TUNE_NTT, default)
    # property at full size: slot products of encoded vectors
    za, zb = W.slot_values(1, p.op.K), W.slot_values(2, p.op.K)
    ca = H.hc_encrypt(p.ctx, p.g_pk, H.hc_encode(p.ctx, za, p.op.scale, p.op.L), 3, 0)
    cb = H.hc_encrypt(p.ctx, p.g_pk, H.hc_encode(p.ctx, zb, p.op.scale, p.op.L), 3, 1)
    r = H.hc_mul_relin_rescale_batch(p.ctx, p.g_evk, [ca] * 3, [cb] * 3)
    for c in r:
        assert np.max(np.abs(p.decrypt_gpu(c) - za * zb)) < TOL


@pytest.fixture(scope="module")
def batch14():
    from hc_pair import Pair
    ps = W.BATCH_N14
    return Pair(ps.log_n, ps.q_bits, ps.p_bits, ps.log2_scale, seed=W.MASTER_SEED + 2)


def test_batch_cnn_n14_logits_within_tolerance(batch14):
    """The whole batch-packed CNN on 8192 synthetic 28x28 images: conv 5x5
    stride 2, 5 channels -> x^2 -> mean pool -> FC 180 -> 10; every image's
    decrypted logits within 2^-15 of the FP64 network."""
    p = batch14
    c = W.CNN_BATCH
    ctx, evk, K = p.ctx, p.g_evk, p.op.K
    imgs = W.images(W.MASTER_SEED + 20, K, c["H"], c["W"])
    cw = W.conv_weights(W.MASTER_SEED + 21, c["cout"], c["k"], c["k"])
    Ho = (c["H"] - c["k"]) // c["stride"] + 1
    n_in = (Ho // 2) ** 2 * c["cout"]
    fw = W.fc_weights(W.MASTER_SEED + 22, c["n_out"], n_in)

    def enc(vals, nonce):
        return H.hc_encrypt(ctx, p.g_pk, H.hc_encode(ctx, vals, p.op.scale, p.op.L), 77, nonce)

    xs = [enc(imgs[:, h, w], h * c["W"] + w) for h in range(c["H"]) for w in range(c["W"])]
    ws = [enc(np.full(K, cw[co, a, b, 0]), 1000 + (co * c["k"] + a) * c["k"] + b)
          for co in range(c["cout"]) for a in range(c["k"]) for b in range(c["k"])]
    fws = [enc(np.full(K, fw[r, i]), 2000 + r * n_in + i) for r in range(c["n_out"]) for i in range(n_in)]
    y = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, xs, c["H"], c["W"], 1, ws, c["cout"], c["k"], c["k"], c["stride"])
    a = H.hc_enc_poly_act(ctx, evk, y, c["act"])
    pl = H.hc_enc_pool(ctx, evk, H.HC_PACK_BATCH, a, c["cout"], Ho, Ho)
    z = H.hc_enc_fc(ctx, evk, H.HC_PACK_BATCH, pl, fws, c["n_out"])
    assert [t.level for t in z] == [2] * c["n_out"]
    logits = np.stack([p.decrypt_gpu(t).real for t in z], axis=1)
    ref = cnn.network(imgs[..., None], cw, c["stride"], c["act"], fw)
    assert np.max(np.abs(logits - ref)) < TOL
    assert np.array_equal(np.argmax(logits, 1), np.argmax(ref, 1))


def test_batch_cnn_n14_sampled_conv_pool_bit_exact(batch14):
    """Full conv (784 inputs, 125 weights) and pool layers on the GPU; the
    oracle recomputes conv output (m, n, c) = (3, 7, 2) and pool output
    (i, j, c) = (1, 4, 4) from the same ciphertexts."""
    p = batch14
    c = W.CNN_BATCH
    ctx, evk = p.ctx, p.g_evk
    Hh, Ww, k, s, cout = c["H"], c["W"], c["k"], c["stride"], c["cout"]
    Ho = (Hh - k) // s + 1

    def needed_inputs():
        rows = set(range(3 * s, 3 * s + k)) | set(range(2 * s, 2 * s + k + s))
        cols = set(range(7 * s, 7 * s + k)) | set(range(8 * s, 8 * s + k + s))
        return rows, cols

    rows, cols = needed_inputs()
    gx, ox = [], {}
    for h in range(Hh):
        for w in range(Ww):
            m = W.int_plaintext(5000 + h * Ww + w, p.op.N, 2 ** 40)
            if h in rows and w in cols:
                g, o = p.encrypt(m, nonce=h * Ww + w)
                ox[(h, w)] = o
            else:
                g = H.hc_encrypt(ctx, p.g_pk, H.hc_pt_from_coeffs(ctx, m, p.op.L, p.op.scale), p.seed + 1, h * Ww + w)
            gx.append(g)
    gw, ow = [], []
    cw = W.conv_weights(W.MASTER_SEED + 21, cout, k, k)
    for co in range(cout):
        for a in range(k):
            for b in range(k):
                m = np.zeros(p.op.N, dtype=np.int64)
                m[0] = ckks.llround(cw[co, a, b, 0] * p.op.scale)  # slot constant
                g, o = p.encrypt(m, nonce=1000 + (co * k + a) * k + b)
                gw.append(g)
                ow.append(o)
    gy = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, gx, Hh, Ww, 1, gw, cout, k, k, s)

    def oracle_conv(mm, nn, co):
        xs = [ox[(mm * s + a, nn * s + b)] for a in range(k) for b in range(k)]
        wsel = [ow[(co * k + a) * k + b] for a in range(k) for b in range(k)]
        d = ckks.tensor_sum(p.op, xs, wsel)
        return ckks.rescale(p.op, ckks.relin(p.op, p.o_evk, d))

    p.assert_same(gy[(3 * Ho + 7) * cout + 2], oracle_conv(3, 7, 2), "conv (3,7,2)")
    ga = H.hc_enc_poly_act(ctx, evk, gy, c["act"])
    gp = H.hc_enc_pool(ctx, evk, H.HC_PACK_BATCH, ga, cout, Ho, Ho)
    i, j, ch = 1, 4, 4
    parts = [cnn.enc_square(p.op, p.o_evk, oracle_conv(2 * i + di, 2 * j + dj, ch)) for di, dj in
             ((0, 0), (1, 0), (0, 1), (1, 1))]
    s4 = ckks.add(p.op, ckks.add(p.op, parts[0], parts[1]), ckks.add(p.op, parts[2], parts[3]))
    s4 = ckks.mul_const(p.op, s4, 0.25, float(p.op.q[s4.level]))
    p.assert_same(gp[(i * (Ho // 2) + j) * cout + ch], ckks.rescale(p.op, s4), "pool (1,4,4)")


def test_batch_fc_n14_sampled_bit_exact(batch14):
    """FC 180 -> 10 at level 3 on fresh inputs; class 7 by the oracle."""
    p = batch14
    n_in, n_out, r = 180, 10, 7
    gx, ox = [], []
    for kk in range(n_in):
        g, o = p.encrypt(W.int_plaintext(7000 + kk, p.op.N, 2 ** 40), level=3, nonce=8000 + kk)
        gx.append(g)
        ox.append(o)
    gw, ow = [], []
    for rr in range(n_out):
        for kk in range(n_in):
            m = W.int_plaintext(9000 + rr * n_in + kk, p.op.N, 2 ** 40)
            if rr == r:
                g, o = p.encrypt(m, nonce=20000 + rr * n_in + kk)
                ow.append(o)
            else:
                g = H.hc_encrypt(p.ctx, p.g_pk, H.hc_pt_from_coeffs(p.ctx, m, p.op.L, p.op.scale), p.seed + 1,
                                 20000 + rr * n_in + kk)
            gw.append(g)
    gz = H.hc_enc_fc(p.ctx, p.g_evk, H.HC_PACK_BATCH, gx, gw, n_out)
    exp = cnn.enc_fc(p.op, p.o_evk, ox, ow, 1)[0]
    p.assert_same(gz[r], exp, "fc class 7")
