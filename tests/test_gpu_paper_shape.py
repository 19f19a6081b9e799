"""The paper's own network at N = 2^15 (Sec. "Dataset and Inference
Results", Table 1): 16384 images of 28x28 batch-packed, 28 filters of 3x3
(stride 1, no padding), the Eq. 4 activation g(u) = 0.47 + 0.50 u + 0.09 u^2,
2x2 mean pooling (Eq. 5-6) and a fully connected layer 4732 -> 10, run
filter by filter as the paper does (q_0 60 bits, six 40-bit primes, one
60-bit special prime, scale 2^40).

* every image's decrypted logits within 2^-15 of the FP64 network;
* one filter's conv, activation and pool outputs bit-exact against the
  oracle at a sampled position (the oracle recomputes just those outputs
  from the same ciphertexts);
* one class of the 4732 -> 10 FC bit-exact against the oracle on fresh
  inputs (the oracle's sum of 4732 tensor products runs in spawned worker
  processes; partial sums are added modulo each prime)."""
import numpy as np
import pytest

from oracle import ckks, cnn
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 2.0 ** -15


@pytest.fixture(scope="module")
def paper():
    from hc_pair import Pair
    ps = W.PAPER_N15
    return Pair(ps.log_n, ps.q_bits, ps.p_bits, ps.log2_scale, seed=W.MASTER_SEED + 6)


def _const(p, v, level, nonce):
    """A slot constant encrypted from the constant polynomial round(v scale)."""
    m = np.zeros(p.op.N, dtype=np.int64)
    m[0] = ckks.llround(v * p.op.scale)
    return H.hc_encrypt(p.ctx, p.g_pk, H.hc_pt_from_coeffs(p.ctx, m, level, p.op.scale), 5, nonce)


def test_paper_shape_logits_within_tolerance(paper):
    p = paper
    c = W.PAPER_CNN
    ctx, evk, K, L = p.ctx, p.g_evk, p.op.K, p.op.L
    imgs = W.images(W.MASTER_SEED + 30, K, 28, 28)
    cw = W.conv_weights(W.MASTER_SEED + 31, c["cout"], 3, 3)
    n_in = 13 * 13 * c["cout"]
    fw = W.fc_weights(W.MASTER_SEED + 32, c["n_out"], n_in) * 0.05
    xs = [H.hc_encrypt(ctx, p.g_pk, H.hc_encode(ctx, imgs[:, h, w], p.op.scale, L), 5, h * 28 + w)
          for h in range(28) for w in range(28)]
    pooled = [None] * n_in
    for f in range(c["cout"]):
        ws = [_const(p, cw[f, a, b, 0], L, 10000 + f * 9 + a * 3 + b) for a in range(3) for b in range(3)]
        y = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, xs, 28, 28, 1, ws, 1, 3, 3, 1)
        a = H.hc_enc_poly_act(ctx, evk, y, c["act"])
        del y
        pl = H.hc_enc_pool(ctx, evk, H.HC_PACK_BATCH, a, 1, 26, 26)
        del a
        for i in range(169):
            pooled[i * c["cout"] + f] = pl[i]
    del xs
    fws = [_const(p, fw[r, i], 2, 100000 + r * n_in + i) for r in range(c["n_out"]) for i in range(n_in)]
    z = H.hc_enc_fc(ctx, evk, H.HC_PACK_BATCH, pooled, fws, c["n_out"])
    del fws, pooled
    assert [t.level for t in z] == [1] * c["n_out"]
    logits = np.stack([p.decrypt_gpu(t).real for t in z], axis=1)
    ref = cnn.network(imgs[..., None], cw, 1, c["act"], fw)
    assert np.max(np.abs(logits - ref)) < TOL
    assert np.mean(np.argmax(logits, 1) == np.argmax(ref, 1)) > 0.999


def test_paper_shape_sampled_conv_act_pool_bit_exact(paper):
    """One filter over all 784 input ciphertexts; pool output (5, 8), the four
    conv and activation outputs under it, recomputed by the oracle."""
    p = paper
    c = W.PAPER_CNN
    ctx, evk, L = p.ctx, p.g_evk, p.op.L
    i, j = 5, 8
    rows, cols = range(2 * i, 2 * i + 4), range(2 * j, 2 * j + 4)
    gx, ox = [], {}
    for h in range(28):
        for w in range(28):
            m = W.int_plaintext(30000 + h * 28 + w, p.op.N, 2 ** 40)
            if h in rows and w in cols:
                g, o = p.encrypt(m, nonce=h * 28 + w)
                ox[(h, w)] = o
            else:
                g = H.hc_encrypt(ctx, p.g_pk, H.hc_pt_from_coeffs(ctx, m, L, p.op.scale), p.seed + 1, h * 28 + w)
            gx.append(g)
    cw = W.conv_weights(W.MASTER_SEED + 31, c["cout"], 3, 3)[3]
    gw, ow = [], []
    for a in range(3):
        for b in range(3):
            m = np.zeros(p.op.N, dtype=np.int64)
            m[0] = ckks.llround(cw[a, b, 0] * p.op.scale)
            g, o = p.encrypt(m, nonce=40000 + a * 3 + b)
            gw.append(g)
            ow.append(o)
    gy = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, gx, 28, 28, 1, gw, 1, 3, 3, 1)
    ga = H.hc_enc_poly_act(ctx, evk, gy, c["act"])
    gp = H.hc_enc_pool(ctx, evk, H.HC_PACK_BATCH, ga, 1, 26, 26)
    acts = []
    for di, dj in ((0, 0), (1, 0), (0, 1), (1, 1)):
        mm, nn = 2 * i + di, 2 * j + dj
        d = ckks.tensor_sum(p.op, [ox[(mm + a, nn + b)] for a in range(3) for b in range(3)], ow)
        y = ckks.rescale(p.op, ckks.relin(p.op, p.o_evk, d))
        p.assert_same(gy[mm * 26 + nn], y, "conv (%d,%d)" % (mm, nn))
        act = cnn.enc_poly_act(p.op, p.o_evk, y, c["act"])
        p.assert_same(ga[mm * 26 + nn], act, "activation (%d,%d)" % (mm, nn))
        acts.append(act)
    s4 = ckks.add(p.op, ckks.add(p.op, acts[0], acts[1]), ckks.add(p.op, acts[2], acts[3]))
    s4 = ckks.mul_const(p.op, s4, 0.25, float(p.op.q[s4.level]))
    p.assert_same(gp[i * 13 + j], ckks.rescale(p.op, s4), "pool (%d,%d)" % (i, j))


def test_paper_shape_fc_class_bit_exact(paper):
    """FC 4732 -> 10 at level 2 on fresh inputs; class 6 by the oracle."""
    from hc_pair import oracle_tensor_sum_parallel

    p = paper
    ctx, evk = p.ctx, p.g_evk
    n_in, n_out, r, level, eseed = 13 * 13 * 28, 10, 6, 2, p.seed + 1
    x_spec = [(50000 + k, 2 ** 40, level, eseed, 60000 + k) for k in range(n_in)]
    w_spec = [(70000 + k, 2 ** 40, level, eseed, 80000 + k) for k in range(n_in)]

    def gpu_ct(spec):
        mseed, bound, lv, es, nonce = spec
        m = W.int_plaintext(mseed, p.op.N, bound)
        return H.hc_encrypt(ctx, p.g_pk, H.hc_pt_from_coeffs(ctx, m, lv, p.op.scale), es, nonce)

    gx = [gpu_ct(s) for s in x_spec]
    gw = []
    for rr in range(n_out):
        for k in range(n_in):
            if rr == r:
                gw.append(gpu_ct(w_spec[k]))
            else:
                gw.append(gpu_ct((90000 + rr * n_in + k, 2 ** 40, level, eseed, 200000 + rr * n_in + k)))
    gz = H.hc_enc_fc(ctx, evk, H.HC_PACK_BATCH, gx, gw, n_out)
    del gw, gx
    d = oracle_tensor_sum_parallel(p.op, p.o_pk, list(zip(x_spec, w_spec)))
    want = ckks.rescale(p.op, ckks.relin(p.op, p.o_evk, d))
    p.assert_same(gz[r], want, "fc class %d" % r)
