"""GPU parity of the deep single-ciphertext CNN: conv 3x3 by hoisted
rotations, degree-7 Paterson-Stockmeyer activation, 2x2 mean pool by
rotations, FC by encrypted weight vectors and rotate-and-sum."""
import numpy as np
import pytest

from oracle import ckks, cnn, encoding
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 2.0 ** -15


def setup_net(p, C, n_out, seed):
    img = W.images(seed, 1, 28, 28)[0]
    cw = W.conv_weights(seed + 1, C, 3, 3)[:, :, :, 0]
    fw = W.fc_weights(seed + 2, n_out, 13 * 13 * C)
    return img, cw, fw


def test_deep_small_bit_exact_by_layer():
    from hc_pair import Pair
    p = Pair(11, [60] + [40] * 8, [60, 60], 40, seed=41, rot_steps=W.deep_rot_steps(28, 10))
    op = p.op
    C, n_out = 2, 3
    img, cw, fw = setup_net(p, C, n_out, 50)
    act = W.relu_cheb7()
    z = np.zeros(op.K)
    z[:784] = img.reshape(-1)
    gx, ox = p.encrypt_values(z, nonce=1)
    wc = [p.encrypt_values(np.full(op.K, cw[co, a, b]), nonce=10 + co * 9 + a * 3 + b)
          for co in range(C) for a in range(3) for b in range(3)]
    gy = H.hc_enc_conv2d(p.ctx, p.g_evk, H.HC_PACK_SINGLE_HOISTED, [gx], 28, 28, 1, [g for g, _ in wc], C, 3, 3, 1)
    oy = cnn.enc_conv2d_single_hoisted(op, p.o_evk, ox, 28, [o for _, o in wc], 3, 3, C)
    for i in range(C):
        p.assert_same(gy[i], oy[i], "conv %d" % i)
    ga = H.hc_enc_poly_act(p.ctx, p.g_evk, gy, list(act))
    oa = [cnn.enc_poly7(op, p.o_evk, t, act) for t in oy]
    for i in range(C):
        p.assert_same(ga[i], oa[i], "act %d" % i)
    gp = H.hc_enc_pool(p.ctx, p.g_evk, H.HC_PACK_SINGLE, ga, C, 26, 28)
    opl = [cnn.enc_pool_single(op, p.o_evk, t, 28) for t in oa]
    for i in range(C):
        p.assert_same(gp[i], opl[i], "pool %d" % i)
    V = W.deep_fc_vectors(fw, C, 13, 13, 28, op.K)
    vc = [p.encrypt_values(V[r, c], nonce=100 + r * C + c) for r in range(n_out) for c in range(C)]
    gz = H.hc_enc_fc_rotsum(p.ctx, p.g_evk, gp, [g for g, _ in vc], n_out, 10)
    oz = cnn.enc_fc_rotsum(op, p.o_evk, opl, [o for _, o in vc], n_out, 10)
    for r in range(n_out):
        p.assert_same(gz[r], oz[r], "fc %d" % r)
    got = np.array([p.decrypt_gpu(t)[0].real for t in gz])
    assert np.max(np.abs(got - cnn.deep_network(img, cw, act, fw))) < TOL


def test_deep_n16_logits_and_sampled_channel():
    from hc_pair import Pair
    ps, d = W.DEEP_N16, W.DEEP_CNN
    p = Pair(ps.log_n, ps.q_bits, ps.p_bits, ps.log2_scale, seed=W.MASTER_SEED + 4,
             rot_steps=W.deep_rot_steps(28, 10))
    op, ctx, evk = p.op, p.ctx, p.g_evk
    C, n_out = d["cout"], d["n_out"]
    img, cw, fw = setup_net(p, C, n_out, 60)
    act = W.relu_cheb7()
    # sampled channel 0: integer plaintexts both sides encrypt
    m = W.int_plaintext(61, op.N, 2 ** 45)
    gxi, oxi = p.encrypt(m, nonce=1)
    wints = []
    for co in range(C):
        for t in range(9):
            mm = np.zeros(op.N, dtype=np.int64)
            mm[0] = ckks.llround(cw[co, t // 3, t % 3] * op.scale)
            wints.append(mm)
    wc = [p.encrypt(mm, nonce=10 + i) for i, mm in enumerate(wints)]
    gy = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_SINGLE_HOISTED, [gxi], 28, 28, 1, [g for g, _ in wc], C, 3, 3, 1)
    oy0 = cnn.enc_conv2d_single_hoisted(op, p.o_evk, oxi, 28, [o for _, o in wc[:9]], 3, 3, 1)[0]
    p.assert_same(gy[0], oy0, "conv channel 0")
    ga = H.hc_enc_poly_act(ctx, evk, gy, list(act))
    p.assert_same(ga[0], cnn.enc_poly7(op, p.o_evk, oy0, act), "activation channel 0")
    # the whole network on the image: logits against FP64
    z = np.zeros(op.K)
    z[:784] = img.reshape(-1)
    x = H.hc_encrypt(ctx, p.g_pk, H.hc_encode(ctx, z, op.scale, op.L), 3, 0)
    y = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_SINGLE_HOISTED, [x], 28, 28, 1, [g for g, _ in wc], C, 3, 3, 1)
    a = H.hc_enc_poly_act(ctx, evk, y, list(act))
    pl = H.hc_enc_pool(ctx, evk, H.HC_PACK_SINGLE, a, C, 26, 28)
    V = W.deep_fc_vectors(fw, C, 13, 13, 28, op.K)
    vc = [H.hc_encrypt(ctx, p.g_pk, H.hc_encode(ctx, V[r, c], op.scale, op.L), 3, 100 + r * C + c)
          for r in range(n_out) for c in range(C)]
    out = H.hc_enc_fc_rotsum(ctx, evk, pl, vc, n_out, 10)
    assert out[0].level == op.L - 7
    got = np.array([p.decrypt_gpu(t)[0].real for t in out])
    ref = cnn.deep_network(img, cw, act, fw)
    assert np.max(np.abs(got - ref)) < TOL


def test_deep_small_batch_of_images_matches_one_by_one():
    """Three images through the deep network at once (the hoisted batched
    conv, one activation call and one pool call over every image's channels,
    the FC per image) give each image's single-image words."""
    from hc_pair import Pair
    p = Pair(11, [60] + [40] * 8, [60, 60], 40, seed=43, rot_steps=W.deep_rot_steps(28, 10))
    op = p.op
    C, n_out, B = 2, 3, 3
    _, cw, fw = setup_net(p, C, n_out, 80)
    act = list(W.relu_cheb7())
    xs = []
    for b in range(B):
        z = np.zeros(op.K)
        z[:784] = W.images(90 + b, 1, 28, 28)[0].reshape(-1)
        xs.append(p.encrypt_values(z, nonce=1 + b)[0])
    wc = [p.encrypt_values(np.full(op.K, cw[co, a, b]), nonce=10 + co * 9 + a * 3 + b)[0]
          for co in range(C) for a in range(3) for b in range(3)]
    V = W.deep_fc_vectors(fw, C, 13, 13, 28, op.K)
    vc = [p.encrypt_values(V[r, c], nonce=100 + r * C + c)[0] for r in range(n_out) for c in range(C)]
    y = H.hc_enc_conv2d_single_hoisted_batch(p.ctx, p.g_evk, xs, 28, wc, C, 3, 3)
    a = H.hc_enc_poly_act(p.ctx, p.g_evk, y, act)
    pl = H.hc_enc_pool(p.ctx, p.g_evk, H.HC_PACK_SINGLE, a, B * C, 26, 28)
    for b in range(B):
        zb = H.hc_enc_fc_rotsum(p.ctx, p.g_evk, pl[b * C:(b + 1) * C], vc, n_out, 10)
        y1 = H.hc_enc_conv2d(p.ctx, p.g_evk, H.HC_PACK_SINGLE_HOISTED, [xs[b]], 28, 28, 1, wc, C, 3, 3, 1)
        a1 = H.hc_enc_poly_act(p.ctx, p.g_evk, y1, act)
        p1 = H.hc_enc_pool(p.ctx, p.g_evk, H.HC_PACK_SINGLE, a1, C, 26, 28)
        z1 = H.hc_enc_fc_rotsum(p.ctx, p.g_evk, p1, vc, n_out, 10)
        for r in range(n_out):
            np.testing.assert_array_equal(H.hc_ct_export(p.ctx, zb[r])[0], H.hc_ct_export(p.ctx, z1[r])[0])
