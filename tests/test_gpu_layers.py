"""GPU parity of the encrypted CNN layers (Eq. 3 convolution, Eq. 4
activation, Eq. 5-6 mean pooling, fully connected) against the CPU oracle's
canonical circuits, bit for bit, and of the decrypted network against the
FP64 plaintext network."""
import numpy as np
import pytest

from oracle import ckks, cnn
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 2.0 ** -15  # decrypted logits vs the FP64 network


@pytest.fixture(scope="module")
def net():
    """A small batch-packed CNN: 9x9 images, conv 3x3 stride 2 (ragged: the
    last column/row of the image is unused) with 3 channels, x^2, 2x2 mean
    pool, FC 12 -> 5; N = 2^10 (512 images), L = 4, Delta = 2^40."""
    from hc_pair import Pair
    p = Pair(10, [60, 40, 40, 40, 40], [60], 40, seed=21)
    Hh, Ww, cout, k, s, n_out = 9, 9, 3, 3, 2, 5
    imgs = W.images(1, p.op.K, Hh, Ww)
    cw = W.conv_weights(2, cout, k, k)
    Ho = (Hh - k) // s + 1
    n_in = (Ho // 2) * (Ho // 2) * cout
    fw = W.fc_weights(3, n_out, n_in)
    xs = [p.encrypt_values(imgs[:, h, w], nonce=h * Ww + w) for h in range(Hh) for w in range(Ww)]
    ws = [p.encrypt_values(np.full(p.op.K, cw[co, a, b, 0]), nonce=1000 + (co * k + a) * k + b)
          for co in range(cout) for a in range(k) for b in range(k)]
    fws = [p.encrypt_values(np.full(p.op.K, fw[r, i]), nonce=2000 + r * n_in + i) for r in range(n_out) for i in range(n_in)]
    return dict(p=p, imgs=imgs, cw=cw, fw=fw, xs=xs, ws=ws, fws=fws, H=Hh, W=Ww, cout=cout, k=k, s=s, Ho=Ho,
                n_in=n_in, n_out=n_out)


def test_cnn_layers_bit_exact_and_close_to_fp64(net):
    p = net["p"]
    op, ctx, evk = p.op, p.ctx, p.g_evk
    gx = [g for g, _ in net["xs"]]
    ox = [o for _, o in net["xs"]]
    gw = [g for g, _ in net["ws"]]
    ow = [o for _, o in net["ws"]]
    gy = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, gx, net["H"], net["W"], 1, gw, net["cout"], net["k"], net["k"],
                         net["s"])
    oy = cnn.enc_conv2d_batch(op, p.o_evk, ox, net["H"], net["W"], 1, ow, net["cout"], net["k"], net["k"], net["s"])
    assert len(gy) == len(oy) == net["Ho"] * net["Ho"] * net["cout"]
    for i, (g, o) in enumerate(zip(gy, oy)):
        p.assert_same(g, o, "conv %d" % i)
    ga = H.hc_enc_poly_act(ctx, evk, gy, (0.0, 0.0, 1.0))
    oa = [cnn.enc_poly_act(op, p.o_evk, c, (0.0, 0.0, 1.0)) for c in oy]
    for i, (g, o) in enumerate(zip(ga, oa)):
        p.assert_same(g, o, "act %d" % i)
    gp = H.hc_enc_pool(ctx, evk, H.HC_PACK_BATCH, ga, net["cout"], net["Ho"], net["Ho"])
    opl = cnn.enc_pool_batch(op, oa, net["cout"], net["Ho"], net["Ho"])
    for i, (g, o) in enumerate(zip(gp, opl)):
        p.assert_same(g, o, "pool %d" % i)
    gf = H.hc_enc_fc(ctx, evk, H.HC_PACK_BATCH, gp, [g for g, _ in net["fws"]], net["n_out"])
    of = cnn.enc_fc(op, p.o_evk, opl, [o for _, o in net["fws"]], net["n_out"])
    for i, (g, o) in enumerate(zip(gf, of)):
        p.assert_same(g, o, "fc %d" % i)
    logits = np.stack([p.decrypt_gpu(z).real for z in gf], axis=1)
    ref = cnn.network(net["imgs"][..., None], net["cw"], net["s"], (0.0, 0.0, 1.0), net["fw"])
    assert np.max(np.abs(logits - ref)) < TOL


def test_paper_activation_bit_exact(net):
    """g(u) = 0.47 + 0.50 u + 0.09 u^2 (Eq. 4), two levels, and its FP64 value."""
    p = net["p"]
    coeffs = (0.47, 0.50, 0.09)
    z = W.slot_values(40, p.op.K, -1.4, 1.4)
    gs, os_ = zip(*[p.encrypt_values(z * (1 - 0.1 * i), nonce=3000 + i) for i in range(3)])
    gout = H.hc_enc_poly_act(p.ctx, p.g_evk, list(gs), coeffs)
    for i, (g, o) in enumerate(zip(gout, os_)):
        exp = cnn.enc_poly_act(p.op, p.o_evk, o, coeffs)
        p.assert_same(g, exp, "g(u) %d" % i)
        got = p.decrypt_gpu(g).real
        assert np.max(np.abs(got - cnn.poly_act(z * (1 - 0.1 * i), coeffs))) < TOL


def test_fc_with_bias(net):
    p = net["p"]
    op = p.op
    xs = [p.encrypt_values(W.slot_values(50 + i, op.K), level=2, nonce=4000 + i) for i in range(4)]
    ws = [p.encrypt_values(np.full(op.K, 0.1 * (i - 3)), nonce=4100 + i) for i in range(8)]
    # the bias carries scale(x) * scale(w); bit-exactness needs only its integers
    bscale = xs[0][1].scale * ws[0][1].scale
    bias = [p.encrypt(W.int_plaintext(4300 + r, op.N, 2 ** 40), level=2, nonce=4200 + r, scale=bscale)
            for r in range(2)]
    gf = H.hc_enc_fc(p.ctx, p.g_evk, H.HC_PACK_BATCH, [g for g, _ in xs], [g for g, _ in ws], 2,
                     bias=[g for g, _ in bias])
    of = cnn.enc_fc(op, p.o_evk, [o for _, o in xs], [o for _, o in ws], 2, bias_cts=[o for _, o in bias])
    for g, o in zip(gf, of):
        p.assert_same(g, o, "fc+bias")


def test_single_packing_conv_then_square():
    """One 8x8 U[0,1] image in one ciphertext, a 3x3 N(0, 0.3) filter as nine
    slot-constant ciphertexts, conv by rotations, then x^2 (N = 2^12,
    q = 50/30/30 bits, P = 50 bits, Delta = 2^30)."""
    from hc_pair import Pair
    ps = W.SINGLE_N12
    rots = cnn.conv_rotations(8, 3, 3)
    p = Pair(ps.log_n, ps.q_bits, ps.p_bits, ps.log2_scale, seed=W.MASTER_SEED + 1, rot_steps=rots)
    img = W.images(5, 1, 8, 8)[0]
    w = W.conv_weights(6, 1, 3, 3)[0, :, :, 0]
    z = np.zeros(p.op.K)
    z[:64] = img.reshape(-1)
    gx, ox = p.encrypt_values(z, nonce=1)
    wcts = [p.encrypt_values(np.full(p.op.K, w[a, b]), nonce=10 + a * 3 + b) for a in range(3) for b in range(3)]
    gy = H.hc_enc_conv2d(p.ctx, p.g_evk, H.HC_PACK_SINGLE, [gx], 8, 8, 1, [g for g, _ in wcts], 1, 3, 3, 1)
    oy = cnn.enc_conv2d_single(p.op, p.o_evk, ox, 8, [o for _, o in wcts], 3, 3)
    p.assert_same(gy[0], oy, "single conv")
    g2 = H.hc_enc_poly_act(p.ctx, p.g_evk, gy, (0.0, 0.0, 1.0))
    o2 = cnn.enc_poly_act(p.op, p.o_evk, oy, (0.0, 0.0, 1.0))
    p.assert_same(g2[0], o2, "single x^2")
    ref = cnn.conv2d(img[None, :, :, None], w[None, :, :, None])[0, :, :, 0] ** 2
    got = p.decrypt_gpu(g2[0]).real
    valid = np.array([got[m * 8 + n] for m in range(6) for n in range(6)])
    # Delta = 2^30 leaves about 2^-12 of precision after two products
    assert np.max(np.abs(valid - ref.reshape(-1))) < 2.0 ** -10


def test_layer_edge_cases(net):
    p = net["p"]
    ctx, evk = p.ctx, p.g_evk
    assert H.hc_enc_poly_act(ctx, evk, [], (0.0, 0.0, 1.0)) == []
    g0, _ = p.encrypt_values(W.slot_values(60, p.op.K), level=0, nonce=5000)
    with pytest.raises(H.HcError) as e:
        H.hc_enc_poly_act(ctx, evk, [g0], (0.0, 0.0, 1.0))
    assert e.value.code == -5
    g1, _ = p.encrypt_values(W.slot_values(61, p.op.K), level=1, nonce=5001)
    with pytest.raises(H.HcError) as e:
        H.hc_enc_poly_act(ctx, evk, [g1], (0.47, 0.5, 0.09))  # needs two levels
    assert e.value.code == -5
    g2, _ = p.encrypt_values(W.slot_values(62, p.op.K), level=2, nonce=5002)
    with pytest.raises(H.HcError) as e:  # mixed levels in one conv
        H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, [g1, g2, g1, g1], 2, 2, 1, [g1], 1, 1, 1, 1)
    assert e.value.code == -2
    with pytest.raises(H.HcError) as e:  # weights below the activations
        H.hc_enc_fc(ctx, evk, H.HC_PACK_BATCH, [g2], [g1], 1)
    assert e.value.code == -2
    # odd pooling extents drop the last row / column (Eq. 5 blocks)
    xs = [p.encrypt_values(W.slot_values(70 + i, p.op.K), level=2, nonce=5100 + i) for i in range(15)]
    gp = H.hc_enc_pool(ctx, evk, H.HC_PACK_BATCH, [g for g, _ in xs], 1, 3, 5)
    op_ = cnn.enc_pool_batch(p.op, [o for _, o in xs], 1, 3, 5)
    assert len(gp) == len(op_) == 2
    for g, o in zip(gp, op_):
        p.assert_same(g, o, "odd pool")


def test_fc_long_sum_folds_bit_exact(net):
    """An FC output summing 150 products with a 60-bit prime in the chain: the
    tensor kernel's 128-bit sums fold every 63 terms (Karatsuba middle sum
    carried through the folds); bit-exact against the oracle."""
    p = net["p"]
    op = p.op
    n_in, n_out = 150, 2
    xs = [p.encrypt_values(W.slot_values(300 + i, op.K), level=2, nonce=3000 + i) for i in range(n_in)]
    ws = [p.encrypt_values(W.slot_values(600 + i, op.K), level=3, nonce=4000 + i) for i in range(n_in * n_out)]
    got = H.hc_enc_fc(p.ctx, p.g_evk, H.HC_PACK_BATCH, [g for g, _ in xs], [g for g, _ in ws], n_out)
    want = cnn.enc_fc(op, p.o_evk, [o for _, o in xs], [o for _, o in ws], n_out)
    for g, o in zip(got, want):
        p.assert_same(g, o, "fc 150 terms")


def test_tensor_group_choices_bit_identical(net):
    """Every HC_TUNE_TENSOR_GROUP value (0: one output per thread; 1..5: up to
    that many outputs sharing their x loads) gives the oracle's words for the
    conv (3 channels per position) and an FC with 150 terms over 2 classes
    (several staged tiles of terms, a ragged last tile, folds of the 128-bit
    sums)."""
    p = net["p"]
    op, ctx, evk = p.op, p.ctx, p.g_evk
    gx = [g for g, _ in net["xs"]]
    gw = [g for g, _ in net["ws"]]
    oy = cnn.enc_conv2d_batch(op, p.o_evk, [o for _, o in net["xs"]], net["H"], net["W"], 1,
                              [o for _, o in net["ws"]], net["cout"], net["k"], net["k"], net["s"])
    n_in, n_out = 150, 2
    fx = [p.encrypt_values(W.slot_values(700 + i, op.K), level=2, nonce=5000 + i) for i in range(n_in)]
    fwc = [p.encrypt_values(W.slot_values(900 + i, op.K), level=2, nonce=6000 + i) for i in range(n_in * n_out)]
    of = cnn.enc_fc(op, p.o_evk, [o for _, o in fx], [o for _, o in fwc], n_out)
    default = H.hc_tune_get(ctx, H.HC_TUNE_TENSOR_GROUP)
    assert default == 5
    try:
        for v in range(6):
            H.hc_tune_set(ctx, H.HC_TUNE_TENSOR_GROUP, v)
            gy = H.hc_enc_conv2d(ctx, evk, H.HC_PACK_BATCH, gx, net["H"], net["W"], 1, gw, net["cout"], net["k"],
                                 net["k"], net["s"])
            for i, (g, o) in enumerate(zip(gy, oy)):
                p.assert_same(g, o, "group %d conv %d" % (v, i))
            gf = H.hc_enc_fc(ctx, evk, H.HC_PACK_BATCH, [g for g, _ in fx], [g for g, _ in fwc], n_out)
            for i, (g, o) in enumerate(zip(gf, of)):
                p.assert_same(g, o, "group %d fc %d" % (v, i))
    finally:
        H.hc_tune_set(ctx, H.HC_TUNE_TENSOR_GROUP, default)
    with pytest.raises(H.HcError):
        H.hc_tune_set(ctx, H.HC_TUNE_TENSOR_GROUP, 6)


def test_activation_over_mixed_levels(net):
    """hc_enc_poly_act over inputs at several levels (each level's batch a
    concurrent branch) gives each input the words of a call at its own level
    and of the oracle, for x^2 and for Eq. 4's g."""
    p = net["p"]
    op = p.op
    levels = [4, 2, 3, 4, 2, 3, 4]
    pairs = [p.encrypt_values(W.slot_values(800 + i, op.K, -1.2, 1.2), level=lv, nonce=8000 + i)
             for i, lv in enumerate(levels)]
    gs = [g for g, _ in pairs]
    for coeffs in ((0.0, 0.0, 1.0), (0.47, 0.50, 0.09)):
        got = H.hc_enc_poly_act(p.ctx, p.g_evk, gs, coeffs)
        for i, (g, o) in enumerate(pairs):
            alone = H.hc_enc_poly_act(p.ctx, p.g_evk, [g], coeffs)[0]
            assert np.array_equal(H.hc_ct_export(p.ctx, got[i])[0], H.hc_ct_export(p.ctx, alone)[0]), (coeffs, i)
            if i < 3:
                p.assert_same(got[i], cnn.enc_poly_act(op, p.o_evk, o, coeffs), "mixed-level g %d" % i)
