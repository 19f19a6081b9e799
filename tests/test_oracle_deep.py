"""Pins of the oracle's deep single-ciphertext circuits (hoisted conv,
degree-7 Paterson-Stockmeyer activation, pooling by rotations, FC by
rotate-and-sum) against the FP64 network and plain polynomial evaluation."""
import numpy as np
import pytest

from oracle import ckks, cnn, encoding
from paper_2102_00319_gb300 import workloads as W


def test_relu_interpolant_nodes():
    c = W.relu_cheb7()
    k = np.arange(8)
    nodes = 2 ** 0.5 * np.cos((2 * k + 1) * np.pi / 16)
    assert np.allclose(cnn.poly_eval(nodes, c), np.maximum(nodes, 0), atol=1e-12)
    xs = np.linspace(-1.4, 1.4, 101)
    assert np.max(np.abs(cnn.poly_eval(xs, c) - np.maximum(xs, 0))) < 0.1


@pytest.fixture(scope="module")
def small():
    p = ckks.Params(11, [60] + [40] * 8, [60, 60], 40)
    sk, pk, evk = ckks.keygen(p, 31, W.deep_rot_steps(28, 10))
    return p, sk, pk, evk


def enc(p, pk, z, nonce, level=None):
    m = encoding.encode(z, p.N, p.scale)
    return ckks.encrypt(p, pk, ckks.plaintext_from_ints(p, m, p.L if level is None else level, p.scale), 5, nonce)


def dec(p, sk, ct):
    d = ckks.decrypt(p, sk, ct)
    return encoding.decode(d.m, p.q[: ct.level + 1], p.N, ct.scale).real


def test_poly7_matches_fp64(small):
    p, sk, pk, evk = small
    c = W.relu_cheb7()
    z = W.slot_values(3, p.K, -1.4, 1.4)
    y = cnn.enc_poly7(p, evk, enc(p, pk, z, 1, level=6), c)
    assert y.level == 2
    assert np.max(np.abs(dec(p, sk, y) - cnn.poly_eval(z, c))) < 2.0 ** -15


def test_deep_network_matches_fp64(small):
    p, sk, pk, evk = small
    C, n_out = 2, 3
    img = W.images(4, 1, 28, 28)[0]
    cw = W.conv_weights(5, C, 3, 3)[:, :, :, 0]
    fw = W.fc_weights(6, n_out, 13 * 13 * C)
    act = W.relu_cheb7()
    z = np.zeros(p.K)
    z[:784] = img.reshape(-1)
    x = enc(p, pk, z, 1)
    wcts = [enc(p, pk, np.full(p.K, cw[co, a, b]), 10 + co * 9 + a * 3 + b) for co in range(C) for a in range(3)
            for b in range(3)]
    y = cnn.enc_conv2d_single_hoisted(p, evk, x, 28, wcts, 3, 3, C)
    a = [cnn.enc_poly7(p, evk, t, act) for t in y]
    pl = [cnn.enc_pool_single(p, evk, t, 28) for t in a]
    V = W.deep_fc_vectors(fw, C, 13, 13, 28, p.K)
    vcts = [enc(p, pk, V[r, c], 100 + r * C + c) for r in range(n_out) for c in range(C)]
    out = cnn.enc_fc_rotsum(p, evk, pl, vcts, n_out, 10)
    got = np.array([dec(p, sk, t)[0] for t in out])
    ref = cnn.deep_network(img, cw, act, fw)
    assert np.max(np.abs(got - ref)) < 2.0 ** -15
