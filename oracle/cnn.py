"""FP64 plaintext CNN and the canonical encrypted layer circuits (oracle).

TEST INFRASTRUCTURE ONLY.

Plaintext network (the paper's building blocks, Sec. "Convolutional Neural
Network (CNN)" and "Proposed Approach"):
  * convolution, Eq. 1: Y_{m,n} = <X^_{m,n}, W^>, window anchored at its
    top-left element, no padding; a stride s takes windows at (m s, n s);
  * activation: the polynomial g(u) = a0 + a1 u + a2 u^2 of Eq. 4
    (0.47, 0.50, 0.09 in the paper; x^2 is (0, 0, 1));
  * mean pooling 2x2, Eq. 5-6: Z_{i,j} = mean of Y at rows 2i-1, 2i and
    columns 2j-1, 2j (1-based), i.e. non-overlapping 2x2 blocks;
  * fully connected Z = W X (+ bias), softmax left to the client.
Activations are channel-last: flat index (i W + j) C + c.

Encrypted circuits (the canonical circuit both implementations follow):
  * conv, batch packing (Fig. 2, Eq. 3): each output ciphertext is the sum of
    all kh*kw*Cin tensor products X (x) W, then ONE relinearisation and ONE
    rescale.  Weights above the inputs' level are dropped to it first.
  * conv, single-ciphertext packing: Y = sum_{p,q} rot(X, p W + q) (x) W_{p,q},
    then one relinearisation and one rescale.
  * poly_act: see `enc_poly_act`.
  * pool: ((a + b) + (c + d)), times 1/4 encoded at scale q_level, rescale.
  * fc: sum_k X_k (x) W_{r,k} with the weights first dropped to the
    activations' level, (+ bias before the rescale), one relinearisation, one
    rescale.
"""
import numpy as np

from . import ckks


# ---------------------------------------------------------------------------
# FP64 plaintext network
# ---------------------------------------------------------------------------
def conv2d(x, w, stride=1):
    """x: [B][H][W][Cin], w: [Cout][kh][kw][Cin] -> [B][Ho][Wo][Cout]."""
    B, H, W, Cin = x.shape
    Cout, kh, kw, _ = w.shape
    Ho = (H - kh) // stride + 1
    Wo = (W - kw) // stride + 1
    y = np.zeros((B, Ho, Wo, Cout), dtype=np.float64)
    for m in range(Ho):
        for n in range(Wo):
            win = x[:, m * stride: m * stride + kh, n * stride: n * stride + kw, :]  # [B][kh][kw][Cin]
            for co in range(Cout):
                y[:, m, n, co] = np.sum(win * w[co][None], axis=(1, 2, 3))
    return y


def poly_act(x, coeffs):
    a0, a1, a2 = coeffs
    return a0 + a1 * x + a2 * x * x


def mean_pool2(x):
    """[B][H][W][C] -> [B][H//2][W//2][C], non-overlapping 2x2 means."""
    B, H, W, C = x.shape
    Ho, Wo = H // 2, W // 2
    x = x[:, : 2 * Ho, : 2 * Wo, :]
    return (x[:, 0::2, 0::2] + x[:, 1::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 1::2]) / 4.0


def fc(x, w, bias=None):
    """x: [B][n_in] (flattened channel-last), w: [n_out][n_in]."""
    y = x @ w.T
    if bias is not None:
        y = y + bias[None, :]
    return y


def network(x, conv_w, stride, act_coeffs, fc_w, fc_b=None):
    """conv -> poly act -> mean pool -> flatten -> fc (logits)."""
    y = conv2d(x, conv_w, stride)
    y = poly_act(y, act_coeffs)
    y = mean_pool2(y)
    return fc(y.reshape(y.shape[0], -1), fc_w, fc_b)


# ---------------------------------------------------------------------------
# Encrypted circuits (batch packing: one ciphertext per pixel / weight)
# ---------------------------------------------------------------------------
def _at_level(params, cts, level):
    """Weights above the activations' level are dropped to it (as in the FC)."""
    return [c if c.level == level else ckks.drop_to_level(params, c, level) for c in cts]


def enc_conv2d_batch(params, evk, x_cts, H, W, Cin, w_cts, Cout, kh, kw, stride):
    """x_cts[(h W + w) Cin + ci]; w_cts[((co kh + p) kw + q) Cin + ci];
    returns y[(m Wo + n) Cout + co]."""
    w_cts = _at_level(params, w_cts, x_cts[0].level)
    Ho = (H - kh) // stride + 1
    Wo = (W - kw) // stride + 1
    out = []
    for m in range(Ho):
        for n in range(Wo):
            for co in range(Cout):
                xs, ws = [], []
                for p in range(kh):
                    for q in range(kw):
                        for ci in range(Cin):
                            xs.append(x_cts[((m * stride + p) * W + (n * stride + q)) * Cin + ci])
                            ws.append(w_cts[((co * kh + p) * kw + q) * Cin + ci])
                d = ckks.tensor_sum(params, xs, ws)
                out.append(ckks.rescale(params, ckks.relin(params, evk, d)))
    return out


def enc_square(params, evk, u):
    """x^2: relinearised tensor square, rescaled."""
    return ckks.rescale(params, ckks.relin(params, evk, ckks.mul(params, u, u)))


def enc_poly_act(params, evk, u, coeffs):
    """g(u) = a0 + a1 u + a2 u^2 (Eq. 4).

    (0, 0, 1) is x^2 (one level).  Otherwise (two levels):
      1. t = rescale(relin(u (x) u))                  level l-1, scale s_t
      2. t = rescale(t * a2 @ scale q_{l-1})          level l-2, scale ~ s_t
      3. v = rescale(u * a1 @ scale s_t q_l / s_u), dropped to level l-2
      4. out = (t + v) + a0                           scale of t
    A zero a1 skips step 3; a zero a0 skips the constant."""
    a0, a1, a2 = coeffs
    if a0 == 0 and a1 == 0 and a2 == 1:
        return enc_square(params, evk, u)
    lv = u.level
    t = enc_square(params, evk, u)
    t = ckks.rescale(params, ckks.mul_const(params, t, a2, float(params.q[lv - 1])))
    if a1 != 0:
        v = ckks.mul_const(params, u, a1, t.scale * float(params.q[lv]) / u.scale)
        v = ckks.drop_to_level(params, ckks.rescale(params, v), t.level)
        t = ckks.add(params, t, v)
    if a0 != 0:
        t = ckks.add_const(params, t, a0)
    return t


def enc_pool_batch(params, x_cts, C, H, W):
    """Mean 2x2 over channel-last x[(h W + w) C + c] -> [(i Wo + j) C + c]."""
    Ho, Wo = H // 2, W // 2
    out = []
    for i in range(Ho):
        for j in range(Wo):
            for c in range(C):
                a = x_cts[((2 * i) * W + 2 * j) * C + c]
                b = x_cts[((2 * i + 1) * W + 2 * j) * C + c]
                cc = x_cts[((2 * i) * W + 2 * j + 1) * C + c]
                d = x_cts[((2 * i + 1) * W + 2 * j + 1) * C + c]
                s = ckks.add(params, ckks.add(params, a, b), ckks.add(params, cc, d))
                s = ckks.mul_const(params, s, 0.25, float(params.q[s.level]))
                out.append(ckks.rescale(params, s))
    return out


def enc_fc(params, evk, x_cts, w_cts, n_out, bias_cts=None):
    """z_r = rescale(relin(sum_k x_k (x) w_{r,k}) [+ bias_r]);
    w_cts[r n_in + k], dropped to the activations' level first."""
    n_in = len(x_cts)
    lv = x_cts[0].level
    out = []
    for r in range(n_out):
        ws = [ckks.drop_to_level(params, w_cts[r * n_in + k], lv) for k in range(n_in)]
        d = ckks.tensor_sum(params, x_cts, ws)
        z = ckks.relin(params, evk, d)
        if bias_cts is not None:
            z = ckks.add(params, z, ckks.drop_to_level(params, bias_cts[r], lv))
        out.append(ckks.rescale(params, z))
    return out


# ---------------------------------------------------------------------------
# Encrypted circuits (single-ciphertext packing: image row-major in slots)
# ---------------------------------------------------------------------------
def conv_rotations(W, kh, kw):
    return [p * W + q for p in range(kh) for q in range(kw)]


def enc_conv2d_single(params, evk, x_ct, W, w_cts, kh, kw):
    """Y = sum_{p,q} rot(X, p W + q) (x) W_{p,q}; relin; rescale.
    Output slot m W + n holds Y_{m,n} for valid (m, n)."""
    xs = [ckks.rotate(params, evk, x_ct, r) for r in conv_rotations(W, kh, kw)]
    d = ckks.tensor_sum(params, xs, _at_level(params, w_cts, x_ct.level))
    return ckks.rescale(params, ckks.relin(params, evk, d))


# ---------------------------------------------------------------------------
# Deep single-ciphertext network (one image per ciphertext, N = 2^16 class)
# ---------------------------------------------------------------------------
def poly_eval(x, c):
    """sum_i c_i x^i (FP64)."""
    y = np.zeros_like(x)
    for ci in reversed(c):
        y = y * x + ci
    return y


def deep_network(img, conv_w, act, fc_w):
    """img [H][W], conv_w [C][3][3], act: coefficients c_0..c_d, fc_w
    [n_out][(H'/2)(W'/2)C] (channel-last flatten) -> logits [n_out]."""
    y = conv2d(img[None, :, :, None], conv_w[:, :, :, None])[0]  # [Ho][Wo][C]
    y = poly_eval(y, act)
    z = mean_pool2(y[None])[0]
    return fc_w @ z.reshape(-1)


def enc_conv2d_single_hoisted(params, evk, x_ct, W, w_cts, kh, kw, cout):
    """Conv with cout filters by one set of hoisted rotations of x:
    y_co = sum_t rot(x, r_t) (x) w[co kh kw + t]; relin; rescale."""
    rots = ckks.rotate_hoisted(params, evk, x_ct, conv_rotations(W, kh, kw))
    out = []
    T = kh * kw
    for co in range(cout):
        ws = _at_level(params, w_cts[co * T:(co + 1) * T], x_ct.level)
        d = ckks.tensor_sum(params, rots, ws)
        out.append(ckks.rescale(params, ckks.relin(params, evk, d)))
    return out


def enc_poly7(params, evk, u, c):
    """Degree-7 activation sum_i c_i u^i by a Paterson-Stockmeyer split
    (baby steps u, u^2, u^3, giant step u^4), four levels:
      u2 = rs(rl(u u))                       l-1
      u4 = rs(rl(u2 u2)),  u3 = rs(rl(u2 u))  l-2
      deg3(a, b, c, d) = a + b u + c u2 + d u3 at l-3 with the scale of
        rs(u3 * d @ q_{l-2}); the u and u2 terms are brought to it by their
        constant's scale, as in the degree-2 activation
      qa = deg3(c0..c3), qb = deg3(c4..c7)
      out = rs(rl(qb u4)) + rs(qa * 1 @ (target scale) q_{l-3} / s_qa)   l-4"""
    lv = u.level
    q = params.q
    u2 = enc_square(params, evk, u)
    u4 = enc_square(params, evk, u2)
    u3 = ckks.rescale(params, ckks.relin(params, evk, ckks.mul(params, u2, ckks.drop_to_level(params, u, lv - 1))))

    def deg3(a0, a1, a2, a3):
        t3 = ckks.rescale(params, ckks.mul_const(params, u3, a3, float(q[lv - 2])))
        u2d = ckks.drop_to_level(params, u2, lv - 2)
        t2 = ckks.rescale(params, ckks.mul_const(params, u2d, a2, t3.scale * float(q[lv - 2]) / u2d.scale))
        ud = ckks.drop_to_level(params, u, lv - 2)
        t1 = ckks.rescale(params, ckks.mul_const(params, ud, a1, t3.scale * float(q[lv - 2]) / ud.scale))
        return ckks.add_const(params, ckks.add(params, ckks.add(params, t3, t2), t1), a0)

    qa = deg3(*c[0:4])
    qb = deg3(*c[4:8])
    prod = ckks.rescale(params, ckks.relin(params, evk, ckks.mul(params, qb, ckks.drop_to_level(params, u4, lv - 3))))
    qa2 = ckks.rescale(params, ckks.mul_const(params, qa, 1.0, prod.scale * float(q[lv - 3]) / qa.scale))
    return ckks.add(params, prod, qa2)


def enc_pool_single(params, evk, y, W):
    """2x2 mean inside one ciphertext: ((y + rot W) + (rot 1 + rot W+1)) / 4,
    the three rotations hoisted; pooled (i, j) lands in slot 2i W + 2j."""
    rW, r1, rW1 = ckks.rotate_hoisted(params, evk, y, [W, 1, W + 1])
    s = ckks.add(params, ckks.add(params, y, rW), ckks.add(params, r1, rW1))
    s = ckks.mul_const(params, s, 0.25, float(params.q[s.level]))
    return ckks.rescale(params, s)


def enc_fc_rotsum(params, evk, x_cts, w_cts, n_out, span_log2):
    """z_r = rotate-and-sum over 2^span_log2 slots of rs(rl(sum_c x_c (x) w[r C + c]));
    the class score lands in slot 0."""
    C = len(x_cts)
    lv = x_cts[0].level
    out = []
    for r in range(n_out):
        ws = [ckks.drop_to_level(params, w_cts[r * C + c], lv) for c in range(C)]
        z = ckks.rescale(params, ckks.relin(params, evk, ckks.tensor_sum(params, x_cts, ws)))
        for k in range(span_log2):
            z = ckks.add(params, z, ckks.rotate(params, evk, z, 1 << k))
        out.append(z)
    return out
