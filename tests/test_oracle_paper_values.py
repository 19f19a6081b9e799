"""The paper's printed values (tests/golden/paper_printed_values.json, each
entry with its passage) against the oracle's canonical circuits and the
workload definitions.

Operation counts are taken by running the oracle's layer circuits with the
scheme operations replaced by counting stand-ins (the circuits only call
those operations and read levels and scales), so what is counted is exactly
the sequence of operations the oracle, and the library that is bit-exact
with it, performs.  Where the count differs from the paper's, the test
states the reading that explains it."""
import json
import math
import os

import pytest

from oracle import ckks, cnn
from paper_2102_00319_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")))["entries"]


class FakeCt:
    def __init__(self, level, scale=2.0 ** 30, degree=1):
        self.level, self.scale, self.degree = level, scale, degree


class FakeParams:
    def __init__(self, L):
        self.L = L
        self.q = [float(2 ** 30 + 1 + 2 * i) for i in range(L + 1)]


@pytest.fixture
def counter(monkeypatch):
    """Counting stand-ins for the scheme operations the layer circuits call."""
    c = {"ct_ct_mult": 0, "ct_ct_add": 0, "ct_pt_mult": 0, "ct_pt_add": 0, "relin": 0, "rescale": 0}

    def tensor_sum(params, xs, ys):
        assert len(xs) == len(ys) and xs
        c["ct_ct_mult"] += len(xs)
        c["ct_ct_add"] += len(xs) - 1  # an inner product of T terms: T products, T - 1 additions
        return FakeCt(xs[0].level, xs[0].scale * ys[0].scale, 2)

    def mul(params, x, y):
        c["ct_ct_mult"] += 1
        return FakeCt(x.level, x.scale * y.scale, 2)

    def add(params, x, y):
        assert x.level == y.level
        c["ct_ct_add"] += 1
        return FakeCt(x.level, x.scale, max(x.degree, y.degree))

    def mul_const(params, x, v, const_scale):
        c["ct_pt_mult"] += 1
        return FakeCt(x.level, x.scale * const_scale, x.degree)

    def add_const(params, x, v):
        c["ct_pt_add"] += 1
        return FakeCt(x.level, x.scale, x.degree)

    def relin(params, evk, d):
        c["relin"] += 1
        return FakeCt(d.level, d.scale, 1)

    def rescale(params, x):
        c["rescale"] += 1
        return FakeCt(x.level - 1, x.scale / params.q[x.level], x.degree)

    def drop_to_level(params, x, level):
        assert level <= x.level
        return FakeCt(level, x.scale, x.degree)

    for name, fn in dict(tensor_sum=tensor_sum, mul=mul, add=add, mul_const=mul_const, add_const=add_const,
                         relin=relin, rescale=rescale, drop_to_level=drop_to_level).items():
        monkeypatch.setattr(ckks, name, fn)
    return c


def conv_count(M, N, P, Q):
    return (M - P + 1) * (N - Q + 1) * P * Q


@pytest.mark.parametrize("M,N,P,Q", [(5, 5, 3, 3), (6, 4, 2, 3), (28, 28, 3, 3)])
def test_conv_counts_match_the_paper(counter, M, N, P, Q):
    """One filter, no padding, stride 1: the paper's (M-P+1)(N-Q+1)PQ CT-CT
    mults exactly.  It prints the same number of CT-CT adds; an inner product
    of PQ terms needs PQ - 1 additions, so the circuit does (M-P+1)(N-Q+1)
    fewer (the paper counts one accumulation per product).  One
    relinearisation and one rescale per output: depth 1."""
    assert GOLDEN["conv_ct_ct_mults"]["formula"] == "(M-P+1)(N-Q+1)PQ"
    params = FakeParams(3)
    x = [FakeCt(3) for _ in range(M * N)]
    w = [FakeCt(3) for _ in range(P * Q)]
    y = cnn.enc_conv2d_batch(params, None, x, M, N, 1, w, 1, P, Q, 1)
    outs = (M - P + 1) * (N - Q + 1)
    assert len(y) == outs
    assert counter["ct_ct_mult"] == conv_count(M, N, P, Q)
    assert counter["ct_ct_add"] == conv_count(M, N, P, Q) - outs
    assert counter["relin"] == counter["rescale"] == outs
    assert all(3 - c.level == GOLDEN["conv_depth"]["value"] for c in y)


def test_activation_counts_and_coefficients(counter):
    """g(u) = 0.47 + 0.50 u + 0.09 u^2 (Eq. 4): the circuit does the paper's
    1 CT-CT mult, 2 CT-PT mults and 1 CT-PT add; it does 1 CT-CT add where
    the paper prints 2 (a0 + a1 u + a2 u^2 is two additions, one of which adds
    the plaintext constant a0: the reading counts that one as the CT-PT add)."""
    g = GOLDEN["relu_poly"]
    assert tuple(g["coefficients"]) == W.PAPER_CNN["act"] == (0.47, 0.50, 0.09)
    ops = GOLDEN["act_ops"]
    params = FakeParams(4)
    out = cnn.enc_poly_act(params, None, FakeCt(4), tuple(g["coefficients"]))
    assert counter["ct_ct_mult"] == ops["ct_ct_mult"]
    assert counter["ct_pt_mult"] == ops["ct_pt_mult"]
    assert counter["ct_pt_add"] == ops["ct_pt_add"]
    assert counter["ct_ct_add"] == ops["ct_ct_add"] - 1
    # depth: the paper's "depth 1" is one CT-CT mult level; the RNS circuit
    # spends two rescales (the product, then its constant factor)
    assert out.level == 4 - 2


def test_x_squared_is_one_product(counter):
    """x^2 (the activation of the smaller workloads) is the first step of the
    circuit alone: one CT-CT mult, one relinearisation, one rescale."""
    out = cnn.enc_square(FakeParams(2), None, FakeCt(2))
    assert counter["ct_ct_mult"] == counter["relin"] == counter["rescale"] == 1
    assert counter["ct_pt_mult"] == counter["ct_ct_add"] == counter["ct_pt_add"] == 0
    assert out.level == 1


def test_pool_counts(counter):
    """2x2 mean pool: the paper's 1 CT-PT mult (x 1/4) and no CT-CT mult; it
    prints 4 CT-CT adds where a sum of four needs 3, the circuit's
    ((a + b) + (c + d))."""
    ops = GOLDEN["pool_ops"]
    params = FakeParams(2)
    C, H, Wd = 1, 4, 6
    y = cnn.enc_pool_batch(params, [FakeCt(2) for _ in range(H * Wd * C)], C, H, Wd)
    blocks = (H // 2) * (Wd // 2)
    assert len(y) == blocks
    assert counter["ct_ct_mult"] == ops["ct_ct_mult"] * blocks
    assert counter["ct_pt_mult"] == ops["ct_pt_mult"] * blocks
    assert counter["ct_ct_add"] == (ops["ct_ct_add"] - 1) * blocks


def test_mnist_network_shape_and_fc_memory():
    """The paper's network: 28x28 input, 28 filters 3x3 without padding,
    ActPool, flatten 13 x 13 x 28 = 4732, FC 4732 x 10; per filter the FC
    holds (M-P+1)(N-Q+1)(R+1)/4 ciphertexts: the 13 x 13 pooled inputs and
    their R weight ciphertexts each."""
    net = GOLDEN["mnist_network"]
    d = W.PAPER_CNN
    assert [d["H"], d["W"]] == net["image"] and d["cout"] == net["filters"]
    assert [d["k"], d["k"]] == net["kernel"] and d["stride"] == 1 and d["n_out"] == net["fc"][1]
    conv_hw = d["H"] - d["k"] + 1
    pooled = conv_hw // 2
    assert [pooled, pooled, d["cout"]] == net["flatten_shape"]
    assert pooled * pooled * d["cout"] == net["flatten"] == net["fc"][0]
    R = GOLDEN["fc_cts_in_memory_per_filter"]["R"]
    held = conv_hw * conv_hw * (R + 1) / 4
    assert held == pooled * pooled + pooled * pooled * R  # inputs + weights of one filter's FC slice


def test_fc_uses_one_product_per_weight(counter):
    """FC of n_in inputs to R classes: n_in R CT-CT mults, one
    relinearisation and rescale per class, over n_in + n_in R ciphertexts."""
    params = FakeParams(2)
    n_in, R = 7, 3
    x = [FakeCt(2) for _ in range(n_in)]
    w = [FakeCt(2) for _ in range(n_in * R)]
    z = cnn.enc_fc(params, None, x, w, R)
    assert len(z) == R
    assert counter["ct_ct_mult"] == n_in * R and counter["relin"] == counter["rescale"] == R


def test_he_parameters():
    """m = 2^16: phi(m) = 32768 and K = phi(m) / 2 = 16384 slots; the
    paper-shape workload's ring degree is N = phi(m) (reading of the paper's
    m), and its batch fills the K slots."""
    sympy = pytest.importorskip("sympy")
    hp = GOLDEN["he_params"]
    assert int(sympy.totient(hp["m"])) == hp["phi_m"] and hp["phi_m"] // 2 == hp["slots"]
    assert 2 ** W.PAPER_N15.log_n == hp["phi_m"]
    assert math.isclose(hp["slots"], (2 ** W.PAPER_N15.log_n) // 2)
