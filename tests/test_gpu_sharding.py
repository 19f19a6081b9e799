"""The channel-sharded batch-packed CNN (paper_2102_00319_gb300.sharding) on
one GPU: every rank's share (conv -> x^2 -> pool for its channels, the FC's
degree-2 partial sums) is run in turn through the library, the partials are
summed with hc_add and relinearised and rescaled with
hc_relin_rescale_batch, as each rank does after the all-gather.  The
logits ciphertexts equal the oracle's whole network word for word for 1, 2
and 3 shards, and hc_enc_fc's own output."""
import numpy as np
import pytest

from oracle import cnn
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import sharding as S
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    from hc_pair import Pair
    p = Pair(10, [60, 40, 40, 40, 40], [60], 40, seed=23)
    c = dict(H=9, W=9, cin=1, cout=3, kh=3, kw=3, stride=2, n_out=4)
    plan1 = S.ShardPlan(world=1, **c)
    xs = [p.encrypt(W.int_plaintext(10 + i, p.op.N, 2 ** 30), nonce=i) for i in range(c["H"] * c["W"])]
    ws = [p.encrypt(W.int_plaintext(200 + i, p.op.N, 2 ** 30), nonce=1000 + i) for i in range(c["cout"] * 9)]
    fws = [p.encrypt(W.int_plaintext(400 + i, p.op.N, 2 ** 30), nonce=2000 + i)
           for i in range(c["n_out"] * plan1.n_in)]
    oy = cnn.enc_conv2d_batch(p.op, p.o_evk, [o for _, o in xs], c["H"], c["W"], 1, [o for _, o in ws], c["cout"],
                              3, 3, c["stride"])
    oa = [cnn.enc_square(p.op, p.o_evk, t) for t in oy]
    opl = cnn.enc_pool_batch(p.op, oa, c["cout"], plan1.Ho, plan1.Wo)
    want = cnn.enc_fc(p.op, p.o_evk, opl, [o for _, o in fws], c["n_out"])
    return p, c, [g for g, _ in xs], [g for g, _ in ws], [g for g, _ in fws], want


@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_cnn_equals_the_oracle_network(small, world):
    p, c, xs, ws, fws, want = small
    plan = S.ShardPlan(world=world, **c)
    parts = [S.rank_partials(H, p.ctx, p.g_evk, plan, r, xs, ws, fws, (0.0, 0.0, 1.0)) for r in range(world)]
    assert all(t.meta().degree == 2 for part in parts for t in part)
    logits = S.combine(H, p.ctx, p.g_evk, parts)
    assert len(logits) == c["n_out"]
    for r, (g, o) in enumerate(zip(logits, want)):
        p.assert_same(g, o, "class %d with %d shards" % (r, world))


def test_partial_fc_sums_and_batched_tail_equal_hc_enc_fc(small):
    """hc_enc_fc = hc_relin_rescale_batch(hc_enc_fc_partial(.)) word for word,
    and the unfused hc_rescale(hc_relin(.)) gives the same words."""
    p, c, xs, ws, fws, want = small
    plan = S.ShardPlan(world=1, **c)
    y = H.hc_enc_conv2d(p.ctx, p.g_evk, H.HC_PACK_BATCH, xs, c["H"], c["W"], 1, ws, c["cout"], 3, 3, c["stride"])
    a = H.hc_enc_poly_act(p.ctx, p.g_evk, y, (0.0, 0.0, 1.0))
    pl = H.hc_enc_pool(p.ctx, p.g_evk, H.HC_PACK_BATCH, a, c["cout"], plan.Ho, plan.Wo)
    full = H.hc_enc_fc(p.ctx, p.g_evk, H.HC_PACK_BATCH, pl, fws, c["n_out"])
    d = H.hc_enc_fc_partial(p.ctx, H.HC_PACK_BATCH, pl, fws, c["n_out"])
    tail = H.hc_relin_rescale_batch(p.ctx, p.g_evk, d)
    for f, t, dd in zip(full, tail, d):
        ref = H.hc_ct_export(p.ctx, f)[0]
        assert np.array_equal(H.hc_ct_export(p.ctx, t)[0], ref)
        assert np.array_equal(H.hc_ct_export(p.ctx, H.hc_rescale(p.ctx, H.hc_relin(p.ctx, p.g_evk, dd)))[0], ref)
    with pytest.raises(H.HcError):
        H.hc_relin_rescale_batch(p.ctx, p.g_evk, [d[0], full[0]])  # degree 1 among degree 2
