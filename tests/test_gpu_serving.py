"""The serving loop on the GPU: requests of the N = 2^12 single-ciphertext
workload and of the uneven multi-instance workload arrive as a Poisson
stream, are admitted by device footprint and batched continuously; every
result equals the result of the same request served alone, bit for bit, and
decrypts to the plaintext convolution squared."""
import numpy as np
import pytest

from oracle import cnn
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import serving
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu


SETS = [(12, W.SINGLE_N12)] + [(k, W.uneven_params(k)) for k in (13, 14, 15)]


def build_models(streams, hoisted=False):
    models, sks = {}, {}
    for log_n, ps in SETS:
        params = H.hc_params_create(ps.log_n, list(ps.q_bits), list(ps.p_bits), ps.log2_scale)
        ctx = H.hc_ctx_create(params, 0, streams[log_n].cuda_stream)
        sk, pk, evk = H.hc_keygen(ctx, W.MASTER_SEED + 5 + log_n, W.SINGLE_CONV_STEPS)
        filt = W.conv_weights(60 + log_n, 1, 3, 3)[0, :, :, 0].reshape(-1)
        ws = [H.hc_encrypt(ctx, pk, H.hc_encode(ctx, np.full(ctx.n // 2, v), 2.0 ** 30, ctx.L), 3, t)
              for t, v in enumerate(filt)]
        models[log_n] = serving.Model(ctx=ctx, evk=evk, weights=ws, n=ctx.n, n_special=len(ps.p_bits),
                                      hoisted=hoisted)
        sks[log_n] = (sk, pk)
    return models, sks


def make_requests(models, sks, count, seed):
    reqs, imgs = [], []
    inst = W.uneven_instances(count)
    for i in range(count):
        log_n, lv = (12, 2) if i % 2 == 0 else inst[i]
        m = models[log_n]
        img = W.images(seed + i, 1, 8, 8)[0]
        z = np.zeros(m.n // 2)
        z[:64] = img.reshape(-1)
        ct = H.hc_encrypt(m.ctx, sks[log_n][1], H.hc_encode(m.ctx, z, 2.0 ** 30, lv), 11, i)
        reqs.append(serving.Request(i, log_n, ct, 0.0))
        imgs.append(img)
    return reqs, imgs


@pytest.mark.parametrize("per_degree_streams,hoisted", [(False, False), (True, False), (True, True)])
def test_served_results_equal_alone_and_decrypt(per_degree_streams, hoisted):
    """One stream for all ring degrees, or one per ring degree (the steps'
    groups then overlap on the device; completion is the event of every
    stream); plain or hoisted rotations."""
    import torch

    one_stream = torch.cuda.Stream()
    streams = {log_n: (torch.cuda.Stream() if per_degree_streams else one_stream) for log_n, _ in SETS}

    def event():
        evs = []
        for s in set(streams.values()):
            e = torch.cuda.Event()
            e.record(s)
            evs.append(e)
        return serving.AllOf(evs)

    models, sks = build_models(streams, hoisted)
    reqs, imgs = make_requests(models, sks, 24, 500)
    one = serving.footprint_bytes(models[15], 12)
    srv = serving.Server(models=models, budget_bytes=6 * one, max_batch=16)
    stats = serving.run(srv, reqs, serving.poisson_arrivals(200.0, len(reqs), 7), event)
    assert stats["requests"] == 24 and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert srv.peak_bytes <= 6 * one
    for i in (0, 1, 2, 3, 8, 23):
        r = reqs[i]
        m = models[r.log_n]
        alone = serving.Server(models=models, budget_bytes=6 * one)
        solo = serving.Request(1000 + i, r.log_n, r.ct, 0.0)
        serving.run(alone, [solo], np.array([0.0]), event)
        a = H.hc_ct_export(m.ctx, r.result)[0]
        b = H.hc_ct_export(m.ctx, solo.result)[0]
        assert np.array_equal(a, b), i
        v = H.hc_decode(m.ctx, H.hc_decrypt(m.ctx, sks[r.log_n][0], r.result)).real
        filt = W.conv_weights(60 + r.log_n, 1, 3, 3)[0, :, :, 0]
        ref = cnn.conv2d(imgs[i][None, :, :, None], filt[None, :, :, None])[0, :, :, 0] ** 2
        valid = np.array([v[p * 8 + q] for p in range(6) for q in range(6)])
        # scale 2^30 with 30-bit primes and one special prime: about 2^-10
        # per slot with plain rotations; hoisted rotations carry the key
        # switch's structured noise (the uncentred digit lift of the fast
        # basis conversion) into output slot 0, 3-5e-3 in the oracle's own
        # hoisted convolution of these requests, so 2^-7 there
        tol = 2.0 ** -7 if hoisted else 2.0 ** -8
        assert np.max(np.abs(valid - ref.reshape(-1))) < tol, i
