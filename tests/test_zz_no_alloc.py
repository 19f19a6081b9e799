"""The allocation-free relinearisation (hc_relin_noalloc) against hc_relin.

hc_relin_noalloc serves callers that cannot allocate device memory while
they run (memory fixed at start-up, graph capture, allocator-free serving
loops): it takes its scratch from a static device array and writes into an
output ciphertext the caller allocated beforehand.  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pair(log_n, q_bits, p_bits, scale, seed):
    import torch

    params = H.hc_params_create(log_n, q_bits, p_bits, scale)
    ctx = H.hc_ctx_create(params, 0, torch.cuda.current_stream().cuda_stream)
    sk, pk, evk = H.hc_keygen(ctx, seed)
    return ctx, sk, pk, evk


def _enc(ctx, pk, seed, level, nonce):
    pt = H.hc_encode(ctx, W.slot_values(seed, ctx.n // 2), 2.0 ** 40, level)
    return H.hc_encrypt(ctx, pk, pt, seed, nonce)


def test_noalloc_relin_matches_relin_twice():
    # N = 2^12, five q primes, two special primes: dnum = 3, ragged last digit
    ctx, sk, pk, evk = _pair(12, [60, 40, 40, 40, 40], [60, 60], 40, 31)
    level = 4
    out = H.hc_ct_import(ctx, np.zeros((2, level + 1, ctx.n), dtype=np.uint64), level, 1, 1.0)
    for call in range(2):  # two calls in a row share the scratch array
        a = _enc(ctx, pk, 100 + call, level, 2 * call)
        b = _enc(ctx, pk, 200 + call, level, 2 * call + 1)
        d = H.hc_mul(ctx, a, b)
        ref, _ = H.hc_ct_export(ctx, H.hc_relin(ctx, evk, d))
        H.hc_relin_noalloc(ctx, evk, d, out)
        got, meta = H.hc_ct_export(ctx, out)
        assert np.array_equal(got, ref), "call %d differs from hc_relin" % call
        assert meta.scale == d.scale
    # a lower level (fewer digits) after the larger one
    a = _enc(ctx, pk, 300, 2, 9)
    d = H.hc_mul(ctx, a, a)
    out2 = H.hc_ct_import(ctx, np.zeros((2, 3, ctx.n), dtype=np.uint64), 2, 1, 1.0)
    H.hc_relin_noalloc(ctx, evk, d, out2)
    assert np.array_equal(H.hc_ct_export(ctx, out2)[0], H.hc_ct_export(ctx, H.hc_relin(ctx, evk, d))[0])


def test_noalloc_rejects_oversize_and_bad_output():
    # 24 q primes at N = 2^14 need more scratch than the static array holds
    ctx, sk, pk, evk = _pair(14, [40] * 24, [40] * 4, 30, 32)
    a = _enc(ctx, pk, 1, 23, 0)
    d = H.hc_mul(ctx, a, a)
    out = H.hc_ct_import(ctx, np.zeros((2, 24, ctx.n), dtype=np.uint64), 23, 1, 1.0)
    with pytest.raises(H.HcError) as e:
        H.hc_relin_noalloc(ctx, evk, d, out)
    assert e.value.code == -1 and "scratch" in str(e.value)
    wrong = H.hc_ct_import(ctx, np.zeros((2, 23, ctx.n), dtype=np.uint64), 22, 1, 1.0)
    with pytest.raises(H.HcError) as e:
        H.hc_relin_noalloc(ctx, evk, d, wrong)
    assert e.value.code == -2
