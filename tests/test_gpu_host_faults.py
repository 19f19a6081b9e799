"""Failure detection by host-side fault injection (no device fault): a
caller-supplied allocator that returns NULL makes the running call fail
with HC_ERR_OOM instead of aborting, and the context keeps working once the
allocator recovers, giving the oracle's words again."""
import numpy as np
import pytest

from oracle import ckks
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_allocator_returning_null_is_an_error_code():
    import torch

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    state = {"fail": False, "refused": 0}

    def _alloc(nbytes, strm, user):
        if state["fail"]:
            state["refused"] += 1
            return None
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream)
        except Exception:
            return None

    def _free(ptr, strm, user):
        torch.cuda.caching_allocator_delete(ptr)

    a_fn, f_fn = H.ALLOC_FN(_alloc), H.FREE_FN(_free)
    log_n, qb, pb, ls, seed = 10, [60, 40, 40], [60], 40, 21
    op = ckks.Params(log_n, qb, pb, ls)
    ctx = H.hc_ctx_create(H.hc_params_create(log_n, qb, pb, ls), 0, stream.cuda_stream,
                          (H.Allocator(a_fn, f_fn, None), (a_fn, f_fn)))
    sk, pk, evk = H.hc_keygen(ctx, seed)
    o_sk, o_pk, o_evk = ckks.keygen(op, seed)
    cts = []
    for nonce in (1, 2):
        m = W.int_plaintext(30 + nonce, op.N, 2 ** 35)
        cts.append((H.hc_encrypt(ctx, pk, H.hc_pt_from_coeffs(ctx, m, op.L, op.scale), seed + 1, nonce),
                    ckks.encrypt(op, o_pk, ckks.plaintext_from_ints(op, m, op.L, op.scale), seed + 1, nonce)))
    (ga, oa), (gb, ob) = cts
    want = ckks.rescale(op, ckks.relin(op, o_evk, ckks.mul(op, oa, ob)))

    state["fail"] = True
    with pytest.raises(H.HcError) as e:
        H.hc_mul_relin_rescale_batch(ctx, evk, [ga], [gb])
    assert e.value.code == -6  # HC_ERR_OOM
    assert state["refused"] >= 1

    state["fail"] = False
    got = H.hc_mul_relin_rescale_batch(ctx, evk, [ga], [gb])[0]
    data, meta = H.hc_ct_export(ctx, got)
    assert meta.level == want.level and np.array_equal(data, want.c)
