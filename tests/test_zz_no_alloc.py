"""The allocation-free relinearisation (hc_relin_noalloc).

Some callers of this library cannot allocate device memory while they run
its work: memory handed over once at start-up, or a serving loop that must
not enter an allocator.  hc_relin_noalloc takes its scratch from a static
device array and writes into an output ciphertext the caller allocated
beforehand.  These tests check its words against the oracle's relinearisation
and against hc_relin on two calls in a row, that it makes no allocator call
(the context's allocator refuses and counts every request during the call),
the level limits, and its error codes.  This file is collected last so that a
run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

from oracle import ckks
from paper_2102_00319_gb300 import hecnn as H
from paper_2102_00319_gb300 import workloads as W

pytestmark = pytest.mark.gpu


class _CountingAllocator:
    """A context allocator over torch's caching allocator that counts its
    calls and can be told to refuse (return NULL)."""

    def __init__(self, torch, stream):
        self.calls = 0
        self.refuse = False

        def _alloc(nbytes, strm, user):
            self.calls += 1
            if self.refuse:
                return None
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream)
            except Exception:
                return None

        def _free(ptr, strm, user):
            self.calls += 1
            torch.cuda.caching_allocator_delete(ptr)

        self._fns = (H.ALLOC_FN(_alloc), H.FREE_FN(_free))
        self.arg = (H.Allocator(self._fns[0], self._fns[1], None), self._fns)


def _setup(log_n, qb, pb, ls, seed, counting=False):
    import torch

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    alloc = _CountingAllocator(torch, stream) if counting else None
    gp = H.hc_params_create(log_n, qb, pb, ls)
    ctx = H.hc_ctx_create(gp, 0, stream.cuda_stream, alloc.arg if alloc else None)
    op = ckks.Params(log_n, qb, pb, ls)
    return ctx, H.hc_keygen(ctx, seed), op, ckks.keygen(op, seed), alloc


def _degree2_pair(ctx, pk, op, opk, level, seed, nonce):
    """The same degree-2 product on both sides: integer plaintexts encrypted
    from the same seeds, then the tensor product."""
    gs, os_ = [], []
    for k in range(2):
        m = W.int_plaintext(seed + 7 * k, op.N, 2 ** 30)
        gs.append(H.hc_encrypt(ctx, pk, H.hc_pt_from_coeffs(ctx, m, level, op.scale), seed, nonce + k))
        os_.append(ckks.encrypt(op, opk, ckks.plaintext_from_ints(op, m, level, op.scale), seed, nonce + k))
    return H.hc_mul(ctx, gs[0], gs[1]), ckks.mul(op, os_[0], os_[1])


def _empty_out(ctx, level):
    return H.hc_ct_import(ctx, np.zeros((2, level + 1, ctx.n), dtype=np.uint64), level, 1, 1.0)


def _check_level(ctx, keys, op, okeys, level, seed, calls=2, alloc=None):
    sk, pk, evk = keys
    osk, opk, oevk = okeys
    out = _empty_out(ctx, level)
    for call in range(calls):  # calls in a row share the scratch array
        d, od = _degree2_pair(ctx, pk, op, opk, level, seed + 100 * call, 2 * call + 1)
        want = ckks.relin(op, oevk, od)
        lib, _ = H.hc_ct_export(ctx, H.hc_relin(ctx, evk, d))
        H.hc_sync(ctx)
        if alloc is not None:
            before = alloc.calls
            alloc.refuse = True
        try:
            H.hc_relin_noalloc(ctx, evk, d, out)
            H.hc_sync(ctx)
        finally:
            if alloc is not None:
                alloc.refuse = False
        if alloc is not None:
            assert alloc.calls == before, "hc_relin_noalloc called the allocator %d times" % (alloc.calls - before)
        got, meta = H.hc_ct_export(ctx, out)
        assert meta.level == want.level == level and meta.degree == 1
        assert meta.scale == d.scale
        assert np.array_equal(got, want.c), "level %d call %d differs from the oracle" % (level, call)
        assert np.array_equal(got, lib), "level %d call %d differs from hc_relin" % (level, call)


def test_noalloc_matches_oracle_and_relin_twice_without_allocating():
    # N = 2^12, five q primes, two special primes: dnum = 3 with a ragged last
    # digit; the context allocator refuses and counts during every call
    ctx, keys, op, okeys, alloc = _setup(12, [60, 40, 40, 40, 40], [60, 60], 40, 31, counting=True)
    _check_level(ctx, keys, op, okeys, 4, 100, alloc=alloc)
    # a lower level (fewer digits) after the larger one reuses the array
    _check_level(ctx, keys, op, okeys, 2, 300, calls=1, alloc=alloc)


def test_noalloc_more_than_eight_digits():
    # one special prime: one digit per q prime, ten digits at the top level
    # (hc_relin copies the digits' own limbs into the raised basis there)
    ctx, keys, op, okeys, _ = _setup(12, [60] + [40] * 9, [60], 40, 33)
    _check_level(ctx, keys, op, okeys, 9, 500)


def test_noalloc_n14_largest_level_that_fits():
    # N = 2^14, one special prime: a key switch at level l needs
    # 512 + (l + 1)^2 + 6 (l + 1) + 2 limbs of scratch (in units of N words),
    # so level 7 (114 N words + 512) is the largest within 2^21 words and
    # level 8 (137 N words) is rejected
    ctx, keys, op, okeys, _ = _setup(14, [60] + [40] * 9, [60], 40, 34)
    _check_level(ctx, keys, op, okeys, 7, 700)
    sk, pk, evk = keys
    d, _ = _degree2_pair(ctx, pk, op, okeys[1], 8, 800, 1)
    with pytest.raises(H.HcError) as e:
        H.hc_relin_noalloc(ctx, evk, d, _empty_out(ctx, 8))
    assert e.value.code == -1 and "scratch" in str(e.value)


def test_noalloc_rejects_oversize_and_bad_output():
    # 24 q primes at N = 2^14 need more scratch than the static array holds
    ctx, keys, op, okeys, _ = _setup(14, [40] * 24, [40] * 4, 30, 32)
    sk, pk, evk = keys
    pt = H.hc_encode(ctx, W.slot_values(1, ctx.n // 2), 2.0 ** 30, 23)
    a = H.hc_encrypt(ctx, pk, pt, 1, 0)
    d = H.hc_mul(ctx, a, a)
    with pytest.raises(H.HcError) as e:
        H.hc_relin_noalloc(ctx, evk, d, _empty_out(ctx, 23))
    assert e.value.code == -1 and "scratch" in str(e.value)
    with pytest.raises(H.HcError) as e:
        H.hc_relin_noalloc(ctx, evk, d, _empty_out(ctx, 22))
    assert e.value.code == -2  # HC_ERR_LEVEL_MISMATCH
    # a degree-1 input is not a relinearisation input
    with pytest.raises(H.HcError) as e:
        H.hc_relin_noalloc(ctx, evk, a, _empty_out(ctx, 23))
    assert e.value.code == -1
