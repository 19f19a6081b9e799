"""CPU check of the NTT passes' index arithmetic (no GPU): for every ring
degree and block size the library dispatches, the tile parameters chosen in
csrc/hc_ntt.cu (Split, ColTile, RowTile) and the per-thread index formulas
of the column and row passes are replayed on the host.  Each pass must read
and write every coefficient of a limb exactly once, keep every shared-memory
index inside the block's allocation (at most 48 KB), keep the 16-byte vector
accesses aligned, and split the fused-tail epilogue evenly over the threads.
The formulas are restated here from the kernels; a change to the tiling must
change both."""
import numpy as np
import pytest

SMEM_LIMIT = 48 * 1024


def split(n):
    k1 = 3 if n in (5, 6) else 4
    return k1, n - k1, min(k1, n - k1)


def col_tile(n1, n2, tl):
    raw = min(tl - split(n1)[2], n2)
    return raw - 1 if (1 << (n1 + raw)) * 8 > SMEM_LIMIT else raw


def row_tile(n1, n2, tl):
    k2 = split(n2)[1]
    padw = (1 << n2) + (1 << (n2 - k2))
    raw = min(tl - split(n2)[2], n1)
    rpl = raw - 1 if (1 << raw) * padw * 8 > SMEM_LIMIT else raw
    return rpl, padw


def variants():
    for logn in range(10, 17):
        for tl in ((8, 7, 6) if logn >= 13 else (8, 7)):
            yield logn, tl


@pytest.mark.parametrize("logn,tl", list(variants()))
def test_column_pass_covers_each_coefficient_once(logn, tl):
    n1 = logn // 2
    n2 = logn - n1
    k1, k2, _ = split(n1)
    tcl = col_tile(n1, n2, tl)
    tc, threads = 1 << tcl, 1 << tl
    smem_words = 1 << (n1 + tcl)
    assert smem_words * 8 <= SMEM_LIMIT
    reads = np.zeros(1 << logn, dtype=np.int64)
    writes = np.zeros(1 << logn, dtype=np.int64)
    for bx in range(1 << (n2 - tcl)):
        sm_w1 = np.zeros(smem_words, dtype=np.int64)
        sm_r2 = np.zeros(smem_words, dtype=np.int64)
        # first register round: 2^K1 rows strided by 2^K2
        for t in range(threads):
            for w in range(t, tc << k2, threads):
                c, r0 = w & (tc - 1), w >> tcl
                for i in range(1 << k1):
                    e = ((r0 + (i << k2)) << n2) + c
                    reads[bx * tc + e] += 1
                    s = ((r0 + (i << k2)) << tcl) + c
                    assert 0 <= s < smem_words
                    sm_w1[s] += 1
        # second register round: 2^K2 adjacent rows
        for t in range(threads):
            for w in range(t, tc << k1, threads):
                c, g = w & (tc - 1), w >> tcl
                for i in range(1 << k2):
                    s = (((g << k2) + i) << tcl) + c
                    assert 0 <= s < smem_words
                    sm_r2[s] += 1
                    writes[bx * tc + ((((g << k2) + i) << n2) + c)] += 1
        assert np.all(sm_w1 == 1) and np.all(sm_r2 == 1)
    assert np.all(reads == 1) and np.all(writes == 1)


@pytest.mark.parametrize("logn,tl", list(variants()))
def test_row_pass_covers_each_coefficient_once(logn, tl):
    n1 = logn // 2
    n2 = logn - n1
    k1, k2, _ = split(n2)
    rpl, padw = row_tile(n1, n2, tl)
    rp, c_len, threads = 1 << rpl, 1 << n2, 1 << tl
    smem_words = rp * padw
    assert smem_words * 8 <= SMEM_LIMIT

    def sidx(r, j):
        return r * padw + j + (j >> k2)

    reads = np.zeros(1 << logn, dtype=np.int64)
    writes = np.zeros(1 << logn, dtype=np.int64)
    for bx in range(1 << (n1 - rpl)):
        row0 = bx * rp
        sm_w = np.zeros(smem_words, dtype=np.int64)
        sm_r = np.zeros(smem_words, dtype=np.int64)
        for t in range(threads):
            # first register round (forward): 2^K1 points strided by 2^K2, from global
            for w in range(t, rp << k2, threads):
                r, r0 = w >> k2, w & ((1 << k2) - 1)
                for i in range(1 << k1):
                    reads[((row0 + r) << n2) + r0 + (i << k2)] += 1
                    s = sidx(r, r0 + (i << k2))
                    assert 0 <= s < smem_words
                    sm_w[s] += 1
            # inverse first round: 2^K2 adjacent points as 16-byte pairs
            for w in range(t, rp << k1, threads):
                r, g = w >> k1, w & ((1 << k1) - 1)
                assert ((r << n2) + (g << k2)) % 2 == 0
            # second register round: 2^K2 adjacent points through shared memory
            for w in range(t, rp << k1, threads):
                r, g = w >> k1, w & ((1 << k1) - 1)
                for i in range(1 << k2):
                    s = sidx(r, (g << k2) + i)
                    assert 0 <= s < smem_words
                    sm_r[s] += 1
        # the store back to global memory, row-contiguous across the block
        for e in range(rp << n2):
            assert 0 <= sidx(e >> n2, e & (c_len - 1)) < smem_words
            writes[(row0 << n2) + e] += 1
        used = sm_w > 0
        assert np.all(sm_w[used] == 1) and np.array_equal(sm_w > 0, sm_r > 0) and np.all(sm_r[used] == 1)
        # fused-tail epilogue: kU elements per thread per step, an even split
        k_tile = rp << n2
        k_u = 4
        assert k_tile % (threads * k_u) == 0
    assert np.all(reads == 1) and np.all(writes == 1)
