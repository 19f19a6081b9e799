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


@pytest.mark.parametrize("logn", [13, 14, 15, 16])
def test_pipelined_passes_index_arithmetic(logn):
    """The pipelined passes (tuning variant 5, 128-thread CTAs): the 16-byte
    asynchronous copies of a tile land on 16-byte-aligned shared-memory
    words inside the buffer and cover the tile once; both register rounds
    read and write exactly the staged words; the global reads and writes of
    a tile stay inside its limb; two buffers fit in 48 KB."""
    n1 = logn // 2
    n2 = logn - n1
    # column pass: rows of TC words, each group of 2^K2 rows shifted by 8 words
    k1, k2, _ = split(n1)
    tcl = col_tile(n1, n2, 7)
    tc = 1 << tcl
    tile = (1 << (n1 + tcl)) + (8 << k1)

    def sidx(row, c):
        return (row << tcl) + c + ((row >> k2) << 3)

    tiles_x = 1 << (n2 - tcl)
    staged, gmax = set(), 0
    for ch in range((1 << (n1 + tcl)) // 2):
        row, c = ch >> (tcl - 1), (ch & ((tc >> 1) - 1)) << 1
        d = sidx(row, c)
        assert d % 2 == 0 and d + 1 < tile and sidx(row, c + 1) == d + 1
        staged.update((d, d + 1))
        gmax = max(gmax, (tiles_x - 1) * tc + (row << n2) + c + 1)
    assert gmax < (1 << logn) and len(staged) == (1 << n1) * tc
    strided, adjacent, out = set(), set(), set()
    for w in range(tc << k2):
        c, r0 = w & (tc - 1), w >> tcl
        strided.update(sidx(r0 + (i << k2), c) for i in range(1 << k1))
    for w in range(tc << k1):
        c, g = w & (tc - 1), w >> tcl
        for i in range(1 << k2):
            adjacent.add(sidx((g << k2) + i, c))
            out.add((((g << k2) + i) << n2) + c)
    assert strided == adjacent == staged
    assert len(out) == (1 << n1) * tc and max(out) + (tiles_x - 1) * tc < (1 << logn)
    assert 2 * tile * 8 <= SMEM_LIMIT
    # row pass: RP rows of C words, two words of padding per 2^K2
    k1, k2, _ = split(n2)
    rpl, _ = row_tile(n1, n2, 7)
    rp, c_ = 1 << rpl, 1 << n2
    padw = c_ + (c_ >> (k2 - 1))

    def sidr(r, j):
        return r * padw + j + ((j >> k2) << 1)

    staged = set()
    for ch in range((rp << n2) // 2):
        e = ch << 1
        r, j = e >> n2, e & (c_ - 1)
        d = sidr(r, j)
        assert d % 2 == 0 and d + 1 < rp * padw and sidr(r, j + 1) == d + 1
        staged.update((d, d + 1))
    assert len(staged) == rp * c_
    strided, adjacent = set(), set()
    for w in range(rp << k2):
        r, r0 = w >> k2, w & ((1 << k2) - 1)
        strided.update(sidr(r, r0 + (i << k2)) for i in range(1 << k1))
    for w in range(rp << k1):
        r, g = w >> k1, w & ((1 << k1) - 1)
        base = sidr(r, g << k2)
        assert base % 2 == 0 and all(sidr(r, (g << k2) + i) == base + i for i in range(1 << k2))
        adjacent.update(base + i for i in range(1 << k2))
    assert strided == adjacent == staged
    assert (1 << (n1 - rpl)) * rp * c_ == 1 << logn
    assert 2 * rp * padw * 8 <= SMEM_LIMIT
