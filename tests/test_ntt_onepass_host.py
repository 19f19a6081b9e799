"""CPU replay of the single-pass NTT kernel (k_ntt_onepass in csrc/hc_ntt.cu):
one limb of N = CL 2^LQ points over a cluster of CL CTAs, each holding a
chunk of 2^LQ words in padded shared memory (index i at i + i / 16), in
both forms: 2^14-word chunks on 512 threads with rounds of up to 5 stages,
and 2^13-word chunks on 256 threads with rounds of up to 4 (clusters of up
to 8).

Replayed exactly as the kernel indexes: the cross-CTA stages (forward:
CTA r takes offsets j in [r Q / CL, (r+1) Q / CL), loads the CL points
j + k Q, runs stages 0..C-1, stores point k into CTA k's chunk at j;
inverse: the reverse, reading the peers' chunks), then the chunk's local
register rounds (group g: local index ((g >> LS) << (LS + K)) + (g mod 2^LS)
+ (m << LS), LS = LQ - S0 - K).  Checked: every shared-memory index stays
inside the padded chunk, every cross-CTA store lands on a distinct word and
fills every chunk, every round touches each local index exactly once, the
thread loops cover their work exactly (512 threads), and the results are
the negacyclic evaluation (forward, against the definition at sampled
slots and against the two-pass replay everywhere) and its inverse, inside
the lazy bounds the butterflies assume."""
import random

import pytest

from test_modular_bounds_host import largest_prime, shoup_lazy, shoup_of
from test_ntt_replay_host import Replay, brv

ROUNDS = {  # (LQ, WIDE) -> [(S0, K)], forward order, as OnePassRounds
    (14, 1): [(0, 5), (5, 5), (10, 4)],
    (14, 0): [(0, 4), (4, 4), (8, 3), (11, 3)],
    (13, 1): [(0, 5), (5, 4), (9, 4)],
    (13, 0): [(0, 4), (4, 3), (7, 3), (10, 3)],
}


def opad(i):
    return i + (i >> 4)


def form(logn, chunk14):
    """(LQ, threads, WIDE) of launch_onepass<INV, LOGN, CHUNK14>."""
    lq = 14 if (chunk14 and logn >= 14) else 13
    return lq, (512 if chunk14 else 256), (1 if chunk14 else 0)


def check_round_geometry(LQ, S0, K, THREADS):
    LS = LQ - S0 - K
    groups = 1 << (LQ - K)
    # the kernel's thread loop: g = threadIdx.x, += 512, while g < groups
    per_thread = [list(range(t, groups, THREADS)) for t in range(THREADS)]
    assert sorted(sum(per_thread, [])) == list(range(groups))
    seen = []
    for g in range(groups):
        lo, hi = g & ((1 << LS) - 1), g >> LS
        i0 = (hi << (LS + K)) + lo
        seen += [i0 + (m << LS) for m in range(1 << K)]
    assert sorted(seen) == list(range(1 << LQ))
    assert max(opad(i) for i in seen) < (1 << LQ) + (1 << (LQ - 4))


@pytest.mark.parametrize("logn,chunk14", [(l, c) for l in (13, 14, 15, 16) for c in (0, 1)])
def test_round_schedules_cover_the_chunk(logn, chunk14):
    LQ, threads, wide = form(logn, chunk14)
    cl = 1 << (logn - LQ)
    assert cl <= 8  # portable cluster size
    if cl > 1:
        assert ((1 << LQ) // cl) % threads == 0  # cross-CTA offsets per thread
    rounds = ROUNDS[(LQ, wide)]
    assert sum(k for _, k in rounds) == LQ
    s = 0
    for S0, K in rounds:
        assert S0 == s and 1 <= K <= 5
        s += K
        check_round_geometry(LQ, S0, K, threads)


class OnePass(Replay):
    """Replay of k_ntt_onepass<INV, LOGN, LQ, WIDE> for one limb."""

    def __init__(self, logn, q, chunk14):
        super().__init__(logn, 7, q)
        self.LQ, self.threads, wide = form(logn, chunk14)
        self.C = logn - self.LQ
        self.CL = 1 << self.C
        self.Q = 1 << self.LQ
        self.padq = self.Q + (self.Q >> 4)
        self.rounds = ROUNDS[(self.LQ, wide)]

    def _local(self, sm, r, inverse):
        rounds = list(reversed(self.rounds)) if inverse else self.rounds
        for S0, K in rounds:
            LS = self.LQ - S0 - K
            for g in range(1 << (self.LQ - K)):
                lo, hi = g & ((1 << LS) - 1), g >> LS
                i0 = (hi << (LS + K)) + lo
                jb = (r << self.LQ) + i0
                idx = [opad(i0 + (m << LS)) for m in range(1 << K)]
                x = [sm[i] for i in idx]
                if inverse:
                    self.inv_block(x, K, LS, self.C + S0 + K - 1, jb)
                else:
                    self.fwd_block(x, K, LS, self.C + S0, jb)
                for i, v in zip(idx, x):
                    sm[i] = v

    def forward(self, a):
        q, Q, CL, LQ = self.q, self.Q, self.CL, self.LQ
        sms = [[None] * self.padq for _ in range(CL)]
        if CL > 1:
            kJ = Q // CL
            assert kJ % self.threads == 0
            for r in range(CL):
                for t in range(kJ):
                    j = r * kJ + t
                    x = [a[j + (k << LQ)] for k in range(CL)]
                    self.fwd_block(x, self.C, LQ, 0, j)
                    for k in range(CL):
                        assert sms[k][opad(j)] is None, "two stores to one word"
                        sms[k][opad(j)] = x[k]
            for sm in sms:  # every chunk is complete before its local stages
                assert all(sm[opad(e)] is not None for e in range(Q))
        else:
            for e in range(Q):
                sms[0][opad(e)] = a[e]
        out = [None] * self.n
        for r in range(CL):
            self._local(sms[r], r, False)
            for e in range(Q):
                out[(r << LQ) + e] = self.reduce4(sms[r][opad(e)], q)
        return out

    def inverse(self, a, scale=True):
        q, Q, CL, LQ = self.q, self.Q, self.CL, self.LQ
        sms = [[None] * self.padq for _ in range(CL)]
        for r in range(CL):
            for e in range(Q):
                sms[r][opad(e)] = a[(r << LQ) + e]
            self._local(sms[r], r, True)
        ni, nis = self.ninv, shoup_of(self.ninv, q)
        out = [None] * self.n
        if CL > 1:
            kJ = Q // CL
            for r in range(CL):
                for t in range(kJ):
                    j = r * kJ + t
                    x = [sms[k][opad(j)] for k in range(CL)]
                    self.inv_block(x, self.C, LQ, self.C - 1, j)
                    for k in range(CL):
                        v = shoup_lazy(x[k], ni, nis, q) if scale else x[k]
                        assert out[j + (k << LQ)] is None
                        out[j + (k << LQ)] = self.reduce4(v, q)
        else:
            for e in range(Q):
                v = shoup_lazy(sms[0][opad(e)], ni, nis, q) if scale else sms[0][opad(e)]
                out[e] = self.reduce4(v, q)
        assert None not in out
        return out


@pytest.mark.parametrize("logn,chunk14,bits", [(13, 1, 60), (13, 0, 40), (14, 1, 50), (14, 0, 61), (15, 1, 60),
                                               (15, 0, 50), (16, 1, 50), (16, 0, 60)])
def test_onepass_forward_and_inverse(logn, chunk14, bits):
    q = largest_prime(bits, 2 << logn)
    R = OnePass(logn, q, chunk14)
    rng = random.Random(logn * 10 + chunk14)
    a = [rng.randrange(q) for _ in range(R.n)]
    a[0], a[-1] = q - 1, q - 1
    got = R.forward(a)
    for k in rng.sample(range(R.n), 6) + [0, R.n - 1]:
        x = pow(R.psi, 2 * brv(k, logn) + 1, q)
        want = 0
        for c in reversed(a):
            want = (want * x + c) % q
        assert got[k] == want, k
    assert got == Replay.forward(R, a)  # the two-pass kernels' words
    assert R.inverse(got) == a
    assert R.inverse(got, scale=False) == [v * R.n % q for v in a]
