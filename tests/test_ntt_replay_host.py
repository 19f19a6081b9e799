"""CPU replay of the NTT kernels' arithmetic (no GPU): the column and row
passes of csrc/hc_ntt.cu -- their register rounds, shared-memory exchange,
twiddle indexing (pair (j, j + t) of stage st uses table entry
2^st + (j >> (log N - st))) and Harvey's lazy butterflies with Shoup
products -- restated step by step in Python integers with 64-bit wrap, on
the tables the library builds (psi^{brv(k)} and psi^{-brv(k)}).  The forward
result must be the evaluation of the polynomial at psi^{2 brv(k) + 1} in
slot k (the definition, computed directly), the inverse must give the
coefficients back, and every intermediate value must stay inside the lazy
bound its butterfly assumes ([0, 4q) forward, [0, 2q) inverse)."""
import random

import pytest

from test_modular_bounds_host import M64, largest_prime, shoup_lazy, shoup_of
from test_ntt_tiling_host import col_tile, row_tile, split


def brv(k, bits):
    return int(format(k, "0%db" % bits)[::-1], 2) if bits else 0


def primitive_2n_root(logn, q):
    n = 1 << logn
    for g in range(2, 10000):
        psi = pow(g, (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            return psi
    raise AssertionError("no root")


class Replay:
    def __init__(self, logn, tl, q):
        self.logn, self.tl, self.q, self.n = logn, tl, q, 1 << logn
        psi = primitive_2n_root(logn, q)
        ipsi = pow(psi, -1, q)
        self.psi = psi
        self.fwd = [pow(psi, brv(k, logn), q) for k in range(self.n)]
        self.inv = [pow(ipsi, brv(k, logn), q) for k in range(self.n)]
        self.ninv = pow(self.n, -1, q)

    def tw(self, table, idx):
        w = table[idx]
        return w, shoup_of(w, self.q)

    def fwd_block(self, x, K, LS, ST0, jb):
        q, L = self.q, self.logn
        for s in range(K):
            st = ST0 + s
            half = 1 << (K - 1 - s)
            base = (1 << st) + (jb >> (L - st))
            for i in range(1 << K):
                if i & half:
                    continue
                w, wsh = self.tw(self.fwd, base + ((i << LS) >> (L - st)))
                X = x[i]
                assert X < 4 * q and x[i + half] < 4 * q
                X = X - 2 * q if X >= 2 * q else X
                T = shoup_lazy(x[i + half], w, wsh, q)
                x[i] = (X + T) & M64
                x[i + half] = (X - T + 2 * q) & M64

    def inv_block(self, x, K, LS, STH, jb):
        q, L = self.q, self.logn
        for s in range(K):
            st = STH - s
            half = 1 << s
            base = (1 << st) + (jb >> (L - st))
            for i in range(1 << K):
                if i & half:
                    continue
                w, wsh = self.tw(self.inv, base + ((i << LS) >> (L - st)))
                U, V = x[i], x[i + half]
                assert U < 2 * q and V < 2 * q
                S = U + V
                x[i] = S - 2 * q if S >= 2 * q else S
                x[i + half] = shoup_lazy((U - V + 2 * q) & M64, w, wsh, q)

    @staticmethod
    def reduce4(x, q):
        x = x - 2 * q if x >= 2 * q else x
        return x - q if x >= q else x

    def geometry(self):
        n1 = self.logn // 2
        n2 = self.logn - n1
        return n1, n2

    def forward(self, a):
        a, q = list(a), self.q
        n1, n2 = self.geometry()
        # column pass: stages 0 .. n1-1
        k1, k2, _ = split(n1)
        tcl = col_tile(n1, n2, self.tl)
        tc = 1 << tcl
        for bx in range(1 << (n2 - tcl)):
            b0 = bx * tc
            sm = {}
            for w in range(tc << k2):
                c, r0 = w & (tc - 1), w >> tcl
                x = [a[b0 + ((r0 + (i << k2)) << n2) + c] for i in range(1 << k1)]
                self.fwd_block(x, k1, k2 + n2, 0, r0 << n2)
                for i in range(1 << k1):
                    sm[((r0 + (i << k2)) << tcl) + c] = x[i]
            for w in range(tc << k1):
                c, g = w & (tc - 1), w >> tcl
                x = [sm[(((g << k2) + i) << tcl) + c] for i in range(1 << k2)]
                self.fwd_block(x, k2, n2, k1, (g << k2) << n2)
                for i in range(1 << k2):
                    a[b0 + ((((g << k2) + i) << n2) + c)] = self.reduce4(x[i], q)
        # row pass: stages n1 .. log N - 1
        k1, k2, _ = split(n2)
        rpl, padw = row_tile(n1, n2, self.tl)
        rp = 1 << rpl

        def sidx(r, j):
            return r * padw + j + (j >> k2)

        for bx in range(1 << (n1 - rpl)):
            row0 = bx * rp
            sm = {}
            for w in range(rp << k2):
                r, r0 = w >> k2, w & ((1 << k2) - 1)
                x = [a[((row0 + r) << n2) + r0 + (i << k2)] for i in range(1 << k1)]
                self.fwd_block(x, k1, k2, n1, ((row0 + r) << n2) + r0)
                for i in range(1 << k1):
                    sm[sidx(r, r0 + (i << k2))] = x[i]
            for w in range(rp << k1):
                r, g = w >> k1, w & ((1 << k1) - 1)
                x = [sm[sidx(r, (g << k2) + i)] for i in range(1 << k2)]
                self.fwd_block(x, k2, 0, n1 + k1, ((row0 + r) << n2) + (g << k2))
                for i in range(1 << k2):
                    sm[sidx(r, (g << k2) + i)] = self.reduce4(x[i], q)
            for e in range(rp << n2):
                a[(row0 << n2) + e] = sm[sidx(e >> n2, e & ((1 << n2) - 1))]
        return a

    def inverse(self, a, scale=True):
        a, q, L = list(a), self.q, self.logn
        n1, n2 = self.geometry()
        # row pass first: stages log N - 1 .. n1
        k1, k2, _ = split(n2)
        rpl, padw = row_tile(n1, n2, self.tl)
        rp = 1 << rpl

        def sidx(r, j):
            return r * padw + j + (j >> k2)

        for bx in range(1 << (n1 - rpl)):
            row0 = bx * rp
            sm = {}
            for w in range(rp << k1):
                r, g = w >> k1, w & ((1 << k1) - 1)
                x = [a[((row0 + r) << n2) + (g << k2) + i] for i in range(1 << k2)]
                self.inv_block(x, k2, 0, L - 1, ((row0 + r) << n2) + (g << k2))
                for i in range(1 << k2):
                    sm[sidx(r, (g << k2) + i)] = x[i]
            for w in range(rp << k2):
                r, r0 = w >> k2, w & ((1 << k2) - 1)
                x = [sm[sidx(r, r0 + (i << k2))] for i in range(1 << k1)]
                self.inv_block(x, k1, k2, L - 1 - k2, ((row0 + r) << n2) + r0)
                for i in range(1 << k1):
                    a[((row0 + r) << n2) + r0 + (i << k2)] = self.reduce4(x[i], q)
        # column pass: stages n1 - 1 .. 0, then N^{-1}
        k1, k2, _ = split(n1)
        tcl = col_tile(n1, n2, self.tl)
        tc = 1 << tcl
        ni, nis = self.ninv, shoup_of(self.ninv, q)
        for bx in range(1 << (n2 - tcl)):
            b0 = bx * tc
            sm = {}
            for w in range(tc << k1):
                c, g = w & (tc - 1), w >> tcl
                x = [a[b0 + ((((g << k2) + i) << n2) + c)] for i in range(1 << k2)]
                self.inv_block(x, k2, n2, n1 - 1, (g << k2) << n2)
                for i in range(1 << k2):
                    sm[(((g << k2) + i) << tcl) + c] = x[i]
            for w in range(tc << k2):
                c, r0 = w & (tc - 1), w >> tcl
                x = [sm[((r0 + (i << k2)) << tcl) + c] for i in range(1 << k1)]
                self.inv_block(x, k1, k2 + n2, k1 - 1, r0 << n2)
                for i in range(1 << k1):
                    v = shoup_lazy(x[i], ni, nis, q) if scale else x[i]
                    a[b0 + ((r0 + (i << k2)) << n2) + c] = self.reduce4(v, q)
        return a


CASES = [(10, 7, 60), (10, 8, 30), (11, 7, 50), (12, 8, 61), (13, 6, 40)]


@pytest.mark.parametrize("logn,tl,bits", CASES)
def test_forward_pass_pair_is_the_negacyclic_evaluation(logn, tl, bits):
    q = largest_prime(bits, 2 << logn)
    R = Replay(logn, tl, q)
    rng = random.Random(logn * 100 + tl)
    a = [rng.randrange(q) for _ in range(R.n)]
    a[0], a[-1] = q - 1, q - 1
    got = R.forward(a)
    for k in rng.sample(range(R.n), 24) + [0, R.n - 1]:
        x = pow(R.psi, 2 * brv(k, logn) + 1, q)
        want = 0
        for c in reversed(a):
            want = (want * x + c) % q
        assert got[k] == want, k


@pytest.mark.parametrize("logn,tl,bits", CASES)
def test_inverse_pass_pair_returns_the_coefficients(logn, tl, bits):
    q = largest_prime(bits, 2 << logn)
    R = Replay(logn, tl, q)
    rng = random.Random(logn * 7 + tl)
    a = [rng.randrange(q) for _ in range(R.n)]
    assert R.inverse(R.forward(a)) == a
    # without N^{-1} the inverse gives N times the coefficients
    assert R.inverse(R.forward(a), scale=False) == [v * R.n % q for v in a]


@pytest.mark.parametrize("logn,g_steps", [(10, 1), (10, 3), (11, -1), (12, 17)])
def test_automorphism_index_map_in_the_transform_domain(logn, g_steps):
    """k_automorph permutes NTT slots: slot k holds a(psi^{e_k}) with
    e_k = 2 brv(k) + 1, and kappa_g(a)(psi^e) = a(psi^{e g}), so output slot
    k reads input slot brv((e_k g mod 2N - 1) / 2).  Replayed on the
    transform above, it must equal the transform of X -> X^g applied to the
    coefficients (with the negacyclic sign)."""
    q = largest_prime(50, 2 << logn)
    R = Replay(logn, 7, q)
    n = R.n
    g = pow(5, g_steps % (n // 2), 2 * n) if g_steps >= 0 else 2 * n - 1  # a rotation, or conjugation
    rng = random.Random(logn + g)
    a = [rng.randrange(q) for _ in range(n)]
    kappa = [0] * n
    for i, c in enumerate(a):
        e = i * g % (2 * n)
        if e < n:
            kappa[e] = (kappa[e] + c) % q
        else:
            kappa[e - n] = (kappa[e - n] - c) % q
    fa = R.forward(a)
    moved = []
    for k in range(n):
        e = 2 * brv(k, logn) + 1
        e2 = e * g % (2 * n)
        moved.append(fa[brv((e2 - 1) // 2, logn)])
    assert moved == R.forward(kappa)
