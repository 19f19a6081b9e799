"""The algebra of the library's key switch, restated on the CPU against the
oracle's plain relinearise + rescale (no GPU).

The library does not compute ModDown as written in the scheme
((u - FastBConv_{P->Q}([u]_P)) P^{-1}): it stores the switching keys' limbs
of Q multiplied by P^{-1} (so the key product's Q limbs come out divided),
converts [u]_P with the constants p_k^{-1} mod q_i instead of (P/p_k) mod q_i
(so the conversion comes out divided too), and lets the rescale ride on the
same pass: out_k[i] = (d_k[i] + u'_k[i] - z'_k[i] - [c_l]_{q_i}) q_l^{-1}
with c_l the centred last limb of d_k + u'_k - z'_k.  This test restates
that sequence with exact integers and checks it word for word against
rescale(relin(d)) of the oracle, for every level and both key digits'
shapes (full and truncated)."""
import numpy as np
import pytest

from oracle import ckks


def folded_relin_rescale(op, evk, d):
    l = d.level
    nq, L, alpha, n = l + 1, op.L, op.alpha, op.N
    ext = op.ext_indices(l)
    chain = [int(v) for v in op.chain]
    p_idx = list(range(L + 1, L + 1 + alpha))
    P = 1
    for k in p_idx:
        P *= chain[k]
    # keys as the library stores them (the Montgomery factor 2^64 cancels in
    # its reduction and is left out here): Q limbs times P^{-1}
    def stored(key):
        out = key[ext].copy()
        for r, t in enumerate(ext):
            if t <= L:
                f = pow(P % chain[t], -1, chain[t])
                out[r] = ckks.pscalar(out[r][None], np.array([f], dtype=np.uint64),
                                      np.array([chain[t]], dtype=np.uint64))[0]
        return out

    primes = ckks.primes_of(op, ext)
    ys = ckks.modup(op, d.c[2], l)  # the raised digits: unchanged by the folds
    u = []
    for keys in (evk.relin.b, evk.relin.a):
        acc = np.zeros((len(ext), n), dtype=np.uint64)
        for j, y in enumerate(ys):
            acc = ckks.padd(acc, ckks.pmul(y, stored(keys[j]), primes), primes)
        u.append(acc)
    out = np.empty((2, l, n), dtype=np.uint64)
    ql = chain[l]
    for k in range(2):
        # the P limbs of u convert with p_k^{-1} mod q_i: z' = FastBConv([u]_P) P^{-1}
        up = [[int(v) for v in u[k][nq + m]] for m in range(alpha)]
        zq = np.zeros((nq, n), dtype=object)
        for i in range(nq):
            qi = chain[i]
            for c in range(n):
                s = 0
                for m, kp in enumerate(p_idx):
                    pk = chain[kp]
                    hinv = pow((P // pk) % pk, -1, pk)
                    s += (up[m][c] * hinv % pk) * pow(pk % qi, -1, qi)
                zq[i, c] = s % qi
        relin = np.zeros((nq, n), dtype=object)
        for i in range(nq):
            qi = chain[i]
            for c in range(n):
                relin[i, c] = (int(d.c[k][i][c]) + int(u[k][i][c]) - zq[i, c]) % qi
        for i in range(l):
            qi = chain[i]
            qinv = pow(ql % qi, -1, qi)
            for c in range(n):
                cl = relin[l, c]
                cl = cl - ql if cl > (ql - 1) // 2 else cl  # centred
                out[k, i, c] = (relin[i, c] - cl) * qinv % qi
    return out


@pytest.mark.parametrize("q_bits,p_bits", [([40, 30, 30, 30, 30], [40, 40]), ([50, 30, 30], [50])])
def test_folded_keyswitch_rescale_equals_the_scheme(q_bits, p_bits):
    op = ckks.Params(5, q_bits, p_bits, 25)
    sk, pk, evk = ckks.keygen(op, 31)
    rng = np.random.default_rng(5)
    for level in range(op.L, 0, -1):
        m = [rng.integers(-(1 << 20), 1 << 20, op.N) for _ in range(2)]
        a, b = (ckks.encrypt(op, pk, ckks.plaintext_from_ints(op, mi, level, op.scale), 32, 10 * level + t)
                for t, mi in enumerate(m))
        d = ckks.mul(op, a, b)
        want = ckks.rescale(op, ckks.relin(op, evk, d))
        got = folded_relin_rescale(op, evk, d)
        assert np.array_equal(got, want.c), level
