"""Test helper: one parameter set instantiated on both sides (GPU library
through its C ABI, CPU oracle), with the same seeds.  Inputs flow from the
seeded generators (and the oracle's encoder) into both sides; nothing flows
from the GPU into the oracle."""
import numpy as np

from oracle import ckks, encoding
from paper_2102_00319_gb300 import hecnn as H


class Pair:
    def __init__(self, log_n, q_bits, p_bits, log2_scale, seed, rot_steps=(), stream=None):
        import torch

        self.op = ckks.Params(log_n, list(q_bits), list(p_bits), log2_scale)
        self.gp = H.hc_params_create(log_n, list(q_bits), list(p_bits), log2_scale)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.ctx = H.hc_ctx_create(self.gp, 0, stream)
        self.seed = seed
        self.rot_steps = list(rot_steps)
        self.g_sk, self.g_pk, self.g_evk = H.hc_keygen(self.ctx, seed, self.rot_steps)
        self.o_sk, self.o_pk, self.o_evk = ckks.keygen(self.op, seed, self.rot_steps)

    # ---- inputs ------------------------------------------------------
    def encode_int(self, values):
        """Integer plaintext of a slot vector, by the oracle's encoder."""
        return encoding.encode(values, self.op.N, self.op.scale)

    def encrypt(self, m_int, level=None, nonce=0, scale=None, enc_seed=None):
        """Encrypts the same integer plaintext on both sides."""
        lv = self.op.L if level is None else level
        sc = self.op.scale if scale is None else scale
        es = self.seed + 1 if enc_seed is None else enc_seed
        opt = ckks.plaintext_from_ints(self.op, m_int, lv, sc)
        octx = ckks.encrypt(self.op, self.o_pk, opt, es, nonce)
        gpt = H.hc_pt_from_coeffs(self.ctx, m_int, lv, sc)
        gct = H.hc_encrypt(self.ctx, self.g_pk, gpt, es, nonce)
        return gct, octx

    def encrypt_values(self, values, level=None, nonce=0):
        return self.encrypt(self.encode_int(values), level, nonce)

    # ---- comparison -------------------------------------------------
    def export(self, gct):
        data, meta = H.hc_ct_export(self.ctx, gct)
        return data, meta

    def assert_same(self, gct, octx, what=""):
        data, meta = self.export(gct)
        assert meta.level == octx.level, what
        assert meta.degree == octx.degree, what
        assert meta.scale == octx.scale, (what, meta.scale, octx.scale)
        assert data.shape == octx.c.shape, what
        if not np.array_equal(data, octx.c):
            bad = np.argwhere(data != octx.c)
            raise AssertionError("%s: %d of %d words differ, first at %s" % (what, len(bad), data.size, bad[:3].tolist()))

    def decrypt_gpu(self, gct):
        pt = H.hc_decrypt(self.ctx, self.g_sk, gct)
        return H.hc_decode(self.ctx, pt)

    def decrypt_oracle(self, octx):
        d = ckks.decrypt(self.op, self.o_sk, octx)
        return encoding.decode(d.m, self.op.q[: octx.level + 1], self.op.N, octx.scale)


# ---- oracle work in spawned worker processes ----------------------------
# (spawn, never fork, so that the children inherit no CUDA state)
_W = {}


def _oracle_worker_init(param_args, pk_b, pk_a):
    import os

    os.environ["OMP_NUM_THREADS"] = "1"
    _W["op"] = ckks.Params(*param_args)
    _W["pk"] = ckks.PublicKey(pk_b, pk_a)


def oracle_tensor_partial(job):
    """sum_k x_k (x) w_k by the oracle over the terms of `job`, each term a
    pair of (integer-plaintext seed, bound, level, encryption seed, nonce)
    specs encrypted by the oracle itself."""
    from paper_2102_00319_gb300 import workloads as W

    op, pk = _W["op"], _W["pk"]
    acc = None
    for xs, ws in job:
        cts = []
        for (mseed, bound, level, eseed, nonce) in (xs, ws):
            m = W.int_plaintext(mseed, op.N, bound)
            cts.append(ckks.encrypt(op, pk, ckks.plaintext_from_ints(op, m, level, op.scale), eseed, nonce))
        t = ckks.mul(op, cts[0], cts[1])
        if acc is None:
            acc = t.c.copy()
        else:
            qs = ckks.primes_of(op, range(t.level + 1))
            for k in range(3):
                acc[k] = ckks.padd(acc[k], t.c[k], qs)
    return acc


def oracle_tensor_sum_parallel(op, o_pk, terms, workers=None):
    """The oracle's degree-2 sum of tensor products over `terms` (see
    oracle_tensor_partial), split over spawned worker processes; the partial
    sums are added modulo each prime (exact)."""
    import multiprocessing as mp
    import os

    workers = workers or max(1, os.cpu_count() or 1)
    chunks = [terms[i::workers * 2] for i in range(workers * 2)]
    chunks = [c for c in chunks if c]
    ctxm = mp.get_context("spawn")
    args = ((op.log_n, list(op.q_bits), list(op.p_bits), op.log2_scale), o_pk.b, o_pk.a)
    with ctxm.Pool(workers, initializer=_oracle_worker_init, initargs=args) as pool:
        parts = pool.map(oracle_tensor_partial, chunks)
    level = terms[0][0][2]
    qs = ckks.primes_of(op, range(level + 1))
    acc = parts[0]
    for p in parts[1:]:
        for k in range(3):
            acc[k] = ckks.padd(acc[k], p[k], qs)
    return ckks.Ciphertext(acc, level, op.scale * op.scale)
