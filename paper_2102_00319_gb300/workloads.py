"""Parameter sets and seeded synthetic inputs (no homomorphic arithmetic here).

Inputs stand in for the paper's MNIST workload (Sec. "Dataset and Inference
Results": 28x28 grayscale images) and trained weights, which are not
available: images are U[0,1] 28x28, weights N(0, 0.3), drawn from
numpy.random.Generator(PCG64(seed)).  Integer plaintexts for bit-exact
parity runs are drawn the same way.  Both the GPU path and the CPU oracle
consume these arrays; neither side's arithmetic lives in this module.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MASTER_SEED = 0x2102_0031_9000


@dataclass(frozen=True)
class ParamSet:
    name: str
    log_n: int
    q_bits: tuple
    p_bits: tuple
    log2_scale: float
    sigma: float = 3.2

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def slots(self):
        return self.n // 2


# N = 2^12, primes 50, 30, 30 bits + one 50-bit special prime, scale 2^30:
# one 8x8 image per ciphertext, conv by rotations then x^2 (two levels, so a
# second 30-bit rescale prime is added to the 50 + 30 chain).
SINGLE_N12 = ParamSet("single_n12", 12, (50, 30, 30), (50,), 30)
# N = 2^14, q_0 60 bits + six 40-bit primes, one 60-bit special prime,
# scale 2^40 (logQP = 360 <= 438): batch-packed CNN, 8192 images.
BATCH_N14 = ParamSet("batch_n14", 14, (60,) + (40,) * 6, (60,), 40)
# N = 2^16, q_0 60 bits + twenty 50-bit primes, seven 60-bit special primes
# (dnum = 3), scale 2^50: the per-operation HMult + relin + rescale workload.
DEEP_N16 = ParamSet("deep_n16_l20", 16, (60,) + (50,) * 20, (60,) * 7, 50)

PARAM_SETS = {p.name: p for p in (SINGLE_N12, BATCH_N14, DEEP_N16)}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def images(seed: int, count: int, h: int = 28, w: int = 28) -> np.ndarray:
    """count x h x w images with U[0,1] pixels."""
    return rng(seed).uniform(0.0, 1.0, (count, h, w))


def conv_weights(seed: int, cout: int, kh: int, kw: int, cin: int = 1) -> np.ndarray:
    return rng(seed).normal(0.0, 0.3, (cout, kh, kw, cin))


def fc_weights(seed: int, n_out: int, n_in: int) -> np.ndarray:
    return rng(seed).normal(0.0, 0.3, (n_out, n_in))


def slot_values(seed: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, count)


def int_plaintext(seed: int, n: int, bound: int) -> np.ndarray:
    """A random integer polynomial with coefficients in [-bound, bound]."""
    return rng(seed).integers(-bound, bound + 1, n, dtype=np.int64)


# Batch-packed CNN of the N = 2^14 workload: conv 5x5 stride 2 with 5
# channels -> x^2 -> 2x2 mean pool -> FC 180 -> 10.
CNN_BATCH = dict(H=28, W=28, cin=1, cout=5, k=5, stride=2, act=(0.0, 0.0, 1.0), n_out=10)


# Uneven multi-instance batch: 64 independent single-ciphertext inferences
# (8x8 image, 3x3 conv by rotations, x^2) with instance i at ring degree
# N = 2^(13 + i mod 3) and 3 + (7 i mod 10) rescalable primes (3..12).  The
# parameter style is the N = 2^12 workload's: a 50-bit q_0, 30-bit rescale
# primes, one 50-bit special prime, scale 2^30.  One 12-level context per
# ring degree serves every instance of that degree: prime chains and key
# limbs of a shorter chain are prefixes of the longer one.
UNEVEN_LMAX = 12


def uneven_params(log_n):
    return ParamSet("uneven_n%d" % log_n, log_n, (50,) + (30,) * UNEVEN_LMAX, (50,), 30)


def uneven_instances(count=64):
    """(log_n, level) of each instance."""
    return [(13 + i % 3, 3 + (7 * i) % 10) for i in range(count)]


SINGLE_CONV_STEPS = [p * 8 + q for p in range(3) for q in range(3)]


# Deep single-ciphertext CNN at N = 2^16, L = 20: a 28x28 image per
# ciphertext, conv 3x3 with 16 channels by hoisted rotations, a degree-7
# ReLU approximation, 2x2 mean pool by rotations, FC 13*13*16 -> 10 by
# encrypted weight vectors and rotate-and-sum.
DEEP_CNN = dict(H=28, W=28, cout=16, k=3, n_out=10)


def relu_cheb7(bound=2.0 ** 0.5):
    """Monomial coefficients c_0..c_7 of the degree-7 interpolant of ReLU at
    the 8 Chebyshev nodes of [-bound, bound] (the model's activation)."""
    k = np.arange(8)
    nodes = bound * np.cos((2 * k + 1) * np.pi / 16)
    V = np.vander(nodes, 8, increasing=True)
    return np.linalg.solve(V, np.maximum(nodes, 0.0))


def deep_conv_steps(W=28, k=3):
    return [p * W + q for p in range(k) for q in range(k)]


def deep_rot_steps(W=28, span_log2=10):
    steps = set(deep_conv_steps(W)) | {1, W, W + 1} | {1 << j for j in range(span_log2)}
    steps.discard(0)
    return sorted(steps)


def deep_fc_vectors(fc_w, C, Hp, Wp, W, slots):
    """Weight vectors V[r][c]: slot (2i W + 2j) holds fc_w[r, (i Wp + j) C + c]."""
    n_out = fc_w.shape[0]
    V = np.zeros((n_out, C, slots))
    for i in range(Hp):
        for j in range(Wp):
            for c in range(C):
                V[:, c, 2 * i * W + 2 * j] = fc_w[:, (i * Wp + j) * C + c]
    return V


# The paper's network (Sec. "Dataset and Inference Results"): 28 filters
# 3x3 without padding on 28x28 images -> ActPool (Eq. 4 activation, then 2x2
# mean) -> flatten 13*13*28 = 4732 -> FC 4732 x 10, K = 16384 images per batch
# at N = 2^15 (the paper's m = 2^16).  Levels: conv 6 -> 5, activation -> 3,
# pool -> 2, FC -> 1; q_0 60 bits, six 40-bit primes, one 60-bit special prime,
# scale 2^40 (logQP = 360).
PAPER_N15 = ParamSet("paper_n15", 15, (60,) + (40,) * 6, (60,), 40)
PAPER_CNN = dict(H=28, W=28, cout=28, k=3, stride=1, act=(0.47, 0.50, 0.09), n_out=10)
