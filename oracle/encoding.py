"""CKKS encoding by the canonical embedding, as direct sums in FP64 (oracle).

TEST INFRASTRUCTURE ONLY.

The plaintext ring is Z[X]/(X^N + 1) (the paper's Z[X]/(Phi_m(X)) with
m = 2N a power of two); K = N/2 complex slots (Sec. "Impact of FHE
parameters": K = phi(m)/2).  Slot j is the evaluation at zeta^{5^j},
zeta = exp(i pi / N).  Encoding inverts the embedding on the real
polynomials:

    m_i = round( scale * (2/N) * Re sum_{j<K} z_j zeta^{-5^j i} ),

decoding evaluates:  z_j = scale^{-1} sum_i m_i zeta^{5^j i},  with m_i the
centred lift of the residues by the Chinese remainder theorem.  Both are
plain O(N K) sums; angles are reduced exactly in integers before the
trigonometric table lookup.
"""
import math

import numpy as np

from .ckks import llround


def _zeta_table(n: int):
    k = np.arange(2 * n, dtype=np.float64)
    return np.cos(np.pi * k / n), np.sin(np.pi * k / n)


def _rot_group(n: int) -> np.ndarray:
    """5^j mod 2N for j < K."""
    out = np.empty(n // 2, dtype=np.int64)
    g = 1
    for j in range(n // 2):
        out[j] = g
        g = (g * 5) % (2 * n)
    return out


def encode_real_coeffs(z, n: int, scale: float, block: int = 256) -> np.ndarray:
    """The real (unrounded) coefficients scale*(2/N)*Re sum_j z_j zeta^{-5^j i}."""
    K = n // 2
    zz = np.zeros(K, dtype=np.complex128)
    z = np.asarray(z, dtype=np.complex128)
    zz[: len(z)] = z
    cos_t, sin_t = _zeta_table(n)
    g = _rot_group(n)
    out = np.empty(n, dtype=np.float64)
    two_n = 2 * n
    for i0 in range(0, n, block):
        i = np.arange(i0, min(i0 + block, n), dtype=np.int64)
        e = (-(g[None, :] * i[:, None])) % two_n  # exponent of zeta
        re = cos_t[e] @ zz.real - sin_t[e] @ zz.imag
        out[i0: i0 + len(i)] = re
    return out * (2.0 / n) * scale


def encode(z, n: int, scale: float) -> np.ndarray:
    """Integer plaintext coefficients (int64), rounded half away from zero."""
    real = encode_real_coeffs(z, n, scale)
    if np.max(np.abs(real)) >= 2.0 ** 62:
        raise ValueError("encoded coefficient out of range")
    return np.array([llround(float(v)) for v in real], dtype=np.int64)


def crt_centred(residues, primes) -> list:
    """Centred CRT lift of [limbs][N] residues: Python integers in (-Q/2, Q/2]."""
    primes = [int(q) for q in primes]
    Q = math.prod(primes)
    terms = []
    for r, q in zip(residues, primes):
        hat = Q // q
        terms.append((hat, pow(hat % q, -1, q), q, [int(v) for v in r]))
    n = len(terms[0][3])
    out = []
    for i in range(n):
        x = 0
        for hat, hinv, q, r in terms:
            x += (r[i] * hinv % q) * hat
        x %= Q
        if x > Q // 2:
            x -= Q
        out.append(x)
    return out


def decode_coeffs(m, n: int, scale: float, block: int = 256) -> np.ndarray:
    """Slots z_j = scale^{-1} sum_i m_i zeta^{5^j i} from real coefficients m."""
    m = np.asarray(m, dtype=np.float64)
    cos_t, sin_t = _zeta_table(n)
    g = _rot_group(n)
    K = n // 2
    out = np.empty(K, dtype=np.complex128)
    two_n = 2 * n
    i = np.arange(n, dtype=np.int64)
    for j0 in range(0, K, block):
        gj = g[j0: j0 + block]
        e = (gj[:, None] * i[None, :]) % two_n
        out[j0: j0 + len(gj)] = (cos_t[e] @ m) + 1j * (sin_t[e] @ m)
    return out / scale


def decode(residues, primes, n: int, scale: float) -> np.ndarray:
    lifted = crt_centred(residues, primes)
    return decode_coeffs([float(v) for v in lifted], n, scale)
