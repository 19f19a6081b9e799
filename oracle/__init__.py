"""CPU oracle for the encrypted-CNN CKKS hot path.

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously correct CPU implementation
of what the GPU library computes, written from the scheme's definitions and
the paper (Jain et al., "Efficient CNN Building Blocks for Encrypted Data",
arXiv 2102.00319).  Only the test-suite (tests/), the package smoke check and
the benchmark's CPU-baseline leg may import it.  It shares no code with the
GPU library.

Modules:
  ckks_oracle.c  C core: primes, Philox, samplers, negacyclic products
                 (schoolbook; textbook-NTT mode), automorphism, fast basis
                 conversion, rescale.
  ckks.py        the scheme: keygen, encrypt, decrypt, add, constants, mul,
                 ModUp / key product / ModDown, relin, rescale, rotations.
  encoding.py    canonical-embedding encode / decode (direct FP64 sums), CRT.
  gaussian.py    the discrete-Gaussian cumulative table (decimal arithmetic).
  cnn.py         FP64 plaintext CNN and the canonical encrypted layer circuits.

Parity status: every function is pinned by tests/test_oracle_*.py against
brute force, closed forms, invariants or library routines; none is
"parity unpinned".
"""
from . import ckks, cnn, encoding, gaussian  # noqa: F401
from ._lib import build, lib  # noqa: F401
