"""GB300 (sm_103a) implementation of the CKKS ciphertext-by-ciphertext hot path
of encrypted CNN inference (Jain et al., "Efficient CNN Building Blocks for
Encrypted Data", arXiv 2102.00319).

The computation lives in libhecnn.so (CUDA, C ABI in include/hecnn.h);
`hecnn` is its ctypes binding, `workloads` the seeded synthetic inputs and
parameter sets, `build` the in-tree nvcc build.
"""
from . import hecnn  # noqa: F401
