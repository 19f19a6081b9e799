"""Loader for the oracle's C core (ckks_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle is the plain CPU reference that the GPU
library is checked against.  Only tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.

The shared object is compiled with gcc on first use (or by the package build
step) into ``oracle/_build/``.  Nothing here is shared with the GPU library.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libckks_oracle.so")
_lock = threading.Lock()
_lib = None

u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle's C core with gcc (OpenMP over independent limbs)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = ctypes.CDLL(_SO)
        u64 = ctypes.c_uint64
        c_int = ctypes.c_int
        L.or_powmod.restype = u64
        L.or_powmod.argtypes = [u64, u64, u64]
        L.or_invmod.restype = u64
        L.or_invmod.argtypes = [u64, u64]
        L.or_is_prime.restype = c_int
        L.or_is_prime.argtypes = [u64]
        L.or_gen_primes.restype = c_int
        L.or_gen_primes.argtypes = [c_int, i32p, c_int, u64p]
        L.or_philox4x64_10.restype = None
        L.or_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.or_sample_ternary.restype = None
        L.or_sample_ternary.argtypes = [u64, u64, c_int, i64p]
        L.or_sample_gauss.restype = None
        L.or_sample_gauss.argtypes = [u64, u64, c_int, u64p, c_int, i64p]
        L.or_sample_uniform.restype = None
        L.or_sample_uniform.argtypes = [u64, u64, u64, u64, c_int, u64p]
        L.or_reduce_signed.restype = None
        L.or_reduce_signed.argtypes = [i64p, c_int, u64p, c_int, u64p]
        L.or_set_mode.restype = None
        L.or_set_mode.argtypes = [c_int]
        L.or_get_mode.restype = c_int
        L.or_get_mode.argtypes = []
        for name in ("or_poly_add", "or_poly_sub", "or_poly_scalar_mul", "or_poly_add_const", "or_poly_mul"):
            f = getattr(L, name)
            f.restype = None
            f.argtypes = [u64p, u64p, u64p, u64p, c_int, c_int]
        L.or_poly_neg.restype = None
        L.or_poly_neg.argtypes = [u64p, u64p, u64p, c_int, c_int]
        pp = ctypes.POINTER(ctypes.c_void_p)
        L.or_poly_mul_many.restype = None
        L.or_poly_mul_many.argtypes = [pp, pp, pp, c_int, u64p, c_int, c_int]
        L.or_automorph.restype = None
        L.or_automorph.argtypes = [u64p, u64p, u64p, c_int, c_int, u64]
        L.or_fast_bconv.restype = None
        L.or_fast_bconv.argtypes = [u64p, u64p, c_int, u64p, u64p, c_int, c_int]
        L.or_rescale.restype = None
        L.or_rescale.argtypes = [u64p, u64p, u64p, c_int, c_int]
        _lib = L
        return _lib


def as_u64(x):
    return np.ascontiguousarray(x, dtype=np.uint64)
