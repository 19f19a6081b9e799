"""Thin ctypes binding of libhecnn (include/hecnn.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names; handles are wrapped in small Python
objects that call the matching hc_*_destroy when collected.  A missing or
unloadable library raises immediately: there is no fallback.

PyTorch supplies the CUDA stream (``torch.cuda.current_stream()``) and,
optionally, device memory through its caching allocator.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhecnn.so")

HC_OK = 0
ERRORS = {
    -1: "HC_ERR_INVALID", -2: "HC_ERR_LEVEL_MISMATCH", -3: "HC_ERR_SCALE_MISMATCH", -4: "HC_ERR_NO_KEY",
    -5: "HC_ERR_DEPTH", -6: "HC_ERR_OOM", -7: "HC_ERR_CUDA", -8: "HC_ERR_TIMEOUT",
}
HC_TUNE_NTT = 0
HC_TUNE_KEY_PRODUCT_Z = 1
HC_TUNE_MODUP_SPLIT = 2
HC_TUNE_TENSOR_GROUP = 3
HC_TUNE_HOST_STREAMS = 4
HC_PACK_BATCH = 0
HC_PACK_SINGLE = 1
HC_PACK_SINGLE_HOISTED = 2

# every symbol declared in include/hecnn.h
EXPORTS = [
    "hc_params_create", "hc_params_destroy", "hc_params_primes", "hc_params_info", "hc_params_cdt",
    "hc_ctx_create", "hc_ctx_destroy", "hc_sync", "hc_last_error", "hc_kernel_launches",
    "hc_profile_enable", "hc_profile_kernel", "hc_profile_names",
    "hc_keygen", "hc_sk_destroy", "hc_pk_destroy", "hc_evk_destroy", "hc_sk_export", "hc_pk_export",
    "hc_evk_export", "hc_encode", "hc_pt_from_coeffs", "hc_pt_export", "hc_decode", "hc_pt_level",
    "hc_pt_scale", "hc_pt_destroy", "hc_encrypt", "hc_decrypt", "hc_ct_export", "hc_ct_import",
    "hc_ct_meta_of", "hc_ct_destroy", "hc_add", "hc_sub", "hc_add_const", "hc_mul_const", "hc_mul",
    "hc_relin", "hc_rescale", "hc_drop_to_level", "hc_rotate", "hc_rotate_hoisted",
    "hc_mul_relin_rescale_batch", "hc_enc_conv2d", "hc_enc_poly_act", "hc_enc_pool", "hc_enc_fc",
    "hc_relin_noalloc", "hc_graph_begin", "hc_graph_end", "hc_graph_launch", "hc_graph_destroy",
    "hc_enc_conv2d_single_batch", "hc_enc_conv2d_single_hoisted_batch", "hc_enc_fc_rotsum", "hc_ct_import_batch", "hc_ct_export_batch",
    "hc_mul_relin_rescale_host", "hc_mul_relin_rescale_host_eval", "hc_ct_export_eval", "hc_ct_import_eval",
    "hc_mul_relin_rescale_host_eval_async", "hc_host_op_wait",
    "hc_autotune", "hc_tune_set", "hc_tune_get", "hc_int_mul_rates",
    "hc_enc_fc_partial", "hc_relin_rescale_batch", "hc_profile_host_timeline",
]


class HcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code


class ParamsDesc(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int), ("n_q", ctypes.c_int), ("q_bits", ctypes.POINTER(ctypes.c_int)),
                ("n_p", ctypes.c_int), ("p_bits", ctypes.POINTER(ctypes.c_int)),
                ("log2_scale", ctypes.c_double), ("sigma", ctypes.c_double)]


class CtMeta(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("degree", ctypes.c_int), ("scale", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Loads libhecnn.so; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libhecnn.so not built at %s: run paper_2102_00319_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    vp, c_int, u64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "hc_params_create": (c_int, [ctypes.POINTER(ParamsDesc), pp]),
        "hc_params_destroy": (None, [vp]),
        "hc_params_primes": (c_int, [vp, ctypes.POINTER(u64), c_int]),
        "hc_params_info": (c_int, [vp, ctypes.POINTER(c_int)] * 1 + [ctypes.POINTER(c_int)] * 3),
        "hc_params_cdt": (c_int, [vp, ctypes.POINTER(u64), c_int]),
        "hc_ctx_create": (c_int, [vp, c_int, vp, ctypes.POINTER(Allocator), pp]),
        "hc_ctx_destroy": (None, [vp]),
        "hc_sync": (c_int, [vp]),
        "hc_last_error": (ctypes.c_char_p, [vp]),
        "hc_kernel_launches": (u64, [vp]),
        "hc_profile_enable": (c_int, [vp, c_int]),
        "hc_profile_kernel": (c_int, [vp, ctypes.c_char_p, ctypes.POINTER(u64), ctypes.POINTER(dbl),
                                      ctypes.POINTER(u64)]),
        "hc_profile_names": (c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "hc_int_mul_rates": (c_int, [vp, ctypes.POINTER(dbl), c_int]),
        "hc_profile_host_timeline": (c_int, [vp, ctypes.POINTER(dbl), c_int]),
        "hc_keygen": (c_int, [vp, u64, ctypes.POINTER(ctypes.c_int32), c_int, pp, pp, pp]),
        "hc_sk_destroy": (None, [vp]), "hc_pk_destroy": (None, [vp]), "hc_evk_destroy": (None, [vp]),
        "hc_sk_export": (c_int, [vp, vp, ctypes.POINTER(ctypes.c_int8), ctypes.c_size_t]),
        "hc_pk_export": (c_int, [vp, vp, ctypes.POINTER(u64), ctypes.c_size_t]),
        "hc_evk_export": (c_int, [vp, vp, u64, ctypes.POINTER(u64), ctypes.c_size_t]),
        "hc_encode": (c_int, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.c_size_t, dbl, c_int, pp]),
        "hc_pt_from_coeffs": (c_int, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_size_t, c_int, dbl, pp]),
        "hc_pt_export": (c_int, [vp, vp, ctypes.POINTER(u64), ctypes.c_size_t]),
        "hc_decode": (c_int, [vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.c_size_t]),
        "hc_pt_level": (c_int, [vp]), "hc_pt_scale": (dbl, [vp]), "hc_pt_destroy": (None, [vp]),
        "hc_encrypt": (c_int, [vp, vp, vp, u64, u64, pp]),
        "hc_decrypt": (c_int, [vp, vp, vp, pp]),
        "hc_ct_export": (c_int, [vp, vp, ctypes.POINTER(u64), ctypes.c_size_t, ctypes.POINTER(CtMeta)]),
        "hc_ct_import": (c_int, [vp, ctypes.POINTER(u64), ctypes.POINTER(CtMeta), pp]),
        "hc_ct_meta_of": (c_int, [vp, ctypes.POINTER(CtMeta)]),
        "hc_ct_import_batch": (c_int, [vp, pp, ctypes.POINTER(CtMeta), c_int, pp]),
        "hc_ct_export_batch": (c_int, [vp, pp, c_int, pp, ctypes.POINTER(ctypes.c_size_t)]),
        "hc_autotune": (c_int, [vp, vp, c_int, ctypes.c_char_p, ctypes.c_size_t]),
        "hc_tune_set": (c_int, [vp, c_int, c_int]),
        "hc_tune_get": (c_int, [vp, c_int]),
        "hc_mul_relin_rescale_host": (c_int, [vp, vp, pp, ctypes.POINTER(CtMeta), pp, ctypes.POINTER(CtMeta), c_int,
                                              c_int, pp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(CtMeta)]),
        "hc_mul_relin_rescale_host_eval": (c_int, [vp, vp, pp, ctypes.POINTER(CtMeta), pp, ctypes.POINTER(CtMeta),
                                                   c_int, c_int, pp, ctypes.POINTER(ctypes.c_size_t),
                                                   ctypes.POINTER(CtMeta)]),
        "hc_mul_relin_rescale_host_eval_async": (c_int, [vp, vp, pp, ctypes.POINTER(CtMeta), pp,
                                                         ctypes.POINTER(CtMeta), c_int, c_int, pp,
                                                         ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(CtMeta),
                                                         ctypes.POINTER(vp)]),
        "hc_host_op_wait": (c_int, [vp]),
        "hc_ct_export_eval": (c_int, [vp, vp, ctypes.POINTER(u64), ctypes.c_size_t, ctypes.POINTER(CtMeta)]),
        "hc_ct_import_eval": (c_int, [vp, ctypes.POINTER(u64), ctypes.POINTER(CtMeta), pp]),
        "hc_ct_destroy": (None, [vp]),
        "hc_add": (c_int, [vp, vp, vp, pp]), "hc_sub": (c_int, [vp, vp, vp, pp]),
        "hc_add_const": (c_int, [vp, vp, dbl, pp]),
        "hc_mul_const": (c_int, [vp, vp, dbl, dbl, pp]),
        "hc_mul": (c_int, [vp, vp, vp, pp]),
        "hc_relin": (c_int, [vp, vp, vp, pp]),
        "hc_rescale": (c_int, [vp, vp, pp]),
        "hc_drop_to_level": (c_int, [vp, vp, c_int, pp]),
        "hc_rotate": (c_int, [vp, vp, vp, c_int, pp]),
        "hc_rotate_hoisted": (c_int, [vp, vp, vp, ctypes.POINTER(ctypes.c_int32), c_int, pp]),
        "hc_mul_relin_rescale_batch": (c_int, [vp, vp, pp, pp, c_int, pp]),
        "hc_enc_conv2d": (c_int, [vp, vp, c_int, pp, c_int, c_int, c_int, pp, c_int, c_int, c_int, c_int, pp]),
        "hc_enc_poly_act": (c_int, [vp, vp, pp, c_int, ctypes.POINTER(dbl), c_int, pp]),
        "hc_enc_pool": (c_int, [vp, vp, c_int, pp, c_int, c_int, c_int, pp]),
        "hc_enc_fc": (c_int, [vp, vp, c_int, pp, c_int, pp, pp, c_int, pp]),
        "hc_enc_fc_partial": (c_int, [vp, c_int, pp, c_int, pp, c_int, pp]),
        "hc_relin_rescale_batch": (c_int, [vp, vp, pp, c_int, pp]),
        "hc_relin_noalloc": (c_int, [vp, vp, vp, vp]),
        "hc_graph_begin": (c_int, [pp, c_int, ctypes.c_size_t]),
        "hc_graph_end": (c_int, [pp, c_int, pp]),
        "hc_graph_launch": (c_int, [vp]),
        "hc_graph_destroy": (None, [vp]),
        "hc_enc_conv2d_single_batch": (c_int, [vp, vp, pp, c_int, c_int, pp, c_int, c_int, c_int, pp]),
        "hc_enc_conv2d_single_hoisted_batch": (c_int, [vp, vp, pp, c_int, c_int, pp, c_int, c_int, c_int, pp]),
        "hc_enc_fc_rotsum": (c_int, [vp, vp, pp, c_int, pp, c_int, c_int, pp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# ---------------------------------------------------------------- handles
class _Handle:
    _destroy = None

    def __init__(self, ptr, owner=None):
        self.ptr = ctypes.c_void_p(ptr)
        self.owner = owner  # keeps the context alive while the handle lives

    def __del__(self):
        if self.ptr and self._destroy and _lib is not None:
            getattr(_lib, self._destroy)(self.ptr)
            self.ptr = ctypes.c_void_p()

    @property
    def _as_parameter_(self):
        return self.ptr


class Params(_Handle):
    _destroy = "hc_params_destroy"


class Context(_Handle):
    _destroy = "hc_ctx_destroy"

    def __init__(self, ptr, params_info, allocator_refs=None):
        super().__init__(ptr)
        self.n, self.L, self.alpha, self.dnum = params_info
        self._alloc_refs = allocator_refs

    def __del__(self):
        # device-resident handles must go first; they hold a reference to us
        super().__del__()


class SecretKey(_Handle):
    _destroy = "hc_sk_destroy"


class PublicKey(_Handle):
    _destroy = "hc_pk_destroy"


class EvalKeys(_Handle):
    _destroy = "hc_evk_destroy"


class Plaintext(_Handle):
    _destroy = "hc_pt_destroy"


class Ciphertext(_Handle):
    _destroy = "hc_ct_destroy"

    def meta(self):
        m = CtMeta()
        load().hc_ct_meta_of(self.ptr, ctypes.byref(m))
        return m

    @property
    def level(self):
        return self.meta().level

    @property
    def scale(self):
        return self.meta().scale

    @property
    def degree(self):
        return self.meta().degree


def _check(ctx, rc):
    if rc != HC_OK:
        msg = load().hc_last_error(ctx.ptr if ctx is not None else None)
        raise HcError(rc, (msg or b"").decode())


def _out():
    return ctypes.c_void_p()


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _ptr_array(handles):
    arr = (ctypes.c_void_p * max(1, len(handles)))()
    for i, h in enumerate(handles):
        arr[i] = h.ptr.value if h is not None else None
    return arr


# ------------------------------------------------------------- functions
def hc_params_create(log_n, q_bits, p_bits, log2_scale, sigma=3.2) -> Params:
    L = load()
    qb = (ctypes.c_int * len(q_bits))(*q_bits)
    pb = (ctypes.c_int * len(p_bits))(*p_bits)
    d = ParamsDesc(log_n, len(q_bits), qb, len(p_bits), pb, float(log2_scale), float(sigma))
    out = _out()
    rc = L.hc_params_create(ctypes.byref(d), ctypes.byref(out))
    if rc != HC_OK:
        raise HcError(rc, "hc_params_create")
    return Params(out.value)


def hc_params_primes(p: Params) -> list:
    buf = (ctypes.c_uint64 * 128)()
    rc = load().hc_params_primes(p.ptr, buf, 128)
    if rc != HC_OK:
        raise HcError(rc, "hc_params_primes")
    n, L_, a, _ = hc_params_info(p)
    return [int(buf[i]) for i in range(L_ + 1 + a)]


def hc_params_info(p: Params):
    v = [ctypes.c_int() for _ in range(4)]
    load().hc_params_info(p.ptr, *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def hc_params_cdt(p: Params) -> list:
    buf = (ctypes.c_uint64 * 64)()
    n = load().hc_params_cdt(p.ptr, buf, 64)
    if n < 0:
        raise HcError(n, "hc_params_cdt")
    return [int(buf[i]) for i in range(n)]


def torch_allocator(device=0):
    """hc_allocator callbacks backed by PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)
        except Exception:
            return None

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a_fn, f_fn = ALLOC_FN(_alloc), FREE_FN(_free)
    return Allocator(a_fn, f_fn, None), (a_fn, f_fn)


def hc_ctx_create(params: Params, device=0, stream=None, allocator=None) -> Context:
    """stream: a cudaStream_t as int (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    L = load()
    out = _out()
    refs = None
    aptr = None
    if allocator is not None:
        alloc_struct, refs = allocator
        aptr = ctypes.byref(alloc_struct)
        refs = (alloc_struct, refs)
    rc = L.hc_ctx_create(params.ptr, device, ctypes.c_void_p(stream) if stream else None, aptr, ctypes.byref(out))
    if rc != HC_OK:
        raise HcError(rc, "hc_ctx_create")
    return Context(out.value, hc_params_info(params), refs)


def hc_sync(ctx):
    _check(ctx, load().hc_sync(ctx.ptr))


def hc_kernel_launches(ctx) -> int:
    return int(load().hc_kernel_launches(ctx.ptr))


def hc_profile_enable(ctx, on=True):
    _check(ctx, load().hc_profile_enable(ctx.ptr, 1 if on else 0))


def hc_profile_kernel(ctx, name):
    """(launches, total device ms, work units) of kernel `name` since profiling was enabled."""
    n, ms, u = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_uint64()
    _check(ctx, load().hc_profile_kernel(ctx.ptr, name.encode(), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(u)))
    return int(n.value), float(ms.value), int(u.value)


def hc_profile_names(ctx):
    buf = ctypes.create_string_buffer(8192)
    _check(ctx, load().hc_profile_names(ctx.ptr, buf, 8192))
    return [x for x in buf.value.decode().split(",") if x]


def hc_profile_host_timeline(ctx):
    """Per chunk of the last profiled host-to-host call: (copy-in start, end,
    kernels start, end, copy-out start, end) in ms from the call's start."""
    L = load()
    n = L.hc_profile_host_timeline(ctx.ptr, None, 0)
    buf = (ctypes.c_double * max(1, n))()
    L.hc_profile_host_timeline(ctx.ptr, buf, n)
    return [tuple(buf[6 * c: 6 * c + 6]) for c in range(n // 6)]


INT_MUL_FORMS = ("imad32", "umulhi32", "imad_wide32", "mul_lo64", "mul_hi64", "mac128", "shoup_lazy",
                 "ct_butterfly", "split_conv_epilogue")


def hc_int_mul_rates(ctx):
    """{form: (ops per SM per clock at the maximum clock, ops per second)} of
    the integer-multiply forms and the modular units of work, measured on
    the context's GPU."""
    k = len(INT_MUL_FORMS)
    r = (ctypes.c_double * (2 * k))()
    _check(ctx, load().hc_int_mul_rates(ctx.ptr, r, 2 * k))
    return {f: (r[i], r[k + i]) for i, f in enumerate(INT_MUL_FORMS)}


def hc_keygen(ctx, seed, rot_steps=()):
    L = load()
    steps = (ctypes.c_int32 * max(1, len(rot_steps)))(*rot_steps)
    sk, pk, evk = _out(), _out(), _out()
    _check(ctx, L.hc_keygen(ctx.ptr, seed, steps, len(rot_steps), ctypes.byref(sk), ctypes.byref(pk), ctypes.byref(evk)))
    return SecretKey(sk.value, ctx), PublicKey(pk.value, ctx), EvalKeys(evk.value, ctx)


def hc_sk_export(ctx, sk) -> np.ndarray:
    out = np.zeros(ctx.n, dtype=np.int8)
    _check(ctx, load().hc_sk_export(ctx.ptr, sk.ptr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), ctx.n))
    return out


def hc_pk_export(ctx, pk) -> np.ndarray:
    out = np.zeros((2, ctx.L + 1, ctx.n), dtype=np.uint64)
    _check(ctx, load().hc_pk_export(ctx.ptr, pk.ptr, _u64p(out), out.size))
    return out


def hc_evk_export(ctx, evk, galois_elt=1) -> np.ndarray:
    out = np.zeros((ctx.dnum, 2, ctx.L + 1 + ctx.alpha, ctx.n), dtype=np.uint64)
    _check(ctx, load().hc_evk_export(ctx.ptr, evk.ptr, galois_elt, _u64p(out), out.size))
    return out


def hc_encode(ctx, values, scale, level) -> Plaintext:
    v = np.asarray(values)
    re = np.ascontiguousarray(v.real, dtype=np.float64)
    im = np.ascontiguousarray(v.imag, dtype=np.float64) if np.iscomplexobj(v) else None
    out = _out()
    dp = ctypes.POINTER(ctypes.c_double)
    _check(ctx, load().hc_encode(ctx.ptr, re.ctypes.data_as(dp), im.ctypes.data_as(dp) if im is not None else None,
                                 len(re), float(scale), level, ctypes.byref(out)))
    return Plaintext(out.value, ctx)


def hc_pt_from_coeffs(ctx, coeffs, level, scale) -> Plaintext:
    c = np.ascontiguousarray(coeffs, dtype=np.int64)
    out = _out()
    _check(ctx, load().hc_pt_from_coeffs(ctx.ptr, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(c), level,
                                         float(scale), ctypes.byref(out)))
    return Plaintext(out.value, ctx)


def hc_pt_export(ctx, pt) -> np.ndarray:
    lv = load().hc_pt_level(pt.ptr)
    out = np.zeros((lv + 1, ctx.n), dtype=np.uint64)
    _check(ctx, load().hc_pt_export(ctx.ptr, pt.ptr, _u64p(out), out.size))
    return out


def hc_decode(ctx, pt, n=None) -> np.ndarray:
    n = ctx.n // 2 if n is None else n
    re = np.zeros(n)
    im = np.zeros(n)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(ctx, load().hc_decode(ctx.ptr, pt.ptr, re.ctypes.data_as(dp), im.ctypes.data_as(dp), n))
    return re + 1j * im


def hc_encrypt(ctx, pk, pt, seed, nonce) -> Ciphertext:
    out = _out()
    _check(ctx, load().hc_encrypt(ctx.ptr, pk.ptr, pt.ptr, seed, nonce, ctypes.byref(out)))
    return Ciphertext(out.value, ctx)


def hc_decrypt(ctx, sk, ct) -> Plaintext:
    out = _out()
    _check(ctx, load().hc_decrypt(ctx.ptr, sk.ptr, ct.ptr, ctypes.byref(out)))
    return Plaintext(out.value, ctx)


def hc_ct_export(ctx, ct) -> tuple:
    m = ct.meta()
    out = np.zeros((m.degree + 1, m.level + 1, ctx.n), dtype=np.uint64)
    meta = CtMeta()
    _check(ctx, load().hc_ct_export(ctx.ptr, ct.ptr, _u64p(out), out.size, ctypes.byref(meta)))
    return out, meta


def hc_ct_import(ctx, data, level, degree, scale) -> Ciphertext:
    d = np.ascontiguousarray(data, dtype=np.uint64)
    meta = CtMeta(level, degree, float(scale))
    out = _out()
    _check(ctx, load().hc_ct_import(ctx.ptr, _u64p(d), ctypes.byref(meta), ctypes.byref(out)))
    return Ciphertext(out.value, ctx)


def hc_ct_export_eval(ctx, ct) -> tuple:
    """The device words in evaluation (NTT) form, [degree+1][level+1][N]."""
    m = ct.meta()
    out = np.zeros((m.degree + 1, m.level + 1, ctx.n), dtype=np.uint64)
    meta = CtMeta()
    _check(ctx, load().hc_ct_export_eval(ctx.ptr, ct.ptr, _u64p(out), out.size, ctypes.byref(meta)))
    return out, meta


def hc_ct_import_eval(ctx, data, level, degree, scale) -> Ciphertext:
    d = np.ascontiguousarray(data, dtype=np.uint64)
    meta = CtMeta(level, degree, float(scale))
    out = _out()
    _check(ctx, load().hc_ct_import_eval(ctx.ptr, _u64p(d), ctypes.byref(meta), ctypes.byref(out)))
    return Ciphertext(out.value, ctx)


def hc_ct_import_batch(ctx, arrays, metas):
    """arrays: C-contiguous uint64 arrays [degree+1][level+1][N] (pinned for
    asynchronous copies); metas: (level, degree, scale) per ciphertext."""
    n = len(arrays)
    if len(metas) != n:
        raise ValueError("one meta per array")
    for a, (lv, dg, _) in zip(arrays, metas):
        if a.dtype != np.uint64 or not a.flags.c_contiguous or a.size != (dg + 1) * (lv + 1) * ctx.n:
            raise ValueError("each array must be C-contiguous uint64 of (degree+1)*(level+1)*N words")
    ptrs = (ctypes.c_void_p * max(1, n))(*[a.ctypes.data for a in arrays])
    m = (CtMeta * max(1, n))(*[CtMeta(lv, dg, float(sc)) for lv, dg, sc in metas])
    outs = _outs(n)
    _check(ctx, load().hc_ct_import_batch(ctx.ptr, ptrs, m, n, outs))
    return _wrap_outs(ctx, outs, n)


def hc_ct_export_batch(ctx, cts, arrays):
    """Writes each ciphertext (coefficient form) into the matching uint64 array."""
    n = len(cts)
    if len(arrays) != n or any(a.dtype != np.uint64 or not a.flags.c_contiguous for a in arrays):
        raise ValueError("one C-contiguous uint64 array per ciphertext")
    ptrs = (ctypes.c_void_p * max(1, n))(*[a.ctypes.data for a in arrays])
    caps = (ctypes.c_size_t * max(1, n))(*[a.size for a in arrays])
    _check(ctx, load().hc_ct_export_batch(ctx.ptr, _ptr_array(cts), n, ptrs, caps))


def hc_mul_relin_rescale_host(ctx, evk, a_arrays, a_metas, b_arrays, b_metas, out_arrays, chunk=0, eval_form=False):
    """Host-to-host batch: a_arrays/b_arrays are C-contiguous uint64
    [2][level+1][N] ciphertexts (coefficient form, or evaluation form with
    eval_form) with (level, degree, scale) metas; out_arrays receive
    [2][level][N] in the same form.  Returns the output metas."""
    n = len(a_arrays)
    if not (len(b_arrays) == len(a_metas) == len(b_metas) == len(out_arrays) == n):
        raise ValueError("one entry per pair in every list")
    for a, (lv, dg, _) in zip(list(a_arrays) + list(b_arrays), list(a_metas) + list(b_metas)):
        if a.dtype != np.uint64 or not a.flags.c_contiguous or a.size != (dg + 1) * (lv + 1) * ctx.n:
            raise ValueError("inputs must be C-contiguous uint64 of (degree+1)*(level+1)*N words")
    if any(o.dtype != np.uint64 or not o.flags.c_contiguous or not o.flags.writeable for o in out_arrays):
        raise ValueError("outputs must be writeable C-contiguous uint64 arrays")

    def ptrs(arrs):
        return (ctypes.c_void_p * max(1, n))(*[x.ctypes.data for x in arrs])

    def metas(ms):
        return (CtMeta * max(1, n))(*[CtMeta(lv, dg, float(sc)) for lv, dg, sc in ms])

    caps = (ctypes.c_size_t * max(1, n))(*[o.size for o in out_arrays])
    out_m = (CtMeta * max(1, n))()
    fn = load().hc_mul_relin_rescale_host_eval if eval_form else load().hc_mul_relin_rescale_host
    _check(ctx, fn(ctx.ptr, evk.ptr, ptrs(a_arrays), metas(a_metas), ptrs(b_arrays), metas(b_metas), n, int(chunk),
                   ptrs(out_arrays), caps, out_m))
    return [out_m[i] for i in range(n)]


class HostOp:
    """A host-to-host call in flight: keeps its buffers alive until wait()."""

    def __init__(self, ctx, handle, keepalive, metas):
        self.ctx, self.handle, self._keepalive, self.metas = ctx, handle, keepalive, metas

    def wait(self):
        """Returns the output metas once every output is in host memory."""
        if self.handle is None:
            return self.metas
        h, self.handle = self.handle, None
        _check(self.ctx, load().hc_host_op_wait(h))
        self._keepalive = None
        return self.metas


def hc_mul_relin_rescale_host_async(ctx, evk, a_arrays, a_metas, b_arrays, b_metas, out_arrays, chunk=0):
    """The evaluation-form host-to-host batch without waiting: returns a
    HostOp whose wait() returns the output metas; the arrays must not be
    touched before it."""
    n = len(a_arrays)
    if not (len(b_arrays) == len(a_metas) == len(b_metas) == len(out_arrays) == n):
        raise ValueError("one entry per pair in every list")
    for a, (lv, dg, _) in zip(list(a_arrays) + list(b_arrays), list(a_metas) + list(b_metas)):
        if a.dtype != np.uint64 or not a.flags.c_contiguous or a.size != (dg + 1) * (lv + 1) * ctx.n:
            raise ValueError("inputs must be C-contiguous uint64 of (degree+1)*(level+1)*N words")
    if any(o.dtype != np.uint64 or not o.flags.c_contiguous or not o.flags.writeable for o in out_arrays):
        raise ValueError("outputs must be writeable C-contiguous uint64 arrays")
    ptr = lambda arrs: (ctypes.c_void_p * max(1, n))(*[x.ctypes.data for x in arrs])
    meta = lambda ms: (CtMeta * max(1, n))(*[CtMeta(lv, dg, float(sc)) for lv, dg, sc in ms])
    args = [ptr(a_arrays), meta(a_metas), ptr(b_arrays), meta(b_metas), ptr(out_arrays),
            (ctypes.c_size_t * max(1, n))(*[o.size for o in out_arrays]), (CtMeta * max(1, n))()]
    handle = ctypes.c_void_p()
    _check(ctx, load().hc_mul_relin_rescale_host_eval_async(ctx.ptr, evk.ptr, args[0], args[1], args[2], args[3], n,
                                                           int(chunk), args[4], args[5], args[6],
                                                           ctypes.byref(handle)))
    metas = [args[6][i] for i in range(n)]
    return HostOp(ctx, handle.value, (list(a_arrays), list(b_arrays), list(out_arrays), args), metas)


def hc_autotune(ctx, evk, items):
    """Times the tuning knobs' candidates and keeps the fastest; returns the
    report (one line per knob: chosen value, microseconds per candidate)."""
    buf = ctypes.create_string_buffer(4096)
    _check(ctx, load().hc_autotune(ctx.ptr, evk.ptr, int(items), buf, len(buf)))
    return buf.value.decode()


def hc_tune_set(ctx, knob, value):
    _check(ctx, load().hc_tune_set(ctx.ptr, int(knob), int(value)))


def hc_tune_get(ctx, knob):
    v = load().hc_tune_get(ctx.ptr, int(knob))
    if v < 0:
        raise HcError(v, "hc_tune_get")
    return v


def _unary(name, ctx, *args):
    out = _out()
    _check(ctx, getattr(load(), name)(ctx.ptr, *args, ctypes.byref(out)))
    return Ciphertext(out.value, ctx)


def hc_add(ctx, x, y):
    return _unary("hc_add", ctx, x.ptr, y.ptr)


def hc_sub(ctx, x, y):
    return _unary("hc_sub", ctx, x.ptr, y.ptr)


def hc_add_const(ctx, x, c):
    return _unary("hc_add_const", ctx, x.ptr, float(c))


def hc_mul_const(ctx, x, c, const_scale):
    return _unary("hc_mul_const", ctx, x.ptr, float(c), float(const_scale))


def hc_mul(ctx, x, y):
    return _unary("hc_mul", ctx, x.ptr, y.ptr)


def hc_relin(ctx, evk, x):
    return _unary("hc_relin", ctx, evk.ptr, x.ptr)


def hc_relin_noalloc(ctx, evk, x, out):
    """Relinearises x into the caller's existing ciphertext `out` without
    allocating device memory (see include/hecnn.h)."""
    _check(ctx, load().hc_relin_noalloc(ctx.ptr, evk.ptr, x.ptr, out.ptr))
    return out


def hc_rescale(ctx, x):
    return _unary("hc_rescale", ctx, x.ptr)


def hc_drop_to_level(ctx, x, level):
    return _unary("hc_drop_to_level", ctx, x.ptr, level)


def hc_rotate(ctx, evk, x, steps):
    return _unary("hc_rotate", ctx, evk.ptr, x.ptr, steps)


def _outs(n):
    return (ctypes.c_void_p * max(1, n))()


def _wrap_outs(ctx, arr, n):
    return [Ciphertext(arr[i], ctx) for i in range(n)]


def hc_rotate_hoisted(ctx, evk, x, steps):
    st = (ctypes.c_int32 * max(1, len(steps)))(*steps)
    outs = _outs(len(steps))
    _check(ctx, load().hc_rotate_hoisted(ctx.ptr, evk.ptr, x.ptr, st, len(steps), outs))
    return _wrap_outs(ctx, outs, len(steps))


def hc_mul_relin_rescale_batch(ctx, evk, a, b):
    outs = _outs(len(a))
    _check(ctx, load().hc_mul_relin_rescale_batch(ctx.ptr, evk.ptr, _ptr_array(a), _ptr_array(b), len(a), outs))
    return _wrap_outs(ctx, outs, len(a))


def hc_enc_conv2d(ctx, evk, packing, x, H, W, cin, w, cout, kh, kw, stride):
    if packing == HC_PACK_BATCH:
        nout = ((H - kh) // stride + 1) * ((W - kw) // stride + 1) * cout
    else:
        nout = cout
    outs = _outs(nout)
    _check(ctx, load().hc_enc_conv2d(ctx.ptr, evk.ptr, packing, _ptr_array(x), H, W, cin, _ptr_array(w), cout, kh, kw,
                                     stride, outs))
    return _wrap_outs(ctx, outs, nout)


class Graph(_Handle):
    _destroy = "hc_graph_destroy"


def hc_graph_begin(ctxs, arena_bytes):
    arr = _ptr_array(ctxs)
    rc = load().hc_graph_begin(arr, len(ctxs), arena_bytes)
    _check(ctxs[0], rc)


def hc_graph_end(ctxs):
    arr = _ptr_array(ctxs)
    out = _out()
    _check(ctxs[0], load().hc_graph_end(arr, len(ctxs), ctypes.byref(out)))
    return Graph(out.value, list(ctxs))


def hc_graph_launch(g):
    rc = load().hc_graph_launch(g.ptr)
    if rc != HC_OK:
        raise HcError(rc, "hc_graph_launch")


def hc_enc_conv2d_single_batch(ctx, evk, x, W, w, cout, kh, kw):
    nout = len(x) * cout
    outs = _outs(nout)
    _check(ctx, load().hc_enc_conv2d_single_batch(ctx.ptr, evk.ptr, _ptr_array(x), len(x), W, _ptr_array(w), cout,
                                                  kh, kw, outs))
    return _wrap_outs(ctx, outs, nout)


def hc_enc_conv2d_single_hoisted_batch(ctx, evk, x, W, w, cout, kh, kw):
    nout = len(x) * cout
    outs = _outs(nout)
    _check(ctx, load().hc_enc_conv2d_single_hoisted_batch(ctx.ptr, evk.ptr, _ptr_array(x), len(x), W, _ptr_array(w),
                                                          cout, kh, kw, outs))
    return _wrap_outs(ctx, outs, nout)


def hc_enc_poly_act(ctx, evk, x, coeffs):
    """coeffs: 3 values (degree 2) or 8 values (degree 7)."""
    deg = len(coeffs) - 1
    c = (ctypes.c_double * len(coeffs))(*coeffs)
    outs = _outs(len(x))
    _check(ctx, load().hc_enc_poly_act(ctx.ptr, evk.ptr, _ptr_array(x), len(x), c, deg, outs))
    return _wrap_outs(ctx, outs, len(x))


def hc_enc_pool(ctx, evk, packing, x, C, H, W):
    nout = C if packing == HC_PACK_SINGLE else (H // 2) * (W // 2) * C
    outs = _outs(nout)
    _check(ctx, load().hc_enc_pool(ctx.ptr, evk.ptr if evk is not None else None, packing, _ptr_array(x), C, H, W,
                                   outs))
    return _wrap_outs(ctx, outs, nout)


def hc_enc_fc_rotsum(ctx, evk, x, w, n_out, span_log2):
    outs = _outs(n_out)
    _check(ctx, load().hc_enc_fc_rotsum(ctx.ptr, evk.ptr, _ptr_array(x), len(x), _ptr_array(w), n_out, span_log2,
                                        outs))
    return _wrap_outs(ctx, outs, n_out)


def hc_relin_rescale_batch(ctx, evk, d):
    """[rescale(relin(c)) for c in d], one batched pass (degree-2 inputs at one level)."""
    outs = _outs(len(d))
    _check(ctx, load().hc_relin_rescale_batch(ctx.ptr, evk.ptr, _ptr_array(d), len(d), outs))
    return _wrap_outs(ctx, outs, len(d))


def hc_enc_fc_partial(ctx, packing, x, w, n_out):
    """Degree-2 sums y[r] = sum_k x_k (x) w[r n_in + k] (no relinearisation)."""
    outs = _outs(n_out)
    _check(ctx, load().hc_enc_fc_partial(ctx.ptr, packing, _ptr_array(x), len(x), _ptr_array(w), n_out, outs))
    return _wrap_outs(ctx, outs, n_out)


def hc_enc_fc(ctx, evk, packing, x, w, n_out, bias=None):
    outs = _outs(n_out)
    _check(ctx, load().hc_enc_fc(ctx.ptr, evk.ptr, packing, _ptr_array(x), len(x), _ptr_array(w),
                                 _ptr_array(bias) if bias is not None else None, n_out, outs))
    return _wrap_outs(ctx, outs, n_out)
