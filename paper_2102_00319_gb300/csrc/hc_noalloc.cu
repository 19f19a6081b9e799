// Relinearisation that allocates no device memory (hc_relin_noalloc).
//
// Some callers cannot allocate device memory while they run this library's
// work: a process whose device memory was carved out and handed over at
// start-up (a fixed budget, no allocator on the hot path), or a
// latency-bound serving loop that must not take the allocator's locks or
// wait on it.  For them this variant of the key-switching relinearisation
// draws all of its scratch from one file-scope device array instead of the
// context allocator; the caller supplies the input and an already allocated
// output ciphertext.  It calls no cudaMalloc, cudaFree or allocator
// callback.
//
// Scratch: kNoAllocScratchWords 64-bit words (16 MiB) in a static __device__
// array.  Every GPU that loads the library holds this array until the process
// exits.  All calls share it and it keeps the last call's contents; every word
// a call reads is written earlier in the same call, so nothing needs clearing.
// Two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on the array; serialise them.
#include <mutex>

#include "hc_internal.h"

namespace {

constexpr size_t kNoAllocScratchWords = (size_t)1 << 21;  // 16 MiB
constexpr size_t kRefWords = 512;                          // room for 256 CtRef entries

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocScratchWords];

// Device address of the scratch array per device, taken once per device with
// that device current.  The host-side name of the array is only a stand-in,
// never a device address, so kernels get these pointers instead.
constexpr int kMaxDevices = 64;  // devices of one process this table can hold
u64* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

u64* scratch_on(int device) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  int count = 0;
  HC_CUDA(cudaGetDeviceCount(&count));
  HC_CHECK(device >= 0 && device < count && device < kMaxDevices, HC_ERR_INVALID, "device index out of range");
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    HC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[device] = (u64*)p;
  }
  return g_scratch_addr[device];
}

// Keeps the caller's current device across the call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    HC_CUDA(cudaGetDevice(&prev));
    if (prev != dev) HC_CUDA(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" int hc_relin_noalloc(hc_ctx* ctx, const hc_evk* evk, const hc_ct* x, hc_ct* out) {
  if (!ctx) return HC_ERR_INVALID;
  try {
    HC_CHECK(evk && x && out, HC_ERR_INVALID, "null argument");
    HC_CHECK(x->ctx == ctx && out->ctx == ctx, HC_ERR_INVALID, "handle of another context");
    HC_CHECK(x->degree == 2, HC_ERR_INVALID, "relin needs a degree-2 ciphertext");
    HC_CHECK(out->degree == 1 && out->level == x->level, HC_ERR_LEVEL_MISMATCH,
             "output must be a degree-1 ciphertext at the input's level");
    HC_CHECK(out->data != x->data, HC_ERR_INVALID, "output must not alias the input");
    DeviceGuard dg(ctx->device);
    u64* scratch = scratch_on(ctx->device);

    const int n = ctx->P.n, alpha = ctx->P.alpha, level = x->level;
    const int nq = level + 1, next = nq + alpha, dnum = ctx->lv[level].dnum;
    const size_t ext_words = (size_t)next * n;
    const size_t need = kRefWords + (size_t)nq * n + (size_t)dnum * ext_words + 2 * ext_words + 2 * (size_t)nq * n;
    HC_CHECK(need <= kNoAllocScratchWords, HC_ERR_INVALID,
             "hc_relin_noalloc: this level needs " + std::to_string(need) +
                 " scratch words; the static scratch holds " + std::to_string(kNoAllocScratchWords));
    HC_CHECK(2 * dnum + 8 <= (int)(kRefWords / 2), HC_ERR_INVALID, "too many digits for the reference table");

    // scratch layout: [CtRef table][xc][ext][acc][zq]
    CtRef* refs_dev = reinterpret_cast<CtRef*>(scratch);
    u64* xc = scratch + kRefWords;
    u64* ext = xc + (size_t)nq * n;
    u64* acc = ext + (size_t)dnum * ext_words;
    u64* zq = acc + 2 * ext_words;

    // host copy of the reference table (fixed size, on the stack)
    CtRef refs[kRefWords / 2];
    int nref = 0;
    const int r_x2 = nref++, r_x0 = nref++, r_x1 = nref++, r_out = nref++, r_xc = nref++;
    refs[r_x2] = CtRef{x->data + 2 * x->stride, x->stride};
    refs[r_x0] = CtRef{x->data, x->stride};
    refs[r_x1] = CtRef{x->data + x->stride, x->stride};
    refs[r_out] = out->ref();
    refs[r_xc] = CtRef{xc, 0};
    const int r_digits = nref;
    for (int j = 0; j < dnum; ++j) {
      const int d0 = j * alpha;
      refs[nref++] = CtRef{ext + (size_t)j * ext_words + (size_t)d0 * n, 0};  // digit limbs in ext
      refs[nref++] = CtRef{x->data + 2 * x->stride + (size_t)d0 * n, 0};     // same limbs of c2
    }
    static_assert(sizeof(CtRef) == 2 * sizeof(u64), "CtRef is two words");
    upload_words(ctx, reinterpret_cast<u64*>(refs_dev), reinterpret_cast<const u64*>(refs), 2 * (size_t)nref);

    const int* emap = ctx->ext_map_of(level);
    // c2 -> coefficient form
    launch_ew(ctx, 3, refs_dev + r_xc, refs_dev + r_x2, nullptr, 1, 1, nq);
    LimbSet s{};
    s.base = xc;
    s.npoly = 1;
    s.nlimb = nq;
    launch_ntt(ctx, s, 1, true, false);  // N^{-1} is folded into the conversion constants
    // ModUp per digit
    for (int j = 0; j < dnum; ++j) {
      const int d0 = j * alpha, d1 = std::min(d0 + alpha, nq);
      launch_ew(ctx, 3, refs_dev + r_digits + 2 * j, refs_dev + r_digits + 2 * j + 1, nullptr, 1, 1, d1 - d0);
      u64* ej = ext + (size_t)j * ext_words;
      launch_modup_bconv(ctx, level, j, xc, 0, ej, 0, 1);
      LimbSet e{};
      e.base = ej;
      e.npoly = 1;
      e.prime_map = emap;
      if (d0 > 0) {
        e.nlimb = d0;
        e.l0 = 0;
        launch_ntt(ctx, e, 1, false);
      }
      e.nlimb = next - d1;
      e.l0 = d1;
      launch_ntt(ctx, e, 1, false);
    }
    // key inner product, ModDown, add (c0, c1)
    launch_key_product(ctx, level, ext, 0, evk->relin.buf->ptr, acc, 0, 1);
    LimbSet a{};
    a.base = acc;
    a.poly_stride = ext_words;
    a.npoly = 2;
    a.nlimb = alpha;
    a.l0 = nq;
    a.prime_map = emap;
    launch_ntt(ctx, a, 1, true, false);
    launch_moddown_bconv(ctx, level, acc + (size_t)nq * n, 0, zq, 0, 1);
    LimbSet z{};
    z.base = zq;
    z.poly_stride = (u64)nq * n;
    z.npoly = 2;
    z.nlimb = nq;
    launch_ntt(ctx, z, 1, false);
    launch_moddown_combine(ctx, level, acc, 0, zq, 0, refs_dev + r_x0, refs_dev + r_x1, refs_dev + r_out, 1);
    out->scale = x->scale;
    ctx->err.clear();
    return HC_OK;
  } catch (const HcError& e) {
    ctx->err = e.msg;
    return e.code;
  } catch (...) {
    ctx->err = "unexpected error";
    return HC_ERR_INVALID;
  }
}
