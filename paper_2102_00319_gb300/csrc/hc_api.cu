// C ABI of libhecnn (declared in include/hecnn.h): handle lifecycle and the
// composition of the kernels into the scheme's operations and CNN layers.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <numeric>

#include "hc_internal.h"

// ------------------------------------------------------------ memory
DevBuf::~DevBuf() {
  if (ctx && ptr && owned) ctx->free_words(ptr);
}

u64* hc_ctx::alloc_words(size_t words) {
  const size_t bytes = std::max<size_t>(words, 1) * sizeof(u64);
  void* p = nullptr;
  if (user_alloc) {
    p = alloc.alloc(bytes, (void*)stream, alloc.user);
  } else {
    if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (!p) throw HcError{HC_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  if (((uintptr_t)p & 15) != 0) {  // kernels move limbs in 16-byte vectors
    if (user_alloc) alloc.free(p, (void*)stream, alloc.user);
    throw HcError{HC_ERR_INVALID, "allocator returned memory not aligned to 16 bytes"};
  }
  return (u64*)p;
}

void hc_ctx::free_words(u64* p) {
  if (!p) return;
  if (user_alloc) alloc.free(p, (void*)stream, alloc.user);
  else cudaFreeAsync(p, stream);
}

BufPtr hc_ctx::buffer(size_t words) {
  auto b = std::make_shared<DevBuf>();
  b->ctx = this;
  b->bytes = std::max<size_t>(words, 1) * sizeof(u64);
  if (arena) {
    const size_t w = (std::max<size_t>(words, 1) + 31) & ~(size_t)31;  // 256-byte steps
    if (arena_off + w > arena_words)
      throw HcError{HC_ERR_OOM, "capture arena exhausted (" + std::to_string(arena_words * 8) + " bytes)"};
    b->ptr = arena + arena_off;
    arena_off += w;
    b->owned = false;
  } else {
    b->ptr = alloc_words(words);
  }
  return b;
}

ProfScope::ProfScope(hc_ctx* c, const char* n, uint64_t u) : ctx(c), name(n), units(u) {
  if (!ctx->prof) return;
  auto take = [&]() {
    cudaEvent_t e = nullptr;
    if (!ctx->event_pool.empty()) {
      e = ctx->event_pool.back();
      ctx->event_pool.pop_back();
    } else {
      HC_CUDA(cudaEventCreate(&e));
    }
    return e;
  };
  a = take();
  b = take();
  HC_CUDA(cudaEventRecord(a, ctx->stream));
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEventRecord(b, ctx->stream);
  ctx->prof_events[name].push_back({a, b});
  ctx->prof_units[name] += units;
}

namespace {
void recycle_events(hc_ctx* ctx) {
  for (auto& kv : ctx->prof_events)
    for (auto& pr : kv.second) {
      ctx->event_pool.push_back(pr.first);
      ctx->event_pool.push_back(pr.second);
    }
  ctx->prof_events.clear();
  ctx->prof_units.clear();
}
}  // namespace


namespace {

// Device workspace budget of one batched key switch (chunks beyond it run in turn).
constexpr size_t kWorkspaceBytes = (size_t)8 << 30;

// Run `f`, translating exceptions into return codes and the context error.
template <class F>
int guard(hc_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->err.clear();
    return HC_OK;
  } catch (const HcError& e) {
    if (ctx) ctx->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed";
    return HC_ERR_OOM;
  } catch (...) {
    if (ctx) ctx->err = "unexpected error";
    return HC_ERR_INVALID;
  }
}

hc_ct* new_ct(hc_ctx* ctx, int level, int degree, double scale) {
  const size_t stride = (size_t)(level + 1) * ctx->P.n;
  BufPtr b = ctx->buffer(stride * (degree + 1));
  return new hc_ct{ctx, b, b->ptr, stride, level, degree, scale};
}

// Outputs sharing one slab.
// Runs fn(b) for b in [0, nb) on side streams forked from the context
// stream and joined back to it: every launcher inside fn sees ctx->stream
// set to branch b's stream, so independent groups of work (the levels of a
// mixed batch) overlap on the device; captured into a graph the branches
// become concurrent nodes.  Memory a branch allocates and frees is ordered
// on its own stream; results stay usable on the context stream after the
// join.  nb <= 1 runs inline.  On an error the branches already issued are
// still joined before the error propagates.
template <class F>
void fork_join(hc_ctx* ctx, int nb, F&& fn) {
  if (nb <= 1) {
    if (nb == 1) fn(0);
    return;
  }
  const cudaStream_t home = ctx->stream;
  while ((int)ctx->aux_streams.size() < nb) {
    cudaStream_t st = nullptr;
    HC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ctx->aux_streams.push_back(st);
  }
  auto mark = [](cudaStream_t st) {
    cudaEvent_t e = nullptr;
    HC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    const cudaError_t r = cudaEventRecord(e, st);
    if (r != cudaSuccess) {
      cudaEventDestroy(e);
      throw HcError{HC_ERR_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(r)};
    }
    return e;
  };
  cudaEvent_t fork = mark(home);
  int started = 0;
  auto join = [&]() {
    ctx->stream = home;
    for (int b = 0; b < started; ++b) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
        if (cudaEventRecord(e, ctx->aux_streams[b]) == cudaSuccess) cudaStreamWaitEvent(home, e, 0);
        cudaEventDestroy(e);
      }
    }
    cudaEventDestroy(fork);
  };
  try {
    for (int b = 0; b < nb; ++b) {
      const cudaStream_t st = ctx->aux_streams[b];
      HC_CUDA(cudaStreamWaitEvent(st, fork, 0));
      ++started;
      ctx->stream = st;
      fn(b);
      ctx->stream = home;
    }
  } catch (...) {
    join();
    throw;
  }
  join();
}

std::vector<hc_ct*> new_cts(hc_ctx* ctx, int count, int level, int degree, double scale) {
  std::vector<hc_ct*> out;
  if (count <= 0) return out;
  const size_t stride = (size_t)(level + 1) * ctx->P.n;
  const size_t per = stride * (degree + 1);
  BufPtr b = ctx->buffer(per * count);
  for (int i = 0; i < count; ++i) out.push_back(new hc_ct{ctx, b, b->ptr + per * i, stride, level, degree, scale});
  return out;
}

CtRef* refs_dev(hc_ctx* ctx, const std::vector<CtRef>& v, std::vector<BufPtr>& keep) {
  return upload(ctx, v, keep);
}

const int* ids_dev(hc_ctx* ctx, const std::vector<int>& v, std::vector<BufPtr>& keep) {
  return upload(ctx, v, keep);
}

void check_scales(double a, double b) {
  HC_CHECK(std::fabs(a - b) <= std::ldexp(1.0, -40) * std::max(std::fabs(a), std::fabs(b)),
           HC_ERR_SCALE_MISMATCH, "operand scales differ");
}

LimbSet limbset_base(u64* base, u64 item_stride, u64 poly_stride, int npoly, int nlimb, int l0,
                     const int* pmap) {
  LimbSet s{};
  s.refs = nullptr;
  s.base = base;
  s.item_stride = item_stride;
  s.poly_stride = poly_stride;
  s.npoly = npoly;
  s.nlimb = nlimb;
  s.l0 = l0;
  s.prime_map = pmap;
  return s;
}

// identity prime map [0..63] lives at the start of ext_map's buffer tail
const int* ident_map(hc_ctx* ctx) { return ctx->ext_map + (ctx->P.L + 1) * (ctx->P.L + 1 + ctx->P.alpha); }

// ModUp of a batch: for every digit j, the conversions of the digit's limbs
// of xc (coefficient form) to the other slots of Q_l u P, in NTT form.  A
// digit's own slots are taken from x by the specialised key product; with
// more than eight digits they are copied into ext instead.
// ModUp of m items: xs[i] their c1 (NTT form), xc the same in coefficient
// form.  Digits with alpha primes run together: one conversion launch and
// one transform launch over all their raised slots (a 2-D slot map, digit
// by digit); a last, shorter digit gets launches of its own.  With copy_own
// the digits' own slots are copied from xs into ext as well (one launch);
// otherwise the key product reads them from xs.
void modup_digits(hc_ctx* ctx, int level, const std::vector<CtRef>& xs, const u64* xc, u64 x_is, u64* ext, u64 ext_is,
                  int m, std::vector<BufPtr>& keep, bool copy_own) {
  const int n = ctx->P.n, alpha = ctx->P.alpha, nq = level + 1, next = nq + alpha, dnum = ctx->lv[level].dnum;
  const size_t ext_words = (size_t)next * n;
  const int* emap = ctx->ext_map_of(level);
  const int full = nq / alpha;  // digits with alpha primes (the first ones)
  if (copy_own) {
    for (int j0 = 0; j0 < dnum; j0 = std::max(j0 + 1, full)) {
      // the full digits in one launch, then the shorter last one
      const int j1 = j0 < full ? full : dnum, ns = std::min(alpha, nq - j0 * alpha);
      std::vector<CtRef> er, xsh;
      for (int i = 0; i < m; ++i)
        for (int j = j0; j < j1; ++j) {
          er.push_back(CtRef{ext + ext_is * i + (size_t)j * ext_words + (size_t)j * alpha * n, 0});
          xsh.push_back(CtRef{xs[i].p + (size_t)j * alpha * n, 0});
        }
      launch_ew(ctx, 3, refs_dev(ctx, er, keep), refs_dev(ctx, xsh, keep), nullptr, (int)er.size(), 1, ns);
    }
  }
  if (full > 0 && alpha <= 8) {
    launch_modup_bconv_fast(ctx, level, 0, xc, x_is, ext, ext_is, m, full);
    LimbSet e = limbset_base(ext, ext_is, ext_words, full, next - alpha, 0, emap);
    e.slot_map = ctx->modup_slots_of(level, 0);  // digit-major: each full digit's next - alpha raised slots
    e.slot_map_2d = 1;
    launch_ntt(ctx, e, m, false);
  }
  for (int j = (alpha <= 8 ? full : 0); j < dnum; ++j) {
    const int d0 = j * alpha, d1 = std::min(d0 + alpha, nq);
    launch_modup_bconv_fast(ctx, level, j, xc, x_is, ext + (size_t)j * ext_words, ext_is, m);
    LimbSet e = limbset_base(ext + (size_t)j * ext_words, ext_is, 0, 1, next - (d1 - d0), 0, emap);
    e.slot_map = ctx->modup_slots_of(level, j);  // the raised slots, one launch
    launch_ntt(ctx, e, m, false);
  }
}

// ---------------------------------------------------------------------
// Key switching of a batch of single polynomials x (NTT form, level l):
//   out_k = base_k + KS(x)_k,  k = 0, 1 (base_k may be null).
// ---------------------------------------------------------------------
// Per-item switching keys: keys[i] switches item i (runs of equal keys share
// one key-product launch; every other stage is one launch over all items).
void keyswitch_batch_keys(hc_ctx* ctx, const std::vector<const u64*>& keys, int level, const std::vector<CtRef>& x,
                          const std::vector<CtRef>* base0, const std::vector<CtRef>* base1,
                          const std::vector<CtRef>& out);

void keyswitch_batch(hc_ctx* ctx, const u64* key, int level, const std::vector<CtRef>& x,
                     const std::vector<CtRef>* base0, const std::vector<CtRef>* base1,
                     const std::vector<CtRef>& out) {
  keyswitch_batch_keys(ctx, std::vector<const u64*>(x.size(), key), level, x, base0, base1, out);
}

void keyswitch_batch_keys(hc_ctx* ctx, const std::vector<const u64*>& keys, int level, const std::vector<CtRef>& x,
                          const std::vector<CtRef>* base0, const std::vector<CtRef>* base1,
                          const std::vector<CtRef>& out) {
  const int n = ctx->P.n, alpha = ctx->P.alpha;
  const int nq = level + 1, next = nq + alpha, dnum = ctx->lv[level].dnum;
  const int total = (int)x.size();
  const size_t ext_words = (size_t)next * n;
  const size_t per_item = (size_t)nq * n + (size_t)dnum * ext_words + 2 * ext_words + 2 * (size_t)nq * n;
  int chunk = (int)std::max<size_t>(1, kWorkspaceBytes / (per_item * 8));
  chunk = std::min(chunk, 256);
  const int* emap = ctx->ext_map_of(level);
  for (int s0 = 0; s0 < total; s0 += chunk) {
    const int m = std::min(chunk, total - s0);
    std::vector<BufPtr> keep;
    std::vector<CtRef> xs(x.begin() + s0, x.begin() + s0 + m);
    std::vector<CtRef> os(out.begin() + s0, out.begin() + s0 + m);
    const CtRef* xr = refs_dev(ctx, xs, keep);
    const CtRef* orr = refs_dev(ctx, os, keep);
    const CtRef* b0 = nullptr;
    const CtRef* b1 = nullptr;
    if (base0) b0 = refs_dev(ctx, std::vector<CtRef>(base0->begin() + s0, base0->begin() + s0 + m), keep);
    if (base1) b1 = refs_dev(ctx, std::vector<CtRef>(base1->begin() + s0, base1->begin() + s0 + m), keep);
    BufPtr work = ctx->buffer(per_item * m);
    keep.push_back(work);
    u64* xc = work->ptr;                                  // [m][nq][N] coefficient copy of x
    u64* ext = xc + (size_t)m * nq * n;                   // [m][dnum][next][N]
    u64* acc = ext + (size_t)m * dnum * ext_words;        // [m][2][next][N]
    u64* zq = acc + (size_t)m * 2 * ext_words;            // [m][2][nq][N]
    const u64 x_is = (u64)nq * n, ext_is = (u64)dnum * ext_words, acc_is = 2 * (u64)ext_words,
              z_is = 2 * (u64)nq * n;
    // x -> coefficient form, read in place by the first inverse pass
    LimbSet xin{};
    xin.refs = xr;
    xin.npoly = 1;
    xin.nlimb = nq;
    launch_ntt_from(ctx, limbset_base(xc, x_is, 0, 1, nq, 0, nullptr), &xin, m, true, false);
    modup_digits(ctx, level, xs, xc, x_is, ext, ext_is, m, keep, dnum > 8);
    // one key-product launch: a shared key, or a device table of per-item keys
    bool same_key = true;
    for (int r = 1; r < m; ++r) same_key = same_key && keys[s0 + r] == keys[s0];
    const u64* const* item_keys = nullptr;
    if (!same_key) {
      item_keys = upload(ctx, std::vector<const u64*>(keys.begin() + s0, keys.begin() + s0 + m), keep);
    }
    launch_key_product_batched(ctx, level, ext, ext_is, keys[s0], acc, acc_is, m, dnum <= 8 ? xr : nullptr,
                               item_keys);
    // ModDown
    launch_ntt(ctx, limbset_base(acc, acc_is, ext_words, 2, alpha, nq, emap), m, true, false);
    launch_moddown_bconv_fast(ctx, level, acc + (size_t)nq * n, acc_is, zq, z_is, m);
    launch_ntt(ctx, limbset_base(zq, z_is, (u64)nq * n, 2, nq, 0, nullptr), m, false);
    launch_moddown_combine(ctx, level, acc, acc_is, zq, z_is, b0, b1, orr, m);
  }
}

// Key switch of x followed by a rescale, fused: with u = key product over
// Q_l u P and z = FastBConv_{P->Q}([u]_P) (coefficient form), both carrying
// ModDown's P^{-1} on Q (the keys' Q limbs and the conversion constants hold
// it: u' = u P^{-1}, z' = z P^{-1}),
//   relin_k[i]  = base_k[i] + u'_k[i] - NTT(z'_k[i]),
//   rescale_k[i] = (relin_k[i] - NTT([relin_k[l]] mod q_i)) q_l^{-1},
// and NTT is linear, so one NTT of (z'_k[i] + [relin_k[l]] mod q_i) per limb
// serves both; the last limb of relin_k is formed in coefficient form from
// INTT(base_k[l] + u'_k[l]) - z'_k[l].  Bit-identical to keyswitch_batch
// followed by rescale_batch.  out: degree-1, level l-1.
// With coeff_out the results go there in coefficient form instead (2 polys x
// l limbs per item, `out` unused): by linearity the inverse NTT of
// base_k[i] + u'_k[i] minus (z'_k[i] + [c_l]_{q_i}), times q_l^{-1}, is the
// inverse NTT of the NTT-form result, so the same words come out with one
// transform per limb instead of two.
void keyswitch_rescale_batch(hc_ctx* ctx, const u64* key, int level, const std::vector<CtRef>& x,
                             const std::vector<CtRef>* base0, const std::vector<CtRef>* base1,
                             const std::vector<CtRef>& out, const LimbSet* coeff_out = nullptr) {
  const int n = ctx->P.n, alpha = ctx->P.alpha;
  const int nq = level + 1, next = nq + alpha, dnum = ctx->lv[level].dnum;
  const int total = (int)x.size();
  const size_t ext_words = (size_t)next * n;
  const size_t per_item =
      (size_t)nq * n + (size_t)dnum * ext_words + 2 * ext_words + 2 * (size_t)nq * n + 2 * (size_t)n;
  int chunk = (int)std::max<size_t>(1, kWorkspaceBytes / (per_item * 8));
  chunk = std::min(chunk, 256);
  const int* emap = ctx->ext_map_of(level);
  for (int s0 = 0; s0 < total; s0 += chunk) {
    const int m = std::min(chunk, total - s0);
    std::vector<BufPtr> keep;
    std::vector<CtRef> xs(x.begin() + s0, x.begin() + s0 + m);
    const CtRef* xr = refs_dev(ctx, xs, keep);
    const CtRef* orr =
        coeff_out ? nullptr : refs_dev(ctx, std::vector<CtRef>(out.begin() + s0, out.begin() + s0 + m), keep);
    const CtRef* b0 = nullptr;
    const CtRef* b1 = nullptr;
    if (base0) b0 = refs_dev(ctx, std::vector<CtRef>(base0->begin() + s0, base0->begin() + s0 + m), keep);
    if (base1) b1 = refs_dev(ctx, std::vector<CtRef>(base1->begin() + s0, base1->begin() + s0 + m), keep);
    BufPtr work = ctx->buffer(per_item * m);
    keep.push_back(work);
    u64* xc = work->ptr;                            // [m][nq][N]
    u64* ext = xc + (size_t)m * nq * n;             // [m][dnum][next][N]
    u64* acc = ext + (size_t)m * dnum * ext_words;  // [m][2][next][N]
    u64* zq = acc + (size_t)m * 2 * ext_words;      // [m][2][nq][N]
    u64* tl = zq + (size_t)m * 2 * nq * n;          // [m][2][N]
    const u64 x_is = (u64)nq * n, ext_is = (u64)dnum * ext_words, acc_is = 2 * (u64)ext_words,
              z_is = 2 * (u64)nq * n;
    // x -> coefficient form, read in place by the first inverse pass
    LimbSet xin{};
    xin.refs = xr;
    xin.npoly = 1;
    xin.nlimb = nq;
    const LimbSet xcs = limbset_base(xc, x_is, 0, 1, nq, 0, nullptr);
    launch_ntt_from(ctx, xcs, &xin, m, true, false);
    modup_digits(ctx, level, xs, xc, x_is, ext, ext_is, m, keep, dnum > 8);
    // the digits' own slots are read from x itself (specialised key product)
    launch_key_product_batched(ctx, level, ext, ext_is, key, acc, acc_is, m, dnum <= 8 ? xr : nullptr);
    launch_ntt(ctx, limbset_base(acc, acc_is, ext_words, 2, alpha, nq, emap), m, true, false);
    launch_moddown_bconv_fast(ctx, level, acc + (size_t)nq * n, acc_is, zq, z_is, m);
    launch_ksr_last(ctx, level, acc, acc_is, b0, b1, tl, m);
    launch_ntt(ctx, limbset_base(tl, 2 * (u64)n, (u64)n, 2, 1, 0, ident_map(ctx) + level), m, true);
    // c_l (centred, signed) over tl; the forward NTT of z lifts it on load and
    // forms (base + acc - NTT(.)) q_l^{-1} on store (acc and z carry P^{-1})
    launch_ksr_cl(ctx, level, tl, zq, z_is, m);
    KsrFuse f{};
    ksr_constants(ctx, level, f);
    f.cl = tl;
    f.acc = acc;
    f.acc_item_stride = acc_is;
    f.acc_poly_stride = ext_words;
    f.base0 = b0;
    f.base1 = b1;
    f.out = orr;
    if (coeff_out) {
      f.z = zq;
      f.z_item_stride = z_is;
      f.z_poly_stride = (u64)nq * n;
      LimbSet co = *coeff_out;
      co.base += (size_t)s0 * co.item_stride;
      launch_intt_ksr(ctx, co, m, f);
    } else {
      launch_ntt_ksr(ctx, limbset_base(zq, z_is, (u64)nq * n, 2, level, 0, nullptr), m, f);
    }
  }
}

// Rescale a batch in place-free fashion: out (level-1) from in (level).
void rescale_batch(hc_ctx* ctx, const std::vector<CtRef>& in, const std::vector<CtRef>& out, int level,
                   int npoly) {
  const int n = ctx->P.n, total = (int)in.size();
  const size_t per = (size_t)npoly * n * (1 + level);
  int chunk = (int)std::min<size_t>(4096, std::max<size_t>(1, ((size_t)2 << 30) / (per * 8)));
  for (int s0 = 0; s0 < total; s0 += chunk) {
    const int m = std::min(chunk, total - s0);
    std::vector<BufPtr> keep;
    const CtRef* ir = refs_dev(ctx, std::vector<CtRef>(in.begin() + s0, in.begin() + s0 + m), keep);
    const CtRef* orr = refs_dev(ctx, std::vector<CtRef>(out.begin() + s0, out.begin() + s0 + m), keep);
    BufPtr work = ctx->buffer(per * m);
    keep.push_back(work);
    u64* last = work->ptr;                         // [m][npoly][N]
    u64* lift = last + (size_t)m * npoly * n;      // [m][npoly][level][N]
    launch_gather_limb(ctx, ir, level, last, m, npoly);
    launch_ntt(ctx, limbset_base(last, (u64)npoly * n, (u64)n, npoly, 1, 0, ident_map(ctx) + level), m, true);
    launch_rescale_lift(ctx, level, last, lift, m, npoly);
    launch_ntt(ctx, limbset_base(lift, (u64)npoly * level * n, (u64)level * n, npoly, level, 0, nullptr), m, false);
    launch_rescale_combine(ctx, level, ir, lift, orr, m, npoly);
  }
}

void check_ct(const hc_ctx* ctx, const hc_ct* c) {
  HC_CHECK(c != nullptr, HC_ERR_INVALID, "null ciphertext");
  HC_CHECK(c->ctx == ctx, HC_ERR_INVALID, "ciphertext of another context");
}

void relin_batch(hc_ctx* ctx, const hc_evk* evk, const std::vector<const hc_ct*>& d, std::vector<hc_ct*>& out) {
  if (d.empty()) return;
  const int level = d[0]->level;
  std::vector<CtRef> x, b0, b1, o;
  for (size_t i = 0; i < d.size(); ++i) {
    HC_CHECK(d[i]->degree == 2 && d[i]->level == level, HC_ERR_INVALID, "relin batch needs degree-2 cts at one level");
    x.push_back(CtRef{d[i]->data + 2 * d[i]->stride, d[i]->stride});
    b0.push_back(CtRef{d[i]->data, d[i]->stride});
    b1.push_back(CtRef{d[i]->data + d[i]->stride, d[i]->stride});
    o.push_back(out[i]->ref());
  }
  keyswitch_batch(ctx, evk->relin.buf->ptr, level, x, &b0, &b1, o);
}

void rescale_cts(hc_ctx* ctx, const std::vector<const hc_ct*>& in, std::vector<hc_ct*>& out) {
  if (in.empty()) return;
  const int level = in[0]->level, deg = in[0]->degree;
  HC_CHECK(level >= 1, HC_ERR_DEPTH, "no level left to rescale");
  std::vector<CtRef> ir, orr;
  for (size_t i = 0; i < in.size(); ++i) {
    HC_CHECK(in[i]->level == level && in[i]->degree == deg, HC_ERR_LEVEL_MISMATCH, "rescale batch mixes levels");
    ir.push_back(in[i]->ref());
    orr.push_back(out[i]->ref());
  }
  rescale_batch(ctx, ir, orr, level, deg + 1);
}

// Tensor-accumulate products into fresh degree-2 cts.
std::vector<hc_ct*> tensor_acc(hc_ctx* ctx, const std::vector<const hc_ct*>& xs, const std::vector<const hc_ct*>& ws,
                               const std::vector<int>& xi, const std::vector<int>& wi, const std::vector<int>& off,
                               int level, double scale) {
  const int nout = (int)off.size() - 1;
  std::vector<hc_ct*> out = new_cts(ctx, nout, level, 2, scale);
  std::vector<BufPtr> keep;
  std::vector<CtRef> xr, wr, orr;
  for (auto* c : xs) xr.push_back(c->ref());
  for (auto* c : ws) wr.push_back(c->ref());
  for (auto* c : out) orr.push_back(c->ref());
  // Grouped form: the largest G (up to the tuning knob, at most 5) such that
  // the outputs split into consecutive runs of G with identical x sequences
  // (a conv position's channels, an FC layer's classes).
  const int gmax = std::min(5, ctx->tune.tensor_group);
  auto same_x = [&](int a, int b) {
    if (off[a + 1] - off[a] != off[b + 1] - off[b]) return false;
    return std::equal(xi.begin() + off[a], xi.begin() + off[a + 1], xi.begin() + off[b]);
  };
  int G = 0;
  for (int cand = gmax; cand >= 1 && !G; --cand) {
    if (nout % cand) continue;
    bool ok = true;
    for (int g0 = 0; g0 < nout && ok; g0 += cand)
      for (int k = 1; k < cand && ok; ++k) ok = same_x(g0, g0 + k);
    if (ok) G = cand;
  }
  if (G >= 1) {
    const int ngroups = nout / G;
    std::vector<int> gxi, gwi, goff{0};
    for (int g = 0; g < ngroups; ++g) {
      const int o = g * G, nt = off[o + 1] - off[o];
      for (int t = 0; t < nt; ++t) {
        gxi.push_back(xi[off[o] + t]);
        for (int k = 0; k < G; ++k) gwi.push_back(wi[off[o + k] + t]);
      }
      goff.push_back((int)gxi.size());
    }
    const CtRef* xd = refs_dev(ctx, xr, keep);
    const CtRef* wd = refs_dev(ctx, wr, keep);
    const int* gxid = ids_dev(ctx, gxi, keep);
    const int* gwid = ids_dev(ctx, gwi, keep);
    for (int g0 = 0; g0 < ngroups; g0 += 65535) {
      const int m = std::min(65535, ngroups - g0);
      std::vector<int> off_sub(goff.begin() + g0, goff.begin() + g0 + m + 1);
      launch_tensor_acc_grouped(
          ctx, G, refs_dev(ctx, std::vector<CtRef>(orr.begin() + (size_t)g0 * G, orr.begin() + (size_t)(g0 + m) * G), keep),
          xd, wd, gxid, gwid, ids_dev(ctx, off_sub, keep), m, level + 1,
          (uint64_t)(off_sub.back() - off_sub.front()) * G);
    }
    return out;
  }
  for (int o0 = 0; o0 < nout; o0 += 65535) {
    const int m = std::min(65535, nout - o0);
    std::vector<int> off_sub(off.begin() + o0, off.begin() + o0 + m + 1);
    launch_tensor_acc(ctx, refs_dev(ctx, std::vector<CtRef>(orr.begin() + o0, orr.begin() + o0 + m), keep),
                      refs_dev(ctx, xr, keep), refs_dev(ctx, wr, keep), ids_dev(ctx, xi, keep), ids_dev(ctx, wi, keep),
                      ids_dev(ctx, off_sub, keep), m, level + 1, (uint64_t)(off_sub.back() - off_sub.front()));
  }
  return out;
}

// relin + rescale of a batch of degree-2 cts -> fresh degree-1 cts at level-1.
// A bias is added to (d0, d1) before the key switch, which equals adding it
// to the relinearised ciphertext.
std::vector<hc_ct*> relin_rescale(hc_ctx* ctx, const hc_evk* evk, const std::vector<hc_ct*>& d,
                                  const std::vector<const hc_ct*>* bias, const LimbSet* coeff_out = nullptr) {
  if (d.empty()) return {};
  const int level = d[0]->level;
  HC_CHECK(level >= 1, HC_ERR_DEPTH, "no level left to rescale");
  if (bias) {
    std::vector<BufPtr> keep;
    std::vector<CtRef> dr, br;
    for (size_t i = 0; i < d.size(); ++i) {
      const hc_ct* b = (*bias)[i];
      HC_CHECK(b->degree == 1 && b->level >= level, HC_ERR_LEVEL_MISMATCH, "bias level too low");
      check_scales(d[i]->scale, b->scale);
      dr.push_back(d[i]->ref());
      br.push_back(b->ref());
    }
    const CtRef* dd = refs_dev(ctx, dr, keep);
    launch_ew(ctx, 0, dd, dd, refs_dev(ctx, br, keep), (int)d.size(), 2, level + 1);
  }
  // with coeff_out the results are written there and no ciphertexts are made
  std::vector<hc_ct*> out;
  if (!coeff_out) out = new_cts(ctx, (int)d.size(), level - 1, 1, d[0]->scale / (double)ctx->P.chain[level]);
  std::vector<CtRef> x, b0, b1, o;
  for (size_t i = 0; i < d.size(); ++i) {
    HC_CHECK(d[i]->degree == 2 && d[i]->level == level, HC_ERR_INVALID, "relin batch needs degree-2 cts at one level");
    x.push_back(CtRef{d[i]->data + 2 * d[i]->stride, d[i]->stride});
    b0.push_back(CtRef{d[i]->data, d[i]->stride});
    b1.push_back(CtRef{d[i]->data + d[i]->stride, d[i]->stride});
    if (!coeff_out) {
      out[i]->scale = d[i]->scale / (double)ctx->P.chain[level];
      o.push_back(out[i]->ref());
    }
  }
  keyswitch_rescale_batch(ctx, evk->relin.buf->ptr, level, x, &b0, &b1, o, coeff_out);
  return out;
}

void constant_residues(hc_ctx* ctx, int level, double value, bool with_shoup, std::vector<u64>& out) {
  bool ok = false;
  const int64_t m = hch::round_half_away(value, &ok);
  HC_CHECK(ok, HC_ERR_INVALID, "constant out of range (|c * scale| >= 2^62)");
  const int nl = level + 1;
  out.assign(with_shoup ? 2 * nl : nl, 0);
  for (int i = 0; i < nl; ++i) {
    const u64 q = ctx->P.chain[i];
    u64 r = m >= 0 ? (u64)m % q : (q - ((u64)(-(m + 1)) % q) - 1);
    out[i] = r;
    if (with_shoup) out[nl + i] = hch::shoup_of(r, q);
  }
}

std::vector<hc_ct*> mul_const_cts(hc_ctx* ctx, const std::vector<const hc_ct*>& x, double c, double cs) {
  if (x.empty()) return {};
  const int level = x[0]->level, deg = x[0]->degree;
  std::vector<u64> sc;
  constant_residues(ctx, level, c * cs, true, sc);
  std::vector<hc_ct*> out = new_cts(ctx, (int)x.size(), level, deg, x[0]->scale * cs);
  std::vector<BufPtr> keep;
  std::vector<CtRef> xr, orr;
  for (size_t i = 0; i < x.size(); ++i) {
    HC_CHECK(x[i]->level == level && x[i]->degree == deg, HC_ERR_LEVEL_MISMATCH, "batch mixes levels");
    out[i]->scale = x[i]->scale * cs;
    xr.push_back(x[i]->ref());
    orr.push_back(out[i]->ref());
  }
  launch_scalar(ctx, false, refs_dev(ctx, orr, keep), refs_dev(ctx, xr, keep), (int)x.size(), deg + 1, level + 1,
                upload(ctx, sc, keep));
  return out;
}

std::vector<hc_ct*> rotate_one(hc_ctx* ctx, const hc_evk* evk, const hc_ct* x, const std::vector<int>& steps,
                               bool hoisted);
std::vector<hc_ct*> rotate_batch(hc_ctx* ctx, const hc_evk* evk, const std::vector<const hc_ct*>& xs, int step);
std::vector<std::vector<hc_ct*>> rotate_hoisted_batch(hc_ctx* ctx, const hc_evk* evk,
                                                      const std::vector<const hc_ct*>& xs,
                                                      const std::vector<int>& steps);

void free_all(std::vector<hc_ct*>& v) {
  for (auto* c : v) delete c;
  v.clear();
}

}  // namespace

// =====================================================================
// Parameters
// =====================================================================
extern "C" int hc_params_create(const hc_params_desc* d, hc_params** out) {
  return guard(nullptr, [&] {
    HC_CHECK(d && out, HC_ERR_INVALID, "null argument");
    HC_CHECK(d->log_n >= 10 && d->log_n <= 16, HC_ERR_INVALID, "log_n must be 10..16");
    HC_CHECK(d->n_q >= 1 && d->n_p >= 1 && d->n_p <= 16 && d->n_q + d->n_p <= HC_MAX_CHAIN, HC_ERR_INVALID,
             "bad prime counts");
    HC_CHECK(d->q_bits && d->p_bits, HC_ERR_INVALID, "null bit sizes");
    HC_CHECK(d->sigma > 0 && d->sigma < 6.5, HC_ERR_INVALID, "sigma out of range");
    std::vector<int> bits(d->q_bits, d->q_bits + d->n_q);
    bits.insert(bits.end(), d->p_bits, d->p_bits + d->n_p);
    for (int b : bits) HC_CHECK(b >= 20 && b <= 61, HC_ERR_INVALID, "prime bit size must be 20..61");
    auto* p = new hc_params();
    p->log_n = d->log_n;
    p->n = 1 << d->log_n;
    p->L = d->n_q - 1;
    p->alpha = d->n_p;
    p->dnum = (d->n_q + d->n_p - 1) / d->n_p;
    p->chain.resize(bits.size());
    if (hch::gen_primes(d->log_n, bits.data(), (int)bits.size(), p->chain.data()) != 0) {
      delete p;
      throw HcError{HC_ERR_INVALID, "not enough primes of the requested sizes"};
    }
    p->below_2_60 = std::all_of(p->chain.begin(), p->chain.end(), [](u64 q) { return q < (1ull << 60); });
    p->scale = std::exp2(d->log2_scale);
    p->sigma = d->sigma;
    p->cdt = hch::gaussian_cdt(d->sigma);
    *out = p;
  });
}

extern "C" void hc_params_destroy(hc_params* p) { delete p; }

extern "C" int hc_params_primes(const hc_params* p, uint64_t* out, int cap) {
  if (!p || !out || cap < p->nchain()) return HC_ERR_INVALID;
  for (int i = 0; i < p->nchain(); ++i) out[i] = p->chain[i];
  return HC_OK;
}

extern "C" int hc_params_info(const hc_params* p, int* n, int* L, int* alpha, int* dnum) {
  if (!p) return HC_ERR_INVALID;
  if (n) *n = p->n;
  if (L) *L = p->L;
  if (alpha) *alpha = p->alpha;
  if (dnum) *dnum = p->dnum;
  return HC_OK;
}

extern "C" int hc_params_cdt(const hc_params* p, uint64_t* out, int cap) {
  if (!p || !out || cap < (int)p->cdt.size()) return HC_ERR_INVALID;
  for (size_t i = 0; i < p->cdt.size(); ++i) out[i] = p->cdt[i];
  return (int)p->cdt.size();
}

// =====================================================================
// Context
// =====================================================================
namespace {
void build_tables(hc_ctx* ctx) {
  const hc_params& P = ctx->P;
  const int n = P.n, nc = P.nchain(), logn = P.log_n;
  std::vector<u64> fwd(2 * (size_t)nc * n), inv(2 * (size_t)nc * n);  // interleaved (w, w')
  std::vector<u64> ninv(nc), ninv_sh(nc);
  std::vector<DMod> mods(nc);
  std::vector<u64> pw(n), ipw(n);
  for (int c = 0; c < nc; ++c) {
    const u64 q = P.chain[c];
    const u64 psi = hch::primitive_2n_root(logn, q);
    HC_CHECK(psi != 0, HC_ERR_INVALID, "no 2N-th root of unity");
    const u64 ipsi = hch::invmod(psi, q);
    pw[0] = ipw[0] = 1;
    for (int k = 1; k < n; ++k) {
      pw[k] = hch::mulmod(pw[k - 1], psi, q);
      ipw[k] = hch::mulmod(ipw[k - 1], ipsi, q);
    }
    for (int k = 0; k < n; ++k) {
      const int r = hch::bit_reverse(k, logn);
      const size_t o = 2 * ((size_t)c * n + k);
      fwd[o] = pw[r];
      fwd[o + 1] = hch::shoup_of(pw[r], q);
      inv[o] = ipw[r];
      inv[o + 1] = hch::shoup_of(ipw[r], q);
    }
    ninv[c] = hch::invmod((u64)n % q, q);
    ninv_sh[c] = hch::shoup_of(ninv[c], q);
    const u64 r64 = (u64)((((unsigned __int128)1) << 64) % q);
    u64 qinv = q;  // Newton's iteration for q^{-1} mod 2^64 (q odd: q q = 1 mod 8)
    for (int it = 0; it < 5; ++it) qinv *= 2 - q * qinv;
    mods[c] = DMod{q, r64, hch::shoup_of(r64, q), hch::shoup_of(1, q), qinv};
  }
  auto put = [&](const void* src, size_t bytes) {
    void* d = nullptr;
    HC_CUDA(cudaMalloc(&d, bytes));
    ctx->owned.push_back(d);
    HC_CUDA(cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice));
    return d;
  };
  const size_t tb = 2 * (size_t)nc * n * sizeof(u64);
  ctx->tab.fwd2 = (const ulonglong2*)put(fwd.data(), tb);
  ctx->tab.inv2 = (const ulonglong2*)put(inv.data(), tb);
  ctx->tab.ninv = (const u64*)put(ninv.data(), nc * sizeof(u64));
  ctx->tab.ninv_sh = (const u64*)put(ninv_sh.data(), nc * sizeof(u64));
  ctx->tab.mods = (const DMod*)put(mods.data(), nc * sizeof(DMod));
  ctx->tab.log_n = logn;

  // key-switching / rescale constants
  const int L = P.L, alpha = P.alpha;
  std::vector<u64> ks;
  ctx->lv.assign(L + 1, LevelConsts{});
  for (int l = 0; l <= L; ++l) {
    LevelConsts& lc = ctx->lv[l];
    const int nq = l + 1, next = nq + alpha;
    lc.dnum = (nq + alpha - 1) / alpha;
    std::vector<int> emap(next);
    for (int s = 0; s < next; ++s) emap[s] = s < nq ? s : L + 1 + (s - nq);
    for (int j = 0; j < lc.dnum; ++j) {
      const int d0 = j * alpha, d1 = std::min(d0 + alpha, nq), ns = d1 - d0;
      lc.modup_off.push_back((int)ks.size());
      std::vector<u64> hinv(ns);
      for (int i = 0; i < ns; ++i) {
        const u64 qi = P.chain[d0 + i];
        u64 prod = 1;
        for (int k = 0; k < ns; ++k)
          if (k != i) prod = hch::mulmod(prod, P.chain[d0 + k] % qi, qi);
        // N^{-1} folded in: the conversion's input comes from an inverse NTT
        // without its N^{-1} factor
        hinv[i] = hch::mulmod(hch::invmod(prod, qi), hch::invmod((u64)P.n % qi, qi), qi);
      }
      for (int i = 0; i < ns; ++i) ks.push_back(hinv[i]);
      for (int i = 0; i < ns; ++i) ks.push_back(hch::shoup_of(hinv[i], P.chain[d0 + i]));
      for (int s = 0; s < next; ++s) {
        const u64 t = P.chain[emap[s]];
        for (int i = 0; i < ns; ++i) {
          u64 prod = 1 % t;
          for (int k = 0; k < ns; ++k)
            if (k != i) prod = hch::mulmod(prod, P.chain[d0 + k] % t, t);
          ks.push_back(prod);
        }
      }
    }
    if (l >= 1) {
      lc.rescale_off = (int)ks.size();
      const u64 ql = P.chain[l];
      std::vector<u64> inv_l(l);
      for (int i = 0; i < l; ++i) inv_l[i] = hch::invmod(ql % P.chain[i], P.chain[i]);
      for (int i = 0; i < l; ++i) ks.push_back(inv_l[i]);
      for (int i = 0; i < l; ++i) ks.push_back(hch::shoup_of(inv_l[i], P.chain[i]));
      // the coefficient-form relinearise + rescale tail: N^{-1} q_l^{-1}
      std::vector<u64> nq(l);
      for (int i = 0; i < l; ++i) nq[i] = hch::mulmod(hch::invmod((u64)P.n % P.chain[i], P.chain[i]), inv_l[i], P.chain[i]);
      for (int i = 0; i < l; ++i) ks.push_back(nq[i]);
      for (int i = 0; i < l; ++i) ks.push_back(hch::shoup_of(nq[i], P.chain[i]));
    }
  }
  ctx->moddown_off = (int)ks.size();
  {
    std::vector<u64> hinv(alpha);
    for (int k = 0; k < alpha; ++k) {
      const u64 pk = P.chain[L + 1 + k];
      u64 prod = 1;
      for (int m = 0; m < alpha; ++m)
        if (m != k) prod = hch::mulmod(prod, P.chain[L + 1 + m] % pk, pk);
      hinv[k] = hch::mulmod(hch::invmod(prod, pk), hch::invmod((u64)P.n % pk, pk), pk);  // N^{-1} folded in
    }
    for (int k = 0; k < alpha; ++k) ks.push_back(hinv[k]);
    for (int k = 0; k < alpha; ++k) ks.push_back(hch::shoup_of(hinv[k], P.chain[L + 1 + k]));
    // (P/p_k) P^{-1} = p_k^{-1} mod q_i: the conversion's output comes out
    // already multiplied by P^{-1}, matching the key product's Q limbs (the
    // switching keys' Q limbs carry P^{-1}, see key_scale), so ModDown needs
    // no multiplication by P^{-1} of its own
    for (int i = 0; i <= L; ++i) {
      const u64 qi = P.chain[i];
      for (int k = 0; k < alpha; ++k) ks.push_back(hch::invmod(P.chain[L + 1 + k] % qi, qi));
    }
  }
  ctx->ks_dev = (u64*)put(ks.data(), ks.size() * sizeof(u64));
  // ext maps per level followed by an identity map of HC_MAX_CHAIN entries
  const int W = L + 1 + alpha;
  std::vector<int> maps((size_t)(L + 1) * W + HC_MAX_CHAIN, 0);
  for (int l = 0; l <= L; ++l)
    for (int s = 0; s < l + 1 + alpha; ++s) maps[(size_t)l * W + s] = s <= l ? s : L + 1 + (s - l - 1);
  for (int i = 0; i < HC_MAX_CHAIN; ++i) maps[(size_t)(L + 1) * W + i] = i;
  ctx->ext_map = (int*)put(maps.data(), maps.size() * sizeof(int));
  // per (level, digit): the ext slots outside the digit, in order
  std::vector<int> slots;
  for (int l = 0; l <= L; ++l) {
    LevelConsts& lc = ctx->lv[l];
    lc.modup_slots_off.clear();
    for (int j = 0; j < lc.dnum; ++j) {
      const int d0 = j * alpha, d1 = std::min(d0 + alpha, l + 1);
      lc.modup_slots_off.push_back((int)slots.size());
      for (int t = 0; t < l + 1 + alpha; ++t)
        if (t < d0 || t >= d1) slots.push_back(t);
    }
  }
  ctx->modup_slots = (int*)put(slots.data(), std::max<size_t>(1, slots.size()) * sizeof(int));
}
}  // namespace

extern "C" int hc_ctx_create(const hc_params* p, int device, void* stream, const hc_allocator* alloc, hc_ctx** out) {
  hc_ctx* ctx = nullptr;
  int rc = guard(nullptr, [&] {
    HC_CHECK(p && out, HC_ERR_INVALID, "null argument");
    HC_CUDA(cudaSetDevice(device));
    ctx = new hc_ctx();
    ctx->P = *p;
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    if (!alloc) {
      // keep freed pool memory cached instead of returning it at every sync
      cudaMemPool_t pool;
      HC_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
      uint64_t keep_all = UINT64_MAX;
      HC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep_all));
    }
    if (alloc) {
      HC_CHECK(alloc->alloc && alloc->free, HC_ERR_INVALID, "allocator needs alloc and free");
      ctx->alloc = *alloc;
      ctx->user_alloc = true;
    }
    build_tables(ctx);
    *out = ctx;
  });
  if (rc != HC_OK && ctx) hc_ctx_destroy(ctx);
  return rc;
}

extern "C" void hc_ctx_destroy(hc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  recycle_events(ctx);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  for (void* d : ctx->owned) cudaFree(d);
  for (cudaStream_t st : ctx->aux_streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaStream_t st : ctx->copy_streams)
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  if (ctx->flag_stream) cudaStreamDestroy(ctx->flag_stream);
  delete ctx;
}

extern "C" int hc_sync(hc_ctx* ctx) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] { HC_CUDA(cudaStreamSynchronize(ctx->stream)); });
}

extern "C" const char* hc_last_error(const hc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" uint64_t hc_kernel_launches(const hc_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" int hc_profile_enable(hc_ctx* ctx, int on) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    if (on) {
      HC_CUDA(cudaStreamSynchronize(ctx->stream));
      recycle_events(ctx);
    }
    ctx->prof = on != 0;
  });
}

extern "C" int hc_profile_kernel(hc_ctx* ctx, const char* name, uint64_t* launches, double* total_ms,
                                 uint64_t* units) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(name && launches && total_ms && units, HC_ERR_INVALID, "null argument");
    *launches = 0;
    *total_ms = 0;
    *units = 0;
    auto it = ctx->prof_events.find(name);
    if (it == ctx->prof_events.end()) return;
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
    double ms = 0;
    for (auto& pr : it->second) {
      float t = 0;
      HC_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
      ms += t;
    }
    *launches = it->second.size();
    *total_ms = ms;
    *units = ctx->prof_units[name];
  });
}

extern "C" int hc_profile_host_timeline(const hc_ctx* ctx, double* out, int cap) {
  if (!ctx) return HC_ERR_INVALID;
  const int n = (int)ctx->host_timeline.size();
  if (out)
    for (int i = 0; i < n && i < cap; ++i) out[i] = ctx->host_timeline[i];
  return n;
}

extern "C" int hc_profile_names(hc_ctx* ctx, char* buf, size_t cap) {
  if (!ctx || !buf || cap == 0) return HC_ERR_INVALID;
  std::string all;
  for (auto& kv : ctx->prof_events) {
    if (!all.empty()) all += ",";
    all += kv.first;
  }
  if (all.size() + 1 > cap) return HC_ERR_INVALID;
  std::memcpy(buf, all.c_str(), all.size() + 1);
  return HC_OK;
}

// =====================================================================
// Keys
// =====================================================================
namespace {
const u64 TAG_S = 1, TAG_PK_A = 2, TAG_PK_E = 3;
u64 tag_swk_a(int j, u64 g) { return (g << 16) | (u64)(0x100 + 2 * j); }
u64 tag_swk_e(int j, u64 g) { return (g << 16) | (u64)(0x101 + 2 * j); }
u64 tag_enc(u64 nonce, int which) { return (1ull << 63) | (nonce << 2) | (u64)which; }

u64 galois_elt(const hc_params& P, long long r) {
  const long long K = P.n / 2;
  long long rr = r % K;
  if (rr < 0) rr += K;
  return hch::powmod(5, (u64)rr, 2 * (u64)P.n);
}

// Multiplies every limb of a switching key ([npoly][chain][N]) by 2^64 mod q
// (into Montgomery form: the key product reduces its sums with one
// Montgomery reduction) and its limbs of Q (t <= L) also by P^{-1} mod q_t
// (ModDown's division by P, folded into the key product), or by the inverse
// of that (back to the plain key), in place.
void key_scale(hc_ctx* ctx, u64* key, int npoly, bool inverse, std::vector<BufPtr>& keep) {
  const hc_params& P = ctx->P;
  const int nc = P.nchain();
  std::vector<u64> sc(2 * nc);
  for (int t = 0; t < nc; ++t) {
    const u64 q = P.chain[t];
    u64 f = (u64)(((unsigned __int128)1 << 64) % q);
    if (t <= P.L) {
      u64 pm = 1;
      for (int k = 0; k < P.alpha; ++k) pm = hch::mulmod(pm, P.chain[P.L + 1 + k] % q, q);
      f = hch::mulmod(f, hch::invmod(pm, q), q);
    }
    sc[t] = inverse ? hch::invmod(f, q) : f;
    sc[nc + t] = hch::shoup_of(sc[t], q);
  }
  std::vector<CtRef> rk{CtRef{key, (u64)nc * ctx->P.n}};
  const CtRef* dk = refs_dev(ctx, rk, keep);
  launch_scalar(ctx, false, dk, dk, 1, npoly, nc, upload(ctx, sc, keep));
}

// Switching key for s' (NTT form over the whole chain) -> s.
void make_switch_key(hc_ctx* ctx, const u64* s_ntt, const u64* sp_ntt, u64 seed, u64 g, SwitchKeyDev& out) {
  const hc_params& P = ctx->P;
  const int nc = P.nchain(), n = P.n;
  const size_t poly = (size_t)nc * n;
  out.buf = ctx->buffer(2 * poly * P.dnum);
  std::vector<BufPtr> keep;
  std::vector<int> ids(nc);
  std::iota(ids.begin(), ids.end(), 0);
  const int* idd = ids_dev(ctx, ids, keep);
  BufPtr tmp = ctx->buffer(poly);
  keep.push_back(tmp);
  u64 Pmod[HC_MAX_CHAIN];
  for (int t = 0; t < nc; ++t) {
    u64 pr = 1 % P.chain[t];
    for (int k = 0; k < P.alpha; ++k) pr = hch::mulmod(pr, P.chain[P.L + 1 + k] % P.chain[t], P.chain[t]);
    Pmod[t] = pr;
  }
  for (int j = 0; j < P.dnum; ++j) {
    u64* b = out.buf->ptr + (size_t)(2 * j) * poly;
    u64* a = b + poly;
    launch_sample_uniform(ctx, seed, tag_swk_a(j, g), a, idd, nc);
    launch_ntt(ctx, limbset_base(a, 0, 0, 1, nc, 0, nullptr), 1, false);
    launch_sample_gauss(ctx, seed, tag_swk_e(j, g), b, idd, nc);
    launch_ntt(ctx, limbset_base(b, 0, 0, 1, nc, 0, nullptr), 1, false);
    // b = e - a s + P [t in digit j] s'
    std::vector<CtRef> rb{CtRef{b, 0}}, ra{CtRef{a, 0}}, rs{CtRef{const_cast<u64*>(s_ntt), 0}},
        rt{CtRef{tmp->ptr, 0}}, rsp{CtRef{const_cast<u64*>(sp_ntt), 0}};
    const CtRef *db = refs_dev(ctx, rb, keep), *da = refs_dev(ctx, ra, keep), *ds = refs_dev(ctx, rs, keep),
                *dt = refs_dev(ctx, rt, keep), *dsp = refs_dev(ctx, rsp, keep);
    launch_ew(ctx, 2, dt, da, ds, 1, 1, nc);
    launch_ew(ctx, 1, db, db, dt, 1, 1, nc);
    std::vector<u64> sc(2 * nc, 0);
    const int d0 = j * P.alpha, d1 = std::min(d0 + P.alpha, P.L + 1);
    for (int t = 0; t < nc; ++t) {
      const u64 v = (t >= d0 && t < d1) ? Pmod[t] : 0;
      sc[t] = v;
      sc[nc + t] = hch::shoup_of(v, P.chain[t]);
    }
    launch_scalar(ctx, false, dt, dsp, 1, 1, nc, upload(ctx, sc, keep));
    launch_ew(ctx, 0, db, db, dt, 1, 1, nc);
  }
  // stored in Montgomery form, the limbs of Q times P^{-1}
  key_scale(ctx, out.buf->ptr, 2 * P.dnum, false, keep);
  HC_CUDA(cudaStreamSynchronize(ctx->stream));
}
}  // namespace

extern "C" int hc_keygen(hc_ctx* ctx, uint64_t seed, const int32_t* rot_steps, int n_rot, hc_sk** sk_out,
                         hc_pk** pk_out, hc_evk** evk_out) {
  if (!ctx) return HC_ERR_INVALID;
  hc_sk* sk = nullptr;
  hc_pk* pk = nullptr;
  hc_evk* evk = nullptr;
  int rc = guard(ctx, [&] {
    HC_CHECK(sk_out && pk_out && evk_out && (n_rot == 0 || rot_steps), HC_ERR_INVALID, "null argument");
    const hc_params& P = ctx->P;
    const int nc = P.nchain(), n = P.n, nq = P.L + 1;
    std::vector<BufPtr> keep;
    std::vector<int> ids(nc);
    std::iota(ids.begin(), ids.end(), 0);
    const int* idd = ids_dev(ctx, ids, keep);
    sk = new hc_sk{ctx, ctx->buffer((size_t)nc * n), {}};
    launch_sample_ternary(ctx, seed, TAG_S, sk->s_ntt->ptr, idd, nc);
    {
      // keep the ternary coefficients on the host for export
      std::vector<u64> l0(n);
      HC_CUDA(cudaMemcpyAsync(l0.data(), sk->s_ntt->ptr, n * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
      HC_CUDA(cudaStreamSynchronize(ctx->stream));
      sk->s_coeff.resize(n);
      for (int i = 0; i < n; ++i) sk->s_coeff[i] = l0[i] == 0 ? 0 : (l0[i] == 1 ? 1 : -1);
    }
    launch_ntt(ctx, limbset_base(sk->s_ntt->ptr, 0, 0, 1, nc, 0, nullptr), 1, false);
    // public key over q_0..q_L
    pk = new hc_pk{ctx, ctx->buffer(2 * (size_t)nq * n)};
    u64* b = pk->buf->ptr;
    u64* a = b + (size_t)nq * n;
    launch_sample_uniform(ctx, seed, TAG_PK_A, a, idd, nq);
    launch_ntt(ctx, limbset_base(a, 0, 0, 1, nq, 0, nullptr), 1, false);
    launch_sample_gauss(ctx, seed, TAG_PK_E, b, idd, nq);
    launch_ntt(ctx, limbset_base(b, 0, 0, 1, nq, 0, nullptr), 1, false);
    BufPtr tmp = ctx->buffer((size_t)nc * n);
    keep.push_back(tmp);
    std::vector<CtRef> rb{CtRef{b, 0}}, ra{CtRef{a, 0}}, rs{CtRef{sk->s_ntt->ptr, 0}}, rt{CtRef{tmp->ptr, 0}};
    const CtRef *db = refs_dev(ctx, rb, keep), *da = refs_dev(ctx, ra, keep), *ds = refs_dev(ctx, rs, keep),
                *dt = refs_dev(ctx, rt, keep);
    launch_ew(ctx, 2, dt, da, ds, 1, 1, nq);
    launch_ew(ctx, 1, db, db, dt, 1, 1, nq);
    // relinearisation key: s' = s^2
    evk = new hc_evk{ctx, {}, {}};
    BufPtr s2 = ctx->buffer((size_t)nc * n);
    keep.push_back(s2);
    std::vector<CtRef> rs2{CtRef{s2->ptr, 0}};
    launch_ew(ctx, 2, refs_dev(ctx, rs2, keep), ds, ds, 1, 1, nc);
    make_switch_key(ctx, sk->s_ntt->ptr, s2->ptr, seed, 0, evk->relin);
    for (int i = 0; i < n_rot; ++i) {
      const u64 g = galois_elt(P, rot_steps[i]);
      if (g == 1 || evk->galois.count(g)) continue;
      BufPtr sg = ctx->buffer((size_t)nc * n);
      std::vector<BufPtr> k2;
      std::vector<CtRef> rsg{CtRef{sg->ptr, 0}};
      launch_automorph(ctx, refs_dev(ctx, rsg, k2), ds, 1, 1, nc, g);
      make_switch_key(ctx, sk->s_ntt->ptr, sg->ptr, seed, g, evk->galois[g]);
    }
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
    *sk_out = sk;
    *pk_out = pk;
    *evk_out = evk;
  });
  if (rc != HC_OK) {
    delete sk;
    delete pk;
    delete evk;
  }
  return rc;
}

extern "C" void hc_sk_destroy(hc_sk* k) { delete k; }
extern "C" void hc_pk_destroy(hc_pk* k) { delete k; }
extern "C" void hc_evk_destroy(hc_evk* k) { delete k; }

namespace {
// Coefficient-form copy of `npoly` polys of `nl` limbs (poly stride ps) to host.
void export_coeff(hc_ctx* ctx, const u64* src, u64 ps, int npoly, int nl, const int* pmap, u64* host) {
  const int n = ctx->P.n;
  std::vector<BufPtr> keep;
  BufPtr tmp = ctx->buffer((size_t)npoly * nl * n);
  keep.push_back(tmp);
  for (int k = 0; k < npoly; ++k)
    HC_CUDA(cudaMemcpyAsync(tmp->ptr + (size_t)k * nl * n, src + k * ps, (size_t)nl * n * sizeof(u64),
                            cudaMemcpyDeviceToDevice, ctx->stream));
  launch_ntt(ctx, limbset_base(tmp->ptr, 0, (u64)nl * n, npoly, nl, 0, pmap), 1, true);
  HC_CUDA(cudaMemcpyAsync(host, tmp->ptr, (size_t)npoly * nl * n * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
  HC_CUDA(cudaStreamSynchronize(ctx->stream));
}
}  // namespace

extern "C" int hc_sk_export(hc_ctx* ctx, const hc_sk* sk, int8_t* out, size_t n) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(sk && out && n >= (size_t)ctx->P.n, HC_ERR_INVALID, "bad arguments");
    std::copy(sk->s_coeff.begin(), sk->s_coeff.end(), out);
  });
}

extern "C" int hc_pk_export(hc_ctx* ctx, const hc_pk* pk, uint64_t* out, size_t cap) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    const int nq = ctx->P.L + 1;
    HC_CHECK(pk && out && cap >= 2 * (size_t)nq * ctx->P.n, HC_ERR_INVALID, "bad arguments");
    export_coeff(ctx, pk->buf->ptr, (u64)nq * ctx->P.n, 2, nq, nullptr, (u64*)out);
  });
}

extern "C" int hc_evk_export(hc_ctx* ctx, const hc_evk* evk, uint64_t g, uint64_t* out, size_t cap) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    const int nc = ctx->P.nchain();
    const size_t poly = (size_t)nc * ctx->P.n;
    HC_CHECK(evk && out && cap >= 2 * poly * ctx->P.dnum, HC_ERR_INVALID, "bad arguments");
    const SwitchKeyDev* k = nullptr;
    if (g == 1) k = &evk->relin;
    else {
      auto it = evk->galois.find(g);
      HC_CHECK(it != evk->galois.end(), HC_ERR_NO_KEY, "no such Galois key");
      k = &it->second;
    }
    // back from the stored form (Montgomery, the Q limbs times P^{-1}), then
    // as any other polynomial
    std::vector<BufPtr> keep;
    BufPtr plain = ctx->buffer(2 * poly * ctx->P.dnum);
    keep.push_back(plain);
    HC_CUDA(cudaMemcpyAsync(plain->ptr, k->buf->ptr, 2 * poly * ctx->P.dnum * sizeof(u64), cudaMemcpyDeviceToDevice,
                            ctx->stream));
    key_scale(ctx, plain->ptr, 2 * ctx->P.dnum, true, keep);
    export_coeff(ctx, plain->ptr, poly, 2 * ctx->P.dnum, nc, nullptr, (u64*)out);
  });
}

// =====================================================================
// Plaintexts
// =====================================================================
namespace {
hc_pt* pt_from_signed(hc_ctx* ctx, const std::vector<int64_t>& coeffs, int level, double scale) {
  const int n = ctx->P.n, nl = level + 1;
  std::vector<BufPtr> keep;
  BufPtr src = ctx->buffer(n);
  keep.push_back(src);
  HC_CUDA(cudaMemcpyAsync(src->ptr, coeffs.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
  auto* pt = new hc_pt{ctx, ctx->buffer((size_t)nl * n), nullptr, level, scale};
  pt->data = pt->buf->ptr;
  launch_reduce_signed(ctx, (const int64_t*)src->ptr, pt->data, ident_map(ctx), nl);
  launch_ntt(ctx, limbset_base(pt->data, 0, 0, 1, nl, 0, nullptr), 1, false);
  HC_CUDA(cudaStreamSynchronize(ctx->stream));  // host source goes out of scope
  return pt;
}
}  // namespace

extern "C" int hc_encode(hc_ctx* ctx, const double* re, const double* im, size_t n, double scale, int level,
                         hc_pt** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(out && (re || n == 0), HC_ERR_INVALID, "null argument");
    HC_CHECK(n <= (size_t)ctx->P.n / 2, HC_ERR_INVALID, "more values than slots");
    HC_CHECK(level >= 0 && level <= ctx->P.L, HC_ERR_INVALID, "bad level");
    HC_CHECK(scale > 0, HC_ERR_INVALID, "bad scale");
    std::vector<double> c;
    hch::encode_coeffs(re, im, n, ctx->P.log_n, scale, c);
    std::vector<int64_t> m(c.size());
    for (size_t i = 0; i < c.size(); ++i) {
      bool ok = false;
      m[i] = hch::round_half_away(c[i], &ok);
      HC_CHECK(ok, HC_ERR_INVALID, "encoded coefficient out of range");
    }
    *out = pt_from_signed(ctx, m, level, scale);
  });
}

extern "C" int hc_pt_from_coeffs(hc_ctx* ctx, const int64_t* coeffs, size_t n, int level, double scale, hc_pt** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(out && coeffs && n == (size_t)ctx->P.n, HC_ERR_INVALID, "need N coefficients");
    HC_CHECK(level >= 0 && level <= ctx->P.L, HC_ERR_INVALID, "bad level");
    std::vector<int64_t> m(coeffs, coeffs + n);
    for (auto v : m) HC_CHECK(v < (1LL << 62) && v > -(1LL << 62), HC_ERR_INVALID, "coefficient out of range");
    *out = pt_from_signed(ctx, m, level, scale);
  });
}

extern "C" int hc_pt_export(hc_ctx* ctx, const hc_pt* pt, uint64_t* out, size_t cap) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(pt && out && cap >= (size_t)(pt->level + 1) * ctx->P.n, HC_ERR_INVALID, "bad arguments");
    export_coeff(ctx, pt->data, 0, 1, pt->level + 1, nullptr, (u64*)out);
  });
}

extern "C" int hc_decode(hc_ctx* ctx, const hc_pt* pt, double* re, double* im, size_t n) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(pt && re, HC_ERR_INVALID, "null argument");
    const int nl = pt->level + 1, N = ctx->P.n;
    std::vector<u64> res((size_t)nl * N);
    export_coeff(ctx, pt->data, 0, 1, nl, nullptr, res.data());
    std::vector<double> c;
    hch::crt_centred_to_double(res.data(), ctx->P.chain.data(), nl, N, c);
    hch::decode_slots(c, ctx->P.log_n, pt->scale, re, im, std::min(n, (size_t)N / 2));
  });
}

extern "C" int hc_pt_level(const hc_pt* pt) { return pt ? pt->level : -1; }
extern "C" double hc_pt_scale(const hc_pt* pt) { return pt ? pt->scale : 0.0; }
extern "C" void hc_pt_destroy(hc_pt* pt) { delete pt; }

// =====================================================================
// Encrypt / decrypt / import / export
// =====================================================================
extern "C" int hc_encrypt(hc_ctx* ctx, const hc_pk* pk, const hc_pt* pt, uint64_t seed, uint64_t nonce, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(pk && pt && out, HC_ERR_INVALID, "null argument");
    HC_CHECK(nonce < (1ull << 61), HC_ERR_INVALID, "nonce must be < 2^61");
    const int n = ctx->P.n, nl = pt->level + 1, nq = ctx->P.L + 1;
    std::vector<BufPtr> keep;
    BufPtr rnd = ctx->buffer(3 * (size_t)nl * n);
    keep.push_back(rnd);
    u64* v = rnd->ptr;
    u64* e0 = v + (size_t)nl * n;
    u64* e1 = e0 + (size_t)nl * n;
    launch_sample_ternary(ctx, seed, tag_enc(nonce, 0), v, ident_map(ctx), nl);
    launch_sample_gauss(ctx, seed, tag_enc(nonce, 1), e0, ident_map(ctx), nl);
    launch_sample_gauss(ctx, seed, tag_enc(nonce, 2), e1, ident_map(ctx), nl);
    launch_ntt(ctx, limbset_base(v, (u64)nl * n, 0, 1, nl, 0, nullptr), 3, false);
    hc_ct* c = new_ct(ctx, pt->level, 1, pt->scale);
    std::vector<CtRef> r0{CtRef{c->data, 0}}, r1{CtRef{c->data + c->stride, 0}}, rv{CtRef{v, 0}},
        re0{CtRef{e0, 0}}, re1{CtRef{e1, 0}}, rb{CtRef{pk->buf->ptr, 0}}, ra{CtRef{pk->buf->ptr + (size_t)nq * n, 0}},
        rm{CtRef{pt->data, 0}};
    const CtRef *d0 = refs_dev(ctx, r0, keep), *d1 = refs_dev(ctx, r1, keep), *dv = refs_dev(ctx, rv, keep),
                *de0 = refs_dev(ctx, re0, keep), *de1 = refs_dev(ctx, re1, keep), *db = refs_dev(ctx, rb, keep),
                *da = refs_dev(ctx, ra, keep), *dm = refs_dev(ctx, rm, keep);
    launch_ew(ctx, 2, d0, dv, db, 1, 1, nl);
    launch_ew(ctx, 0, d0, d0, de0, 1, 1, nl);
    launch_ew(ctx, 0, d0, d0, dm, 1, 1, nl);
    launch_ew(ctx, 2, d1, dv, da, 1, 1, nl);
    launch_ew(ctx, 0, d1, d1, de1, 1, 1, nl);
    *out = c;
  });
}

extern "C" int hc_decrypt(hc_ctx* ctx, const hc_sk* sk, const hc_ct* ct, hc_pt** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(sk && ct && out, HC_ERR_INVALID, "null argument");
    check_ct(ctx, ct);
    const int n = ctx->P.n, nl = ct->level + 1;
    std::vector<BufPtr> keep;
    auto* pt = new hc_pt{ctx, ctx->buffer((size_t)nl * n), nullptr, ct->level, ct->scale};
    pt->data = pt->buf->ptr;
    BufPtr tmp = ctx->buffer((size_t)2 * nl * n);
    keep.push_back(tmp);
    u64* t = tmp->ptr;
    u64* sp = t + (size_t)nl * n;
    std::vector<CtRef> rm{CtRef{pt->data, 0}}, rt{CtRef{t, 0}}, rs{CtRef{sk->s_ntt->ptr, 0}}, rsp{CtRef{sp, 0}};
    const CtRef *dm = refs_dev(ctx, rm, keep), *dt = refs_dev(ctx, rt, keep), *ds = refs_dev(ctx, rs, keep),
                *dsp = refs_dev(ctx, rsp, keep);
    std::vector<CtRef> rc0{CtRef{ct->data, 0}};
    launch_ew(ctx, 3, dm, refs_dev(ctx, rc0, keep), nullptr, 1, 1, nl);
    launch_ew(ctx, 3, dsp, ds, nullptr, 1, 1, nl);
    for (int k = 1; k <= ct->degree; ++k) {
      std::vector<CtRef> rck{CtRef{ct->data + k * ct->stride, 0}};
      launch_ew(ctx, 2, dt, refs_dev(ctx, rck, keep), dsp, 1, 1, nl);
      launch_ew(ctx, 0, dm, dm, dt, 1, 1, nl);
      if (k < ct->degree) launch_ew(ctx, 2, dsp, dsp, ds, 1, 1, nl);
    }
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = pt;
  });
}

extern "C" int hc_ct_export(hc_ctx* ctx, const hc_ct* ct, uint64_t* out, size_t cap, hc_ct_meta* meta) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, ct);
    const size_t words = (size_t)(ct->degree + 1) * (ct->level + 1) * ctx->P.n;
    HC_CHECK(out && cap >= words, HC_ERR_INVALID, "output buffer too small");
    export_coeff(ctx, ct->data, ct->stride, ct->degree + 1, ct->level + 1, nullptr, (u64*)out);
    if (meta) *meta = hc_ct_meta{ct->level, ct->degree, ct->scale};
  });
}

extern "C" int hc_ct_import(hc_ctx* ctx, const uint64_t* host, const hc_ct_meta* meta, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(host && meta && out, HC_ERR_INVALID, "null argument");
    HC_CHECK(meta->level >= 0 && meta->level <= ctx->P.L && (meta->degree == 1 || meta->degree == 2),
             HC_ERR_INVALID, "bad metadata");
    hc_ct* c = new_ct(ctx, meta->level, meta->degree, meta->scale);
    std::unique_ptr<hc_ct> hold(c);
    const size_t words = (size_t)(meta->degree + 1) * (meta->level + 1) * ctx->P.n;
    HC_CUDA(cudaMemcpyAsync(c->data, host, words * sizeof(u64), cudaMemcpyHostToDevice, ctx->stream));
    std::vector<BufPtr> keep;
    BufPtr flag = ctx->buffer(1);
    keep.push_back(flag);
    HC_CUDA(cudaMemsetAsync(flag->ptr, 0, sizeof(u64), ctx->stream));
    launch_check_range(ctx, c->data, meta->degree + 1, meta->level + 1, c->stride, (unsigned long long*)flag->ptr);
    u64 bad = 0;
    HC_CUDA(cudaMemcpyAsync(&bad, flag->ptr, sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
    HC_CHECK(bad == 0, HC_ERR_INVALID, "imported residue not below its prime");
    launch_ntt(ctx, limbset_base(c->data, 0, c->stride, meta->degree + 1, meta->level + 1, 0, nullptr), 1, false);
    *out = hold.release();
  });
}

extern "C" int hc_ct_export_eval(hc_ctx* ctx, const hc_ct* ct, uint64_t* out, size_t cap, hc_ct_meta* meta) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, ct);
    const int np = ct->degree + 1, nl = ct->level + 1;
    const size_t limbs = (size_t)nl * ctx->P.n;
    HC_CHECK(out && cap >= np * limbs, HC_ERR_INVALID, "output buffer too small");
    for (int k = 0; k < np; ++k)  // each polynomial's limbs are contiguous on the device
      HC_CUDA(cudaMemcpyAsync(out + k * limbs, ct->data + k * ct->stride, limbs * sizeof(u64), cudaMemcpyDeviceToHost,
                              ctx->stream));
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
    if (meta) *meta = hc_ct_meta{ct->level, ct->degree, ct->scale};
  });
}

extern "C" int hc_ct_import_eval(hc_ctx* ctx, const uint64_t* host, const hc_ct_meta* meta, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(host && meta && out, HC_ERR_INVALID, "null argument");
    HC_CHECK(meta->level >= 0 && meta->level <= ctx->P.L && (meta->degree == 1 || meta->degree == 2),
             HC_ERR_INVALID, "bad metadata");
    hc_ct* c = new_ct(ctx, meta->level, meta->degree, meta->scale);
    std::unique_ptr<hc_ct> hold(c);
    const size_t words = (size_t)(meta->degree + 1) * (meta->level + 1) * ctx->P.n;
    HC_CUDA(cudaMemcpyAsync(c->data, host, words * sizeof(u64), cudaMemcpyHostToDevice, ctx->stream));
    std::vector<BufPtr> keep;
    BufPtr flag = ctx->buffer(1);
    keep.push_back(flag);
    HC_CUDA(cudaMemsetAsync(flag->ptr, 0, sizeof(u64), ctx->stream));
    launch_check_range(ctx, c->data, meta->degree + 1, meta->level + 1, c->stride, (unsigned long long*)flag->ptr);
    u64 bad = 0;
    HC_CUDA(cudaMemcpyAsync(&bad, flag->ptr, sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
    HC_CHECK(bad == 0, HC_ERR_INVALID, "imported residue not below its prime");
    *out = hold.release();
  });
}

extern "C" int hc_ct_import_batch(hc_ctx* ctx, const uint64_t* const* host, const hc_ct_meta* metas, int n,
                                  hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  std::vector<hc_ct*> made;
  int rc = guard(ctx, [&] {
    HC_CHECK(n >= 0 && (n == 0 || (host && metas && out)), HC_ERR_INVALID, "null argument");
    if (n == 0) return;
    std::vector<BufPtr> keep;
    BufPtr flag = ctx->buffer(1);
    keep.push_back(flag);
    HC_CUDA(cudaMemsetAsync(flag->ptr, 0, sizeof(u64), ctx->stream));
    for (int i = 0; i < n; ++i) {
      const hc_ct_meta& m = metas[i];
      HC_CHECK(host[i] && m.level >= 0 && m.level <= ctx->P.L && (m.degree == 1 || m.degree == 2), HC_ERR_INVALID,
               "bad metadata");
      hc_ct* c = new_ct(ctx, m.level, m.degree, m.scale);
      made.push_back(c);
      const size_t words = (size_t)(m.degree + 1) * (m.level + 1) * ctx->P.n;
      HC_CUDA(cudaMemcpyAsync(c->data, host[i], words * sizeof(u64), cudaMemcpyHostToDevice, ctx->stream));
      launch_check_range(ctx, c->data, m.degree + 1, m.level + 1, c->stride, (unsigned long long*)flag->ptr);
    }
    u64 bad = 0;
    HC_CUDA(cudaMemcpyAsync(&bad, flag->ptr, sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
    HC_CHECK(bad == 0, HC_ERR_INVALID, "imported residue not below its prime");
    // one forward NTT launch per (level, degree) group
    std::map<std::pair<int, int>, std::vector<CtRef>> groups;
    for (auto* c : made) groups[{c->level, c->degree}].push_back(c->ref());
    for (auto& kv : groups) {
      LimbSet sset{};
      sset.refs = refs_dev(ctx, kv.second, keep);
      sset.npoly = kv.first.second + 1;
      sset.nlimb = kv.first.first + 1;
      launch_ntt(ctx, sset, (int)kv.second.size(), false);
    }
    for (int i = 0; i < n; ++i) out[i] = made[i];
    made.clear();
  });
  for (auto* c : made) delete c;
  return rc;
}

extern "C" int hc_ct_export_batch(hc_ctx* ctx, const hc_ct* const* cts, int n, uint64_t* const* host,
                                  const size_t* cap) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(n >= 0 && (n == 0 || (cts && host && cap)), HC_ERR_INVALID, "null argument");
    if (n == 0) return;
    const int N = ctx->P.n;
    size_t total = 0;
    std::vector<size_t> off(n);
    for (int i = 0; i < n; ++i) {
      check_ct(ctx, cts[i]);
      const size_t words = (size_t)(cts[i]->degree + 1) * (cts[i]->level + 1) * N;
      HC_CHECK(host[i] && cap[i] >= words, HC_ERR_INVALID, "output buffer too small");
      off[i] = total;
      total += words;
    }
    std::vector<BufPtr> keep;
    BufPtr tmp = ctx->buffer(total);
    keep.push_back(tmp);
    std::map<std::pair<int, int>, std::vector<std::pair<CtRef, CtRef>>> groups;  // (src, dst)
    for (int i = 0; i < n; ++i) {
      const hc_ct* c = cts[i];
      const u64 ps = (u64)(c->level + 1) * N;
      groups[{c->level, c->degree}].push_back({c->ref(), CtRef{tmp->ptr + off[i], ps}});
    }
    for (auto& kv : groups) {
      std::vector<CtRef> src, dst;
      for (auto& pr : kv.second) {
        src.push_back(pr.first);
        dst.push_back(pr.second);
      }
      LimbSet in{}, out{};
      in.refs = refs_dev(ctx, src, keep);
      out.refs = refs_dev(ctx, dst, keep);
      in.npoly = out.npoly = kv.first.second + 1;
      in.nlimb = out.nlimb = kv.first.first + 1;
      launch_ntt_from(ctx, out, &in, (int)src.size(), true);
    }
    for (int i = 0; i < n; ++i) {
      const size_t words = (size_t)(cts[i]->degree + 1) * (cts[i]->level + 1) * N;
      HC_CUDA(cudaMemcpyAsync(host[i], tmp->ptr + off[i], words * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    }
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

extern "C" int hc_ct_meta_of(const hc_ct* ct, hc_ct_meta* meta) {
  if (!ct || !meta) return HC_ERR_INVALID;
  *meta = hc_ct_meta{ct->level, ct->degree, ct->scale};
  return HC_OK;
}

extern "C" void hc_ct_destroy(hc_ct* ct) { delete ct; }

// =====================================================================
// Arithmetic
// =====================================================================
namespace {
int add_sub(hc_ctx* ctx, const hc_ct* x, const hc_ct* y, hc_ct** out, int op) {
  return guard(ctx, [&] {
    check_ct(ctx, x);
    check_ct(ctx, y);
    HC_CHECK(out, HC_ERR_INVALID, "null output");
    HC_CHECK(x->level == y->level, HC_ERR_LEVEL_MISMATCH, "operands at different levels");
    HC_CHECK(x->degree == y->degree, HC_ERR_INVALID, "operands of different degree");
    check_scales(x->scale, y->scale);
    hc_ct* c = new_ct(ctx, x->level, x->degree, x->scale);
    std::vector<BufPtr> keep;
    std::vector<CtRef> ro{c->ref()}, rx{x->ref()}, ry{y->ref()};
    launch_ew(ctx, op, refs_dev(ctx, ro, keep), refs_dev(ctx, rx, keep), refs_dev(ctx, ry, keep), 1, x->degree + 1,
              x->level + 1);
    *out = c;
  });
}
}  // namespace

extern "C" int hc_add(hc_ctx* ctx, const hc_ct* x, const hc_ct* y, hc_ct** out) {
  return ctx ? add_sub(ctx, x, y, out, 0) : HC_ERR_INVALID;
}
extern "C" int hc_sub(hc_ctx* ctx, const hc_ct* x, const hc_ct* y, hc_ct** out) {
  return ctx ? add_sub(ctx, x, y, out, 1) : HC_ERR_INVALID;
}

extern "C" int hc_add_const(hc_ctx* ctx, const hc_ct* x, double c, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, x);
    HC_CHECK(out, HC_ERR_INVALID, "null output");
    std::vector<u64> sc;
    constant_residues(ctx, x->level, c * x->scale, false, sc);
    hc_ct* o = new_ct(ctx, x->level, x->degree, x->scale);
    std::vector<BufPtr> keep;
    std::vector<CtRef> ro{o->ref()}, rx{x->ref()};
    launch_scalar(ctx, true, refs_dev(ctx, ro, keep), refs_dev(ctx, rx, keep), 1, x->degree + 1, x->level + 1,
                  upload(ctx, sc, keep));
    *out = o;
  });
}

extern "C" int hc_mul_const(hc_ctx* ctx, const hc_ct* x, double c, double cs, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, x);
    HC_CHECK(out && cs > 0, HC_ERR_INVALID, "bad arguments");
    std::vector<hc_ct*> r = mul_const_cts(ctx, {x}, c, cs);
    *out = r[0];
  });
}

extern "C" int hc_mul(hc_ctx* ctx, const hc_ct* x, const hc_ct* y, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, x);
    check_ct(ctx, y);
    HC_CHECK(out, HC_ERR_INVALID, "null output");
    HC_CHECK(x->degree == 1 && y->degree == 1, HC_ERR_INVALID, "mul needs degree-1 ciphertexts");
    HC_CHECK(x->level == y->level, HC_ERR_LEVEL_MISMATCH, "operands at different levels");
    std::vector<hc_ct*> r = tensor_acc(ctx, {x}, {y}, {0}, {0}, {0, 1}, x->level, x->scale * y->scale);
    *out = r[0];
  });
}

extern "C" int hc_relin(hc_ctx* ctx, const hc_evk* evk, const hc_ct* x, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, x);
    HC_CHECK(evk && out, HC_ERR_INVALID, "null argument");
    HC_CHECK(x->degree == 2, HC_ERR_INVALID, "relin needs a degree-2 ciphertext");
    hc_ct* o = new_ct(ctx, x->level, 1, x->scale);
    std::vector<hc_ct*> os{o};
    relin_batch(ctx, evk, {x}, os);
    *out = o;
  });
}

extern "C" int hc_rescale(hc_ctx* ctx, const hc_ct* x, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, x);
    HC_CHECK(out, HC_ERR_INVALID, "null output");
    HC_CHECK(x->level >= 1, HC_ERR_DEPTH, "no level left to rescale");
    hc_ct* o = new_ct(ctx, x->level - 1, x->degree, x->scale / (double)ctx->P.chain[x->level]);
    std::vector<hc_ct*> os{o};
    rescale_cts(ctx, {x}, os);
    *out = o;
  });
}

extern "C" int hc_drop_to_level(hc_ctx* ctx, const hc_ct* x, int level, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, x);
    HC_CHECK(out && level >= 0 && level <= x->level, HC_ERR_INVALID, "bad level");
    // a view: same polys, fewer limbs
    *out = new hc_ct{ctx, x->buf, x->data, x->stride, level, x->degree, x->scale};
  });
}

namespace {
// The same rotation of many ciphertexts at one level (plain form, bit-identical
// to rotate_one of each): one automorphism launch and one batched key switch.
std::vector<hc_ct*> rotate_batch(hc_ctx* ctx, const hc_evk* evk, const std::vector<const hc_ct*>& xs, int step) {
  const int m = (int)xs.size();
  if (m == 0) return {};
  const int n = ctx->P.n, level = xs[0]->level, nq = level + 1;
  for (auto* c : xs)
    HC_CHECK(c->degree == 1 && c->level == level, HC_ERR_INVALID, "rotate batch needs degree-1 cts at one level");
  const u64 g = galois_elt(ctx->P, step);
  std::vector<hc_ct*> outs = new_cts(ctx, m, level, 1, xs[0]->scale);
  for (int i = 0; i < m; ++i) outs[i]->scale = xs[i]->scale;
  std::vector<BufPtr> keep;
  std::vector<CtRef> xr, orr;
  for (int i = 0; i < m; ++i) {
    xr.push_back(xs[i]->ref());
    orr.push_back(outs[i]->ref());
  }
  if (g == 1) {
    launch_ew(ctx, 3, refs_dev(ctx, orr, keep), refs_dev(ctx, xr, keep), nullptr, m, 2, nq);
    return outs;
  }
  HC_CHECK(evk->galois.count(g), HC_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(step));
  const u64 ps = (u64)nq * n;
  BufPtr tmp = ctx->buffer(2 * ps * m);  // kappa_g of (c0, c1) per item
  keep.push_back(tmp);
  std::vector<CtRef> tr, t1, t0;
  for (int i = 0; i < m; ++i) {
    tr.push_back(CtRef{tmp->ptr + 2 * ps * i, ps});
    t0.push_back(CtRef{tmp->ptr + 2 * ps * i, ps});
    t1.push_back(CtRef{tmp->ptr + 2 * ps * i + ps, ps});
  }
  launch_automorph(ctx, refs_dev(ctx, tr, keep), refs_dev(ctx, xr, keep), m, 2, nq, g);
  keyswitch_batch(ctx, evk->galois.at(g).buf->ptr, level, t1, &t0, nullptr, orr);
  return outs;
}

// Hoisted rotations of m ciphertexts at one level by every step in `steps`:
// one ModUp of all the c1's, then the key product (reading the raised digits
// through the automorphism) and ModDown (adding c0 read through the
// automorphism), each one launch over the (step, ciphertext) items of as
// many steps as the workspace holds, every item with its own Galois element
// and key.  out[step][item];
// the same words as m separate hoisted calls.
std::vector<std::vector<hc_ct*>> rotate_hoisted_batch(hc_ctx* ctx, const hc_evk* evk,
                                                      const std::vector<const hc_ct*>& xs,
                                                      const std::vector<int>& steps) {
  const int total = (int)xs.size();
  std::vector<std::vector<hc_ct*>> outs(steps.size());
  if (total == 0) return outs;
  const int n = ctx->P.n, level = xs[0]->level, nq = level + 1, alpha = ctx->P.alpha;
  const int next = nq + alpha, dnum = ctx->lv[level].dnum;
  for (auto* c : xs)
    HC_CHECK(c->degree == 1 && c->level == level, HC_ERR_INVALID, "hoisted batch needs degree-1 cts at one level");
  std::vector<u64> gs;
  for (int r : steps) {
    const u64 g = galois_elt(ctx->P, r);
    if (g != 1) HC_CHECK(evk->galois.count(g), HC_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(r));
    gs.push_back(g);
  }
  for (size_t k = 0; k < steps.size(); ++k) {
    outs[k] = new_cts(ctx, total, level, 1, xs[0]->scale);
    for (int i = 0; i < total; ++i) outs[k][i]->scale = xs[i]->scale;
  }
  const size_t ext_words = (size_t)next * n;
  const int* emap = ctx->ext_map_of(level);
  const u64 x_is = (u64)nq * n, ext_is = (u64)dnum * ext_words, acc_is = 2 * (u64)ext_words,
            z_is = 2 * (u64)nq * n;
  // the steps that rotate; groups of them share each launch after ModUp
  std::vector<int> rk;
  for (size_t k = 0; k < gs.size(); ++k) {
    if (gs[k] != 1) rk.push_back((int)k);
  }
  const size_t item_words = x_is + ext_is;                     // c1 in coefficient form, raised digits
  const size_t step_words = acc_is + z_is;                     // per (step, item): key product, ModDown
  const size_t ws_words = kWorkspaceBytes / 8;
  const int chunk = (int)std::min<size_t>(256, std::max<size_t>(1, ws_words / (item_words + step_words)));
  for (int s0 = 0; s0 < total; s0 += chunk) {
    const int m = std::min(chunk, total - s0);
    // as many rotating steps per launch as the workspace holds (at least one)
    const size_t room = ws_words / m > item_words ? (ws_words / m - item_words) / step_words : 0;
    const int sg = (int)std::max<size_t>(1, std::min<size_t>(rk.size(), room));
    std::vector<BufPtr> keep;
    BufPtr work = ctx->buffer(item_words * m + step_words * (size_t)m * std::max(1, sg));
    keep.push_back(work);
    u64* xc = work->ptr;                      // [m][nq][N]
    u64* ext = xc + x_is * m;                 // [m][dnum][next][N]
    u64* acc = ext + ext_is * m;              // [sg][m][2][next][N]
    u64* zq = acc + acc_is * m * sg;          // [sg][m][2][nq][N]
    std::vector<CtRef> c1s, c0s, xsr;
    for (int i = 0; i < m; ++i) {
      const hc_ct* x = xs[s0 + i];
      c1s.push_back(CtRef{x->data + x->stride, 0});
      c0s.push_back(CtRef{x->data, 0});
      xsr.push_back(x->ref());
    }
    // c1 -> coefficient form (N^{-1} left to the conversion constants)
    LimbSet c1in{};
    c1in.refs = refs_dev(ctx, c1s, keep);
    c1in.npoly = 1;
    c1in.nlimb = nq;
    launch_ntt_from(ctx, limbset_base(xc, x_is, 0, 1, nq, 0, nullptr), &c1in, m, true, false);
    // the digits' own slots are c1 itself, copied (the key product reads
    // every slot through the automorphism)
    modup_digits(ctx, level, c1s, xc, x_is, ext, ext_is, m, keep, true);
    for (size_t k = 0; k < gs.size(); ++k) {  // steps that do not rotate: a copy
      if (gs[k] != 1) continue;
      std::vector<CtRef> orr;
      for (int i = 0; i < m; ++i) orr.push_back(outs[k][s0 + i]->ref());
      launch_ew(ctx, 3, refs_dev(ctx, orr, keep), refs_dev(ctx, xsr, keep), nullptr, m, 2, nq);
    }
    for (size_t r0 = 0; r0 < rk.size(); r0 += sg) {
      const int ns = (int)std::min<size_t>(sg, rk.size() - r0), mi = ns * m;  // items: (step, ciphertext)
      std::vector<CtRef> c0src, od;
      std::vector<const u64*> keys;
      std::vector<u64> gitem;
      for (int t = 0; t < ns; ++t) {
        const int k = rk[r0 + t];
        for (int i = 0; i < m; ++i) {
          c0src.push_back(c0s[i]);
          od.push_back(outs[k][s0 + i]->ref());
          keys.push_back(evk->galois.at(gs[k]).buf->ptr);
          gitem.push_back(gs[k]);
        }
      }
      const u64* gd = upload(ctx, gitem, keep);
      const u64* const* kd = ns > 1 ? upload(ctx, keys, keep) : nullptr;
      // the key product reads kappa_g of every raised digit in place (the
      // NTT-domain permutation is the same for every prime): item t m + i
      // uses ciphertext i's digits
      launch_key_product_batched(ctx, level, ext, ext_is, keys[0], acc, acc_is, mi, nullptr, kd, gd, m);
      launch_ntt(ctx, limbset_base(acc, acc_is, ext_words, 2, alpha, nq, emap), mi, true, false);
      launch_moddown_bconv_fast(ctx, level, acc + (size_t)nq * n, acc_is, zq, z_is, mi);
      launch_ntt(ctx, limbset_base(zq, z_is, (u64)nq * n, 2, nq, 0, nullptr), mi, false);
      // out = kappa_g(c0) + ModDown(key product): c0 read through the automorphism
      launch_moddown_combine(ctx, level, acc, acc_is, zq, z_is, refs_dev(ctx, c0src, keep), nullptr,
                             refs_dev(ctx, od, keep), mi, gd);
    }
  }
  return outs;
}

std::vector<hc_ct*> rotate_one(hc_ctx* ctx, const hc_evk* evk, const hc_ct* x, const std::vector<int>& steps,
                               bool hoisted) {
  HC_CHECK(x->degree == 1, HC_ERR_INVALID, "rotate needs a degree-1 ciphertext");
  const int n = ctx->P.n, level = x->level, nq = level + 1;
  std::vector<u64> gs;
  for (int r : steps) {
    const u64 g = galois_elt(ctx->P, r);
    if (g != 1) HC_CHECK(evk->galois.count(g), HC_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(r));
    gs.push_back(g);
  }
  if (hoisted) {  // one ModUp of c1, automorphism applied to the raised digits
    std::vector<hc_ct*> outs;
    for (auto& v : rotate_hoisted_batch(ctx, evk, {x}, steps)) outs.push_back(v[0]);
    return outs;
  }
  std::vector<hc_ct*> outs = new_cts(ctx, (int)steps.size(), level, 1, x->scale);
  std::vector<BufPtr> keep;
  const CtRef* xr = refs_dev(ctx, {x->ref()}, keep);
  // kappa_g(x) of every step into one slab, then one key switch over the
  // steps with each step's Galois key
  int nrot = 0;
  for (u64 g : gs) nrot += g != 1;
  BufPtr tmp = ctx->buffer(std::max<size_t>(1, 2 * (size_t)nrot * nq * n));
  keep.push_back(tmp);
  std::vector<CtRef> xs, b0, o, src;
  std::vector<const u64*> ks;
  std::vector<u64> gitem;
  for (size_t i = 0; i < gs.size(); ++i) {
    if (gs[i] == 1) {
      launch_ew(ctx, 3, refs_dev(ctx, {outs[i]->ref()}, keep), xr, nullptr, 1, 2, nq);
      continue;
    }
    u64* base = tmp->ptr + xs.size() * 2 * (size_t)nq * n;
    xs.push_back(CtRef{base + (size_t)nq * n, (u64)nq * n});
    b0.push_back(CtRef{base, (u64)nq * n});
    src.push_back(x->ref());
    o.push_back(outs[i]->ref());
    ks.push_back(evk->galois.at(gs[i]).buf->ptr);
    gitem.push_back(gs[i]);
  }
  if (!xs.empty()) {  // b0 holds each step's (c0, c1) pair: one automorphism launch for all steps
    launch_automorph_items(ctx, refs_dev(ctx, b0, keep), refs_dev(ctx, src, keep), (int)xs.size(), 2, nq,
                           upload(ctx, gitem, keep));
    keyswitch_batch_keys(ctx, ks, level, xs, &b0, nullptr, o);
  }
  return outs;
}
}  // namespace

extern "C" int hc_rotate(hc_ctx* ctx, const hc_evk* evk, const hc_ct* x, int steps, hc_ct** out) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, x);
    HC_CHECK(evk && out, HC_ERR_INVALID, "null argument");
    *out = rotate_one(ctx, evk, x, {steps}, false)[0];
  });
}

extern "C" int hc_rotate_hoisted(hc_ctx* ctx, const hc_evk* evk, const hc_ct* x, const int32_t* steps, int n,
                                 hc_ct** outs) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    check_ct(ctx, x);
    HC_CHECK(evk && outs && (n == 0 || steps) && n >= 0, HC_ERR_INVALID, "null argument");
    std::vector<int> st(steps, steps + n);
    std::vector<hc_ct*> r = rotate_one(ctx, evk, x, st, true);
    for (int i = 0; i < n; ++i) outs[i] = r[i];
  });
}

namespace {
// n products a[i] b[i], relinearised and rescaled (one pass of each kernel).
// With coeff_out the results are written there in coefficient form (2 polys
// x level-1 limbs per item) and no ciphertexts are returned.
std::vector<hc_ct*> mul_relin_rescale_cts(hc_ctx* ctx, const hc_evk* evk, const hc_ct* const* a,
                                          const hc_ct* const* b, int n, const LimbSet* coeff_out = nullptr) {
  const int level = a[0]->level;
  for (int i = 0; i < n; ++i) {
    check_ct(ctx, a[i]);
    check_ct(ctx, b[i]);
    HC_CHECK(a[i]->level == level && b[i]->level == level, HC_ERR_LEVEL_MISMATCH, "batch mixes levels");
    HC_CHECK(a[i]->degree == 1 && b[i]->degree == 1, HC_ERR_INVALID, "degree-1 operands expected");
  }
  HC_CHECK(level >= 1, HC_ERR_DEPTH, "no level left to rescale");
  std::vector<hc_ct*> d = new_cts(ctx, n, level, 2, a[0]->scale * b[0]->scale);
  {
    std::vector<BufPtr> keep;
    std::vector<CtRef> ar, br, dr;
    for (int i = 0; i < n; ++i) {
      ar.push_back(a[i]->ref());
      br.push_back(b[i]->ref());
      dr.push_back(d[i]->ref());
    }
    for (int o0 = 0; o0 < n; o0 += 65535) {
      const int m = std::min(65535, n - o0);
      launch_tensor_pair(ctx, refs_dev(ctx, std::vector<CtRef>(dr.begin() + o0, dr.begin() + o0 + m), keep),
                         refs_dev(ctx, std::vector<CtRef>(ar.begin() + o0, ar.begin() + o0 + m), keep),
                         refs_dev(ctx, std::vector<CtRef>(br.begin() + o0, br.begin() + o0 + m), keep), m, level + 1);
    }
  }
  for (int i = 0; i < n; ++i) d[i]->scale = a[i]->scale * b[i]->scale;
  std::vector<hc_ct*> r = relin_rescale(ctx, evk, d, nullptr, coeff_out);
  for (size_t i = 0; i < r.size(); ++i) r[i]->scale = d[i]->scale / (double)ctx->P.chain[level];
  free_all(d);
  return r;
}
}  // namespace

extern "C" int hc_mul_relin_rescale_batch(hc_ctx* ctx, const hc_evk* evk, const hc_ct* const* a,
                                          const hc_ct* const* b, int n, hc_ct** outs) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(evk && n >= 0 && (n == 0 || (a && b && outs)), HC_ERR_INVALID, "null argument");
    if (n == 0) return;
    std::vector<hc_ct*> r = mul_relin_rescale_cts(ctx, evk, a, b, n);
    for (int i = 0; i < n; ++i) outs[i] = r[i];
  });
}

// =====================================================================
// Autotuning
// =====================================================================
extern "C" int hc_tune_set(hc_ctx* ctx, int knob, int value) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    switch (knob) {
      case HC_TUNE_NTT:
        HC_CHECK(value >= 0 && value <= (ctx->P.log_n >= 13 ? 5 : 1), HC_ERR_INVALID,
                 "NTT variant must be 0, 1 (or 2..5 for N >= 2^13)");
        ctx->tune.ntt_variant[ctx->P.log_n] = value;
        break;
      case HC_TUNE_KEY_PRODUCT_Z:
        HC_CHECK(value >= 1 && value <= 64, HC_ERR_INVALID, "key-product groups must be 1..64");
        ctx->tune.kp_zmul = value;
        break;
      case HC_TUNE_MODUP_SPLIT:
        HC_CHECK(value >= 1 && value <= 64, HC_ERR_INVALID, "ModUp split must be 1..64");
        ctx->tune.modup_split = value;
        break;
      case HC_TUNE_TENSOR_GROUP:
        HC_CHECK(value >= 0 && value <= 5, HC_ERR_INVALID, "tensor group must be 0..5");
        ctx->tune.tensor_group = value;
        break;
      case HC_TUNE_HOST_STREAMS:
        HC_CHECK(value >= 1 && value <= 4, HC_ERR_INVALID, "host streams must be 1..4");
        ctx->tune.host_streams = value;
        break;
      default:
        throw HcError{HC_ERR_INVALID, "unknown tuning knob"};
    }
  });
}

extern "C" int hc_tune_get(const hc_ctx* ctx, int knob) {
  if (!ctx) return HC_ERR_INVALID;
  switch (knob) {
    case HC_TUNE_NTT: return ctx->tune.ntt_variant[ctx->P.log_n];
    case HC_TUNE_KEY_PRODUCT_Z: return ctx->tune.kp_zmul;
    case HC_TUNE_MODUP_SPLIT: return ctx->tune.modup_split;
    case HC_TUNE_TENSOR_GROUP: return ctx->tune.tensor_group;
    case HC_TUNE_HOST_STREAMS: return ctx->tune.host_streams;
    default: return HC_ERR_INVALID;
  }
}

// A candidate replaces the current value only when it is at least 2 %
// faster, so timing noise does not flip the choice.
constexpr double kSwitchGain = 0.98;

extern "C" int hc_autotune(hc_ctx* ctx, const hc_evk* evk, int items, char* report, size_t cap) {
  if (!ctx) return HC_ERR_INVALID;
  std::vector<cudaEvent_t> evs;
  int rc = guard(ctx, [&] {
    HC_CHECK(evk && items >= 1, HC_ERR_INVALID, "bad arguments");
    HC_CHECK(!ctx->arena, HC_ERR_INVALID, "autotuning cannot be captured");
    const int n = ctx->P.n, level = ctx->P.L, nq = level + 1, alpha = ctx->P.alpha;
    const int next = nq + alpha, dnum = ctx->lv[level].dnum;
    const size_t limb = (size_t)n, ext_words = (size_t)next * limb;
    // scratch for `m` items, at most ~6 GiB
    const size_t per_item = (size_t)2 * nq * limb + (size_t)dnum * ext_words + 2 * ext_words;
    const int m = (int)std::max<size_t>(1, std::min<size_t>((size_t)items, ((size_t)6 << 30) / (per_item * 8)));
    std::vector<BufPtr> keep;
    BufPtr work = ctx->buffer(per_item * m);
    keep.push_back(work);
    HC_CUDA(cudaMemsetAsync(work->ptr, 0, per_item * m * sizeof(u64), ctx->stream));
    u64* cts = work->ptr;                              // [m][2][nq][N]
    u64* ext = cts + (size_t)m * 2 * nq * limb;        // [m][dnum][next][N]
    u64* acc = ext + (size_t)m * dnum * ext_words;     // [m][2][next][N]
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      HC_CUDA(cudaEventCreate(&e));
      evs.push_back(e);
    }
    auto time_us = [&](const std::function<void()>& f) {
      f();  // warm-up
      HC_CUDA(cudaEventRecord(evs[0], ctx->stream));
      for (int r = 0; r < 3; ++r) f();
      HC_CUDA(cudaEventRecord(evs[1], ctx->stream));
      HC_CUDA(cudaEventSynchronize(evs[1]));
      float ms = 0;
      HC_CUDA(cudaEventElapsedTime(&ms, evs[0], evs[1]));
      return 1000.0 * ms / 3;
    };
    std::string rep;
    char line[256];
    // NTT: forward and inverse transforms of m degree-1 ciphertexts
    {
      const LimbSet cs = limbset_base(cts, 2 * nq * limb, nq * limb, 2, nq, 0, nullptr);
      const int incumbent = ctx->tune.ntt_variant[ctx->P.log_n];
      double best = 1e300, inc_us = 1e300;
      int pick = incumbent;
      std::string t;
      for (int v = 0; v <= (ctx->P.log_n >= 13 ? 5 : 1); ++v) {
        ctx->tune.ntt_variant[ctx->P.log_n] = v;
        const double us = time_us([&] {
          launch_ntt(ctx, cs, m, false);
          launch_ntt(ctx, cs, m, true);
        });
        std::snprintf(line, sizeof line, " %d:%.1f", v, us);
        t += line;
        if (v == incumbent) inc_us = us;
        if (us < best) best = us, pick = v;
      }
      if (best > kSwitchGain * inc_us) pick = incumbent;
      ctx->tune.ntt_variant[ctx->P.log_n] = pick;
      std::snprintf(line, sizeof line, "ntt_variant %d us%s\n", pick, t.c_str());
      rep += line;
    }
    // key product over the raised digits
    {
      const int incumbent = ctx->tune.kp_zmul;
      double best = 1e300, inc_us = 1e300;
      int pick = incumbent;
      std::string t;
      for (int z : {1, 2, 4, 8}) {
        ctx->tune.kp_zmul = z;
        const double us = time_us([&] {
          launch_key_product_batched(ctx, level, ext, (u64)dnum * ext_words, evk->relin.buf->ptr, acc,
                                     2 * (u64)ext_words, m);
        });
        std::snprintf(line, sizeof line, " %d:%.1f", z, us);
        t += line;
        if (z == incumbent) inc_us = us;
        if (us < best) best = us, pick = z;
      }
      if (best > kSwitchGain * inc_us) pick = incumbent;
      ctx->tune.kp_zmul = pick;
      std::snprintf(line, sizeof line, "key_product_z %d us%s\n", pick, t.c_str());
      rep += line;
    }
    // ModUp conversion of digit 0
    {
      const int incumbent = ctx->tune.modup_split;
      double best = 1e300, inc_us = 1e300;
      int pick = incumbent;
      std::string t;
      for (int sp : {1, 2, 4}) {
        ctx->tune.modup_split = sp;
        const double us = time_us([&] {
          launch_modup_bconv_fast(ctx, level, 0, cts, 2 * (u64)nq * limb, ext, (u64)dnum * ext_words, m);
        });
        std::snprintf(line, sizeof line, " %d:%.1f", sp, us);
        t += line;
        if (sp == incumbent) inc_us = us;
        if (us < best) best = us, pick = sp;
      }
      if (best > kSwitchGain * inc_us) pick = incumbent;
      ctx->tune.modup_split = pick;
      std::snprintf(line, sizeof line, "modup_split %d us%s\n", pick, t.c_str());
      rep += line;
    }
    HC_CUDA(cudaStreamSynchronize(ctx->stream));
    if (report && cap > 0) {
      std::snprintf(report, cap, "%s", rep.c_str());
    }
  });
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
  return rc;
}

namespace {
// Chunk sizes of the host-to-host pipeline for n pairs: equal chunks of
// `chunk` pairs, the last one ragged; automatic (chunk = 0): sixteen chunks
// from 32 pairs up (measured best with the chunks' kernels on two streams:
// 4 pairs of 64), about eight below, and from 32 pairs up the last chunk
// split into halves (4 -> 2, 1, 1), so that less work and copying is left
// after the last copy in.
// Asynchronous calls (several in flight, each call's tail hidden behind the
// next call's copies in) take eighths without a split tail: measured at 64
// pairs with two in flight, 15.70 ms per call against 16.53 ms for the
// synchronous schedule.
std::vector<int> host_chunks(int n, int chunk, bool async) {
  const int m = chunk > 0 ? chunk
                          : (n >= 32 ? (async ? (n + 7) / 8 : (n + 15) / 16) : std::max(1, (n + 7) / 8));
  std::vector<int> sizes;
  for (int r = n; r > 0; r -= m) sizes.push_back(std::min(m, r));
  if (chunk == 0 && n >= 32 && !async) {  // measured at 64 pairs: 17.17 against 17.44-17.50 ms per call
    int last = sizes.back();
    sizes.pop_back();
    while (last > 1) {
      sizes.push_back(last / 2);
      last -= last / 2;
    }
    sizes.push_back(last);
  }
  return sizes;
}
}  // namespace

// Host-to-host pipeline: all input slabs are allocated up front (so the copy
// stream never waits on the compute stream), every chunk's inputs are queued
// on the copy-in stream at once, and chunk c's compute waits only for its own
// copies; its outputs go back on the copy-out stream while chunk c + 1 runs.
// eval: host buffers in evaluation (NTT) form, so the chunks' inputs need no
// forward transforms and the products keep the device batch's forward tail.
namespace {
// Waits for a host-to-host call's copies out, reads its range-check flags
// on a stream of their own (the context's other streams may already carry
// the next call), records its timeline and releases its buffers and events.
int host_op_finish(hc_host_op* op_raw) {
  std::unique_ptr<hc_host_op> op(op_raw);
  hc_ctx* ctx = op->ctx;
  const int rc = guard(ctx, [&] {
    if (!op->drained) return;  // an empty call
    HC_CUDA(cudaEventSynchronize(op->drained));
    if (!ctx->flag_stream) HC_CUDA(cudaStreamCreateWithFlags(&ctx->flag_stream, cudaStreamNonBlocking));
    std::vector<u64> bad(op->nch);
    HC_CUDA(cudaStreamWaitEvent(ctx->flag_stream, op->drained, 0));
    HC_CUDA(cudaMemcpyAsync(bad.data(), op->flags->ptr, op->nch * sizeof(u64), cudaMemcpyDeviceToHost,
                            ctx->flag_stream));
    HC_CUDA(cudaStreamSynchronize(ctx->flag_stream));
    if (op->t_start) {
      ctx->host_timeline.assign(op->tev.size(), 0.0);
      for (size_t k = 0; k < op->tev.size(); ++k) {
        float ms = 0;
        HC_CUDA(cudaEventElapsedTime(&ms, op->t_start, op->tev[k]));
        ctx->host_timeline[k] = ms;
      }
    }
    for (u64 b : bad) HC_CHECK(b == 0, HC_ERR_INVALID, "input residue not below its prime (outputs not valid)");
  });
  op->flags.reset();
  op->keep.clear();
  for (cudaEvent_t e : op->evs) cudaEventDestroy(e);
  return rc;
}

int host_pipeline(hc_ctx* ctx, const hc_evk* evk, const uint64_t* const* a_host, const hc_ct_meta* a_meta,
                  const uint64_t* const* b_host, const hc_ct_meta* b_meta, int n, int chunk,
                  uint64_t* const* out_host, const size_t* out_cap, hc_ct_meta* out_meta, bool eval,
                  hc_host_op** async_out) {
  if (!ctx) return HC_ERR_INVALID;
  if (async_out) *async_out = nullptr;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  std::unique_ptr<hc_host_op> op(new hc_host_op);
  op->ctx = ctx;
  std::vector<cudaEvent_t>& evs = op->evs;
  std::vector<std::vector<hc_ct*>> ins;
  std::vector<BufPtr>& keep = op->keep;  // released only after the side streams are drained
  int rc = guard(ctx, [&] {
    HC_CHECK(evk && n >= 0 && (n == 0 || (a_host && b_host && a_meta && b_meta && out_host && out_cap && out_meta)),
             HC_ERR_INVALID, "null argument");
    HC_CHECK(!ctx->arena, HC_ERR_INVALID, "host-buffer calls cannot be captured");
    if (n == 0) return;
    const int level = a_meta[0].level, N = ctx->P.n;
    HC_CHECK(level >= 0 && level <= ctx->P.L, HC_ERR_INVALID, "bad level");
    HC_CHECK(level >= 1, HC_ERR_DEPTH, "no level left to rescale");
    const size_t out_words = (size_t)2 * level * N;
    for (int i = 0; i < n; ++i) {
      HC_CHECK(a_meta[i].level == level && b_meta[i].level == level, HC_ERR_LEVEL_MISMATCH, "batch mixes levels");
      HC_CHECK(a_meta[i].degree == 1 && b_meta[i].degree == 1, HC_ERR_INVALID, "degree-1 operands expected");
      HC_CHECK(a_host[i] && b_host[i] && out_host[i], HC_ERR_INVALID, "null buffer");
      HC_CHECK(out_cap[i] >= out_words, HC_ERR_INVALID, "output buffer too small");
    }
    HC_CHECK(chunk >= 0, HC_ERR_INVALID, "negative chunk");
    const std::vector<int> sizes = host_chunks(n, chunk, async_out != nullptr);
    const int nch = (int)sizes.size();
    std::vector<int> first(nch + 1, 0);  // pair index of each chunk's first pair
    for (int c = 0; c < nch; ++c) first[c + 1] = first[c] + sizes[c];
    // the copy streams live as long as the context (no stream creation per call)
    for (cudaStream_t& st : ctx->copy_streams)
      if (!st) HC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    h2d = ctx->copy_streams[0];
    d2h = ctx->copy_streams[1];
    auto event = [&]() {
      cudaEvent_t e;
      HC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      evs.push_back(e);
      return e;
    };
    // the extra compute streams start after the work already on the context stream
    const int ncs = std::max(1, std::min(4, ctx->tune.host_streams));
    const cudaEvent_t start2 = event();
    HC_CUDA(cudaEventRecord(start2, ctx->stream));
    for (int k = 2; k < 1 + ncs; ++k) HC_CUDA(cudaStreamWaitEvent(ctx->copy_streams[k], start2, 0));
    // timing events around each chunk's copies in, its kernels and its copies
    // out, relative to the call's start (read back by hc_profile_host_timeline)
    const bool tl = true;  // 48 events per call: cheap, and every call's timeline can be read back
    std::vector<cudaEvent_t>& tev = op->tev;  // [chunk][h2d b, h2d e, compute b, compute e, d2h b, d2h e]
    auto tmark = [&](cudaStream_t st) -> cudaEvent_t {
      cudaEvent_t e;
      HC_CUDA(cudaEventCreate(&e));
      evs.push_back(e);
      HC_CUDA(cudaEventRecord(e, st));
      return e;
    };
    op->t_start = tl ? tmark(ctx->stream) : nullptr;
    if (tl) tev.assign((size_t)6 * nch, nullptr);
    BufPtr flags = ctx->buffer(nch);
    keep.push_back(flags);
    op->flags = flags;
    op->nch = nch;
    HC_CUDA(cudaMemsetAsync(flags->ptr, 0, nch * sizeof(u64), ctx->stream));
    const size_t stride = (size_t)(level + 1) * N;  // one polynomial
    for (int c = 0; c < nch; ++c) ins.push_back(new_cts(ctx, 2 * sizes[c], level, 1, 1.0));  // a's, b's: one slab
    const cudaEvent_t allocated = event();
    HC_CUDA(cudaEventRecord(allocated, ctx->stream));
    HC_CUDA(cudaStreamWaitEvent(h2d, allocated, 0));
    std::vector<cudaEvent_t> copied(nch);
    for (int c = 0; c < nch; ++c) {
      const int m = (int)ins[c].size() / 2;
      if (tl) tev[6 * c + 0] = tmark(h2d);
      for (int j = 0; j < m; ++j) {
        const int i = first[c] + j;
        HC_CUDA(cudaMemcpyAsync(ins[c][j]->data, a_host[i], 2 * stride * sizeof(u64), cudaMemcpyHostToDevice, h2d));
        HC_CUDA(cudaMemcpyAsync(ins[c][m + j]->data, b_host[i], 2 * stride * sizeof(u64), cudaMemcpyHostToDevice,
                                h2d));
      }
      if (tl) tev[6 * c + 1] = tmark(h2d);
      copied[c] = event();
      HC_CUDA(cudaEventRecord(copied[c], h2d));
    }
    for (int c = 0; c < nch; ++c) {
      std::vector<hc_ct*>& x = ins[c];
      const int m = (int)x.size() / 2;
      // chunks round-robin over the compute streams (the context stream and
      // ncs - 1 others), so one chunk's kernels fill the previous one's last
      // waves (their buffers are disjoint; outputs are ordered by the
      // copy-out stream's waits)
      struct StreamSwap {
        hc_ctx* c;
        cudaStream_t home;
        ~StreamSwap() { c->stream = home; }
      } swap{ctx, ctx->stream};
      if (c % ncs != 0) ctx->stream = ctx->copy_streams[1 + c % ncs];
      HC_CUDA(cudaStreamWaitEvent(ctx->stream, copied[c], 0));
      if (tl) tev[6 * c + 2] = tmark(ctx->stream);
      launch_check_range(ctx, x[0]->data, 4 * m, level + 1, stride, (unsigned long long*)(flags->ptr + c));
      if (!eval) launch_ntt(ctx, limbset_base(x[0]->data, 2 * stride, stride, 2, level + 1, 0, nullptr), 2 * m, false);
      for (int j = 0; j < m; ++j) {
        x[j]->scale = a_meta[first[c] + j].scale;
        x[m + j]->scale = b_meta[first[c] + j].scale;
      }
      std::vector<const u64*> src(m);  // each product's [2][level][N] words on the device
      if (eval) {
        // the device batch's products, evaluation form; their slab lives until the copies out are done
        std::vector<hc_ct*> r = mul_relin_rescale_cts(ctx, evk, x.data(), x.data() + m, m);
        for (int j = 0; j < m; ++j) {
          HC_CHECK(r[j]->stride == (size_t)level * N, HC_ERR_INVALID, "unexpected product layout");
          keep.push_back(r[j]->buf);
          src[j] = r[j]->data;
        }
        free_all(r);
      } else {
        // the products come out in coefficient form straight into the staging slab
        BufPtr staged = ctx->buffer(m * out_words);
        keep.push_back(staged);
        const LimbSet co = limbset_base(staged->ptr, out_words, (u64)level * N, 2, level, 0, nullptr);
        mul_relin_rescale_cts(ctx, evk, x.data(), x.data() + m, m, &co);
        for (int j = 0; j < m; ++j) src[j] = staged->ptr + (size_t)j * out_words;
      }
      free_all(x);  // stream-ordered: the copies into x finished before this stream's first use
      for (int j = 0; j < m; ++j) {
        const int i = first[c] + j;
        out_meta[i] = hc_ct_meta{level - 1, 1, a_meta[i].scale * b_meta[i].scale / (double)ctx->P.chain[level]};
      }
      if (tl) tev[6 * c + 3] = tmark(ctx->stream);
      const cudaEvent_t done = event();
      HC_CUDA(cudaEventRecord(done, ctx->stream));
      HC_CUDA(cudaStreamWaitEvent(d2h, done, 0));
      if (tl) tev[6 * c + 4] = tmark(d2h);
      for (int j = 0; j < m; ++j)
        HC_CUDA(cudaMemcpyAsync(out_host[first[c] + j], src[j], out_words * sizeof(u64), cudaMemcpyDeviceToHost, d2h));
      if (tl) tev[6 * c + 5] = tmark(d2h);
    }
    // (the context stream is restored at the end of every chunk)
    // staged buffers go back to the pool only after the copies out
    op->drained = event();
    HC_CUDA(cudaEventRecord(op->drained, d2h));
    // a synchronous call orders the context stream after its copies out; an
    // asynchronous one leaves it free, so that the next call's copies in can
    // start while this call's last chunk still computes and copies out
    if (!async_out) HC_CUDA(cudaStreamWaitEvent(ctx->stream, op->drained, 0));
  });
  if (rc == HC_OK && async_out) {  // the caller waits with hc_host_op_wait
    *async_out = op.release();
    return HC_OK;
  }
  if (rc == HC_OK) return host_op_finish(op.release());
  // on an error the side streams may still be writing into inputs: drain them first
  if (h2d) cudaStreamSynchronize(h2d);
  if (d2h) cudaStreamSynchronize(d2h);
  for (int k = 2; k < 5; ++k)
    if (ctx->copy_streams[k]) cudaStreamSynchronize(ctx->copy_streams[k]);
  keep.clear();
  for (auto& v : ins) free_all(v);
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
  return rc;
}
}  // namespace

extern "C" int hc_mul_relin_rescale_host(hc_ctx* ctx, const hc_evk* evk, const uint64_t* const* a_host,
                                         const hc_ct_meta* a_meta, const uint64_t* const* b_host,
                                         const hc_ct_meta* b_meta, int n, int chunk, uint64_t* const* out_host,
                                         const size_t* out_cap, hc_ct_meta* out_meta) {
  return host_pipeline(ctx, evk, a_host, a_meta, b_host, b_meta, n, chunk, out_host, out_cap, out_meta, false,
                       nullptr);
}

extern "C" int hc_mul_relin_rescale_host_eval(hc_ctx* ctx, const hc_evk* evk, const uint64_t* const* a_host,
                                              const hc_ct_meta* a_meta, const uint64_t* const* b_host,
                                              const hc_ct_meta* b_meta, int n, int chunk, uint64_t* const* out_host,
                                              const size_t* out_cap, hc_ct_meta* out_meta) {
  return host_pipeline(ctx, evk, a_host, a_meta, b_host, b_meta, n, chunk, out_host, out_cap, out_meta, true,
                       nullptr);
}

extern "C" int hc_mul_relin_rescale_host_eval_async(hc_ctx* ctx, const hc_evk* evk, const uint64_t* const* a_host,
                                                    const hc_ct_meta* a_meta, const uint64_t* const* b_host,
                                                    const hc_ct_meta* b_meta, int n, int chunk,
                                                    uint64_t* const* out_host, const size_t* out_cap,
                                                    hc_ct_meta* out_meta, hc_host_op** op) {
  if (!ctx) return HC_ERR_INVALID;
  if (!op) {
    ctx->err = "null op";
    return HC_ERR_INVALID;
  }
  return host_pipeline(ctx, evk, a_host, a_meta, b_host, b_meta, n, chunk, out_host, out_cap, out_meta, true, op);
}

extern "C" int hc_host_op_wait(hc_host_op* op) {
  if (!op) return HC_ERR_INVALID;
  return host_op_finish(op);
}

// =====================================================================
// CNN layers
// =====================================================================
extern "C" int hc_enc_conv2d(hc_ctx* ctx, const hc_evk* evk, hc_packing packing, const hc_ct* const* x, int H,
                             int W, int cin, const hc_ct* const* w, int cout, int kh, int kw, int stride, hc_ct** y) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(evk && x && w && y, HC_ERR_INVALID, "null argument");
    HC_CHECK(H > 0 && W > 0 && cin > 0 && cout > 0 && kh > 0 && kw > 0 && stride > 0 && kh <= H && kw <= W,
             HC_ERR_INVALID, "bad shape");
    if (packing == HC_PACK_BATCH) {
      const int Ho = (H - kh) / stride + 1, Wo = (W - kw) / stride + 1;
      const int nx = H * W * cin, nw = cout * kh * kw * cin;
      std::vector<const hc_ct*> xs(x, x + nx), ws(w, w + nw);
      const int level = xs[0]->level;
      for (auto* c : xs) {
        check_ct(ctx, c);
        HC_CHECK(c->level == level && c->degree == 1, HC_ERR_LEVEL_MISMATCH, "inputs at different levels");
        check_scales(c->scale, xs[0]->scale);
      }
      std::vector<hc_ct*> wviews;  // weights above the inputs' level, dropped to it
      for (auto*& c : ws) {
        check_ct(ctx, c);
        HC_CHECK(c->level >= level && c->degree == 1, HC_ERR_LEVEL_MISMATCH, "weights below the inputs' level");
        check_scales(c->scale, ws[0]->scale);
        if (c->level != level) {
          wviews.push_back(new hc_ct{ctx, c->buf, c->data, c->stride, level, 1, c->scale});
          c = wviews.back();
        }
      }
      HC_CHECK(level >= 1, HC_ERR_DEPTH, "no level left");
      std::vector<int> xi, wi, off{0};
      for (int m = 0; m < Ho; ++m)
        for (int nn = 0; nn < Wo; ++nn)
          for (int co = 0; co < cout; ++co) {
            for (int p = 0; p < kh; ++p)
              for (int q = 0; q < kw; ++q)
                for (int ci = 0; ci < cin; ++ci) {
                  xi.push_back(((m * stride + p) * W + (nn * stride + q)) * cin + ci);
                  wi.push_back(((co * kh + p) * kw + q) * cin + ci);
                }
            off.push_back((int)xi.size());
          }
      std::vector<hc_ct*> d = tensor_acc(ctx, xs, ws, xi, wi, off, level, xs[0]->scale * ws[0]->scale);
      std::vector<hc_ct*> r = relin_rescale(ctx, evk, d, nullptr);
      free_all(d);
      free_all(wviews);
      for (size_t i = 0; i < r.size(); ++i) y[i] = r[i];
    } else {
      HC_CHECK(packing == HC_PACK_SINGLE || packing == HC_PACK_SINGLE_HOISTED, HC_ERR_INVALID, "unknown packing");
      HC_CHECK(cin == 1 && stride == 1, HC_ERR_INVALID, "single packing supports cin = 1, stride 1");
      const hc_ct* x0 = x[0];
      check_ct(ctx, x0);
      std::vector<int> steps;
      for (int p = 0; p < kh; ++p)
        for (int q = 0; q < kw; ++q) steps.push_back(p * W + q);
      std::vector<hc_ct*> rots = rotate_one(ctx, evk, x0, steps, packing == HC_PACK_SINGLE_HOISTED);
      std::vector<const hc_ct*> xs(rots.begin(), rots.end()), ws(w, w + cout * kh * kw);
      std::vector<hc_ct*> wviews;
      for (auto*& c : ws) {
        check_ct(ctx, c);
        HC_CHECK(c->level >= x0->level && c->degree == 1, HC_ERR_LEVEL_MISMATCH, "weights below the input's level");
        if (c->level != x0->level) {
          wviews.push_back(new hc_ct{ctx, c->buf, c->data, c->stride, x0->level, 1, c->scale});
          c = wviews.back();
        }
      }
      std::vector<int> xi, wi, off{0};
      for (int co = 0; co < cout; ++co) {
        for (int t = 0; t < kh * kw; ++t) {
          xi.push_back(t);
          wi.push_back(co * kh * kw + t);
        }
        off.push_back((int)xi.size());
      }
      std::vector<hc_ct*> d = tensor_acc(ctx, xs, ws, xi, wi, off, x0->level, x0->scale * ws[0]->scale);
      std::vector<hc_ct*> r = relin_rescale(ctx, evk, d, nullptr);
      free_all(d);
      free_all(rots);
      free_all(wviews);
      for (size_t i = 0; i < r.size(); ++i) y[i] = r[i];
    }
  });
}

namespace {
std::vector<hc_ct*> views_at(hc_ctx* ctx, const std::vector<const hc_ct*>& xs, int level) {
  std::vector<hc_ct*> v;
  for (auto* c : xs) v.push_back(new hc_ct{ctx, c->buf, c->data, c->stride, level, c->degree, c->scale});
  return v;
}

std::vector<const hc_ct*> to_const(const std::vector<hc_ct*>& v) { return std::vector<const hc_ct*>(v.begin(), v.end()); }

// rs(rl(a (x) b)) elementwise over two equal-length lists at one level
std::vector<hc_ct*> mul_rr(hc_ctx* ctx, const hc_evk* evk, const std::vector<const hc_ct*>& a,
                           const std::vector<const hc_ct*>& b) {
  return mul_relin_rescale_cts(ctx, evk, a.data(), b.data(), (int)a.size());
}

// rescale(x * c @ cs) with cs chosen per element by cs_of(i)
std::vector<hc_ct*> mulc_rs(hc_ctx* ctx, const std::vector<const hc_ct*>& x, double c, double cs) {
  std::vector<hc_ct*> m = mul_const_cts(ctx, x, c, cs);
  const double q = (double)ctx->P.chain[x[0]->level];
  std::vector<hc_ct*> out = new_cts(ctx, (int)x.size(), x[0]->level - 1, x[0]->degree, m[0]->scale / q);
  rescale_cts(ctx, to_const(m), out);
  for (size_t i = 0; i < out.size(); ++i) out[i]->scale = m[i]->scale / q;
  free_all(m);
  return out;
}

// a += b elementwise (scales must agree; a keeps its scale)
void add_into(hc_ctx* ctx, const std::vector<hc_ct*>& a, const std::vector<const hc_ct*>& b, int level) {
  std::vector<BufPtr> keep;
  std::vector<CtRef> ar, br;
  for (size_t i = 0; i < a.size(); ++i) {
    check_scales(a[i]->scale, b[i]->scale);
    ar.push_back(a[i]->ref());
    br.push_back(b[i]->ref());
  }
  const CtRef* ad = refs_dev(ctx, ar, keep);
  launch_ew(ctx, 0, ad, ad, refs_dev(ctx, br, keep), (int)a.size(), 2, level + 1);
}

// Degree-7 activation (Paterson-Stockmeyer split, four levels), batched.
std::vector<hc_ct*> poly7(hc_ctx* ctx, const hc_evk* evk, const std::vector<const hc_ct*>& u, const double* c) {
  const int lv = u[0]->level;
  HC_CHECK(lv >= 4, HC_ERR_DEPTH, "the degree-7 activation needs four levels");
  const double q2 = (double)ctx->P.chain[lv - 2], q3 = (double)ctx->P.chain[lv - 3];
  const size_t n = u.size();
  std::vector<hc_ct*> u2 = mul_rr(ctx, evk, u, u);                                   // lv-1
  std::vector<hc_ct*> ud1 = views_at(ctx, u, lv - 1);
  // u4 = u2 u2 and u3 = u2 u in one batch                                              lv-2
  std::vector<const hc_ct*> la = to_const(u2), lb = to_const(u2);
  la.insert(la.end(), u2.begin(), u2.end());
  lb.insert(lb.end(), ud1.begin(), ud1.end());
  std::vector<hc_ct*> u43 = mul_rr(ctx, evk, la, lb);
  std::vector<hc_ct*> u4(u43.begin(), u43.begin() + n), u3(u43.begin() + n, u43.end());
  std::vector<hc_ct*> u2d = views_at(ctx, to_const(u2), lv - 2);
  std::vector<hc_ct*> ud2 = views_at(ctx, u, lv - 2);
  // the six constant products of both cubic parts, then one rescale for all   lv-3
  // (t3 = u3 a3 @ q_{l-2}; t2 and t1 at t3's scale through their constants' scale)
  const double s3 = u3[0]->scale * q2 / q2;  // scale of rs(u3 * a3 @ q2)
  std::vector<hc_ct*> m;
  for (int h = 0; h < 2; ++h) {
    const double a1 = c[4 * h + 1], a2 = c[4 * h + 2], a3 = c[4 * h + 3];
    for (auto& v : std::vector<std::vector<hc_ct*>>{mul_const_cts(ctx, to_const(u3), a3, q2),
                                                   mul_const_cts(ctx, to_const(u2d), a2, s3 * q2 / u2d[0]->scale),
                                                   mul_const_cts(ctx, to_const(ud2), a1, s3 * q2 / ud2[0]->scale)})
      m.insert(m.end(), v.begin(), v.end());
  }
  std::vector<hc_ct*> t(m.size());
  {
    std::vector<hc_ct*> outs = new_cts(ctx, (int)m.size(), lv - 3, 1, 1.0);
    rescale_cts(ctx, to_const(m), outs);
    for (size_t i = 0; i < m.size(); ++i) {
      outs[i]->scale = m[i]->scale / q2;
      t[i] = outs[i];
    }
  }
  auto deg3 = [&](int h) {  // t3 + t2 + t1 + a0
    std::vector<hc_ct*> t3(t.begin() + 3 * n * h, t.begin() + 3 * n * h + n);
    std::vector<const hc_ct*> t2(t.begin() + 3 * n * h + n, t.begin() + 3 * n * h + 2 * n);
    std::vector<const hc_ct*> t1(t.begin() + 3 * n * h + 2 * n, t.begin() + 3 * n * h + 3 * n);
    add_into(ctx, t3, t2, lv - 3);
    add_into(ctx, t3, t1, lv - 3);
    std::vector<u64> sc;
    constant_residues(ctx, lv - 3, c[4 * h] * t3[0]->scale, false, sc);
    std::vector<BufPtr> keep;
    std::vector<CtRef> tr;
    for (auto* x : t3) tr.push_back(x->ref());
    const CtRef* td = refs_dev(ctx, tr, keep);
    launch_scalar(ctx, true, td, td, (int)t3.size(), 2, lv - 2, upload(ctx, sc, keep));
    return t3;
  };
  std::vector<hc_ct*> qa = deg3(0);
  std::vector<hc_ct*> qb = deg3(1);
  std::vector<hc_ct*> u4d = views_at(ctx, to_const(u4), lv - 3);
  std::vector<hc_ct*> prod = mul_rr(ctx, evk, to_const(qb), to_const(u4d));         // lv-4
  std::vector<hc_ct*> qa2 = mulc_rs(ctx, to_const(qa), 1.0, prod[0]->scale * q3 / qa[0]->scale);
  add_into(ctx, prod, to_const(qa2), lv - 4);
  free_all(u43);  // u4 and u3
  for (size_t i = 0; i < t.size(); ++i)  // the t2, t1 parts (t3 parts are qa, qb)
    if ((i / n) % 3 != 0) delete t[i];
  free_all(m);
  for (auto* v : {&u2, &ud1, &u2d, &ud2, &qa, &qb, &u4d, &qa2}) free_all(*v);
  return prod;
}
}  // namespace

extern "C" int hc_enc_poly_act(hc_ctx* ctx, const hc_evk* evk, const hc_ct* const* x, int n, const double* coeffs,
                               int degree, hc_ct** y) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(evk && coeffs && (degree == 2 || degree == 7) && n >= 0 && (n == 0 || (x && y)), HC_ERR_INVALID,
             "bad arguments");
    if (degree == 7 && n > 0) {
      std::vector<const hc_ct*> xs(x, x + n);
      for (auto* c : xs) {
        check_ct(ctx, c);
        HC_CHECK(c->level == xs[0]->level && c->degree == 1, HC_ERR_LEVEL_MISMATCH, "inputs at different levels");
        check_scales(c->scale, xs[0]->scale);
      }
      std::vector<hc_ct*> r = poly7(ctx, evk, xs, coeffs);
      for (int i = 0; i < n; ++i) y[i] = r[i];
      return;
    }
    if (n == 0) return;
    // inputs may sit at several levels: one group per level, each a branch of
    // its own (fork_join), the same circuit as a call per level
    std::map<int, std::vector<int>> by_level;
    for (int i = 0; i < n; ++i) {
      check_ct(ctx, x[i]);
      HC_CHECK(x[i]->degree == 1, HC_ERR_LEVEL_MISMATCH, "inputs must be degree 1");
      by_level[x[i]->level].push_back(i);
    }
    const double a0 = coeffs[0], a1 = coeffs[1], a2 = coeffs[2];
    const bool square = (a0 == 0 && a1 == 0 && a2 == 1);
    for (auto& kv : by_level) {
      HC_CHECK(kv.first >= (square ? 1 : 2), HC_ERR_DEPTH, "not enough levels for the activation");
      for (int i : kv.second) check_scales(x[i]->scale, x[kv.second[0]]->scale);
    }
    const std::vector<std::pair<int, std::vector<int>>> glist(by_level.begin(), by_level.end());
    std::vector<hc_ct*> res(n, nullptr);
    fork_join(ctx, (int)glist.size(), [&](int branch) {
      const int level = glist[branch].first;
      const std::vector<int>& idx = glist[branch].second;
      const int m = (int)idx.size();
      std::vector<const hc_ct*> xs;
      for (int i : idx) xs.push_back(x[i]);
      std::vector<hc_ct*> t = mul_relin_rescale_cts(ctx, evk, xs.data(), xs.data(), m);  // rs(rl(u u))
      if (square) {
        for (int k = 0; k < m; ++k) res[idx[k]] = t[k];
        return;
      }
      std::vector<const hc_ct*> tc(t.begin(), t.end());
      std::vector<hc_ct*> t2m = mul_const_cts(ctx, tc, a2, (double)ctx->P.chain[level - 1]);
      std::vector<hc_ct*> t2(m);
      {
        std::vector<const hc_ct*> c(t2m.begin(), t2m.end());
        t2 = new_cts(ctx, m, level - 2, 1, t2m[0]->scale / (double)ctx->P.chain[level - 1]);
        rescale_cts(ctx, c, t2);
        for (int k = 0; k < m; ++k) t2[k]->scale = t2m[k]->scale / (double)ctx->P.chain[level - 1];
      }
      free_all(t2m);
      free_all(t);
      if (a1 != 0) {
        const double cs = t2[0]->scale * (double)ctx->P.chain[level] / xs[0]->scale;
        std::vector<hc_ct*> vm = mul_const_cts(ctx, xs, a1, cs);
        std::vector<const hc_ct*> c(vm.begin(), vm.end());
        std::vector<hc_ct*> v = new_cts(ctx, m, level - 1, 1, vm[0]->scale / (double)ctx->P.chain[level]);
        rescale_cts(ctx, c, v);
        free_all(vm);
        std::vector<BufPtr> keep;
        std::vector<CtRef> tr, vr;
        for (int k = 0; k < m; ++k) {
          check_scales(t2[k]->scale, v[k]->scale);
          tr.push_back(t2[k]->ref());
          vr.push_back(v[k]->ref());  // v's limbs 0..level-2 are its drop to t2's level
        }
        const CtRef* td = refs_dev(ctx, tr, keep);
        launch_ew(ctx, 0, td, td, refs_dev(ctx, vr, keep), m, 2, level - 1);
        free_all(v);
      }
      if (a0 != 0) {
        std::vector<u64> sc;
        constant_residues(ctx, level - 2, a0 * t2[0]->scale, false, sc);
        std::vector<BufPtr> keep;
        std::vector<CtRef> tr;
        for (int k = 0; k < m; ++k) tr.push_back(t2[k]->ref());
        const CtRef* td = refs_dev(ctx, tr, keep);
        launch_scalar(ctx, true, td, td, m, 2, level - 1, upload(ctx, sc, keep));
      }
      for (int k = 0; k < m; ++k) res[idx[k]] = t2[k];
    });
    for (int i = 0; i < n; ++i) y[i] = res[i];
  });
}

extern "C" int hc_enc_pool(hc_ctx* ctx, const hc_evk* evk, hc_packing packing, const hc_ct* const* x, int C, int H,
                           int W, hc_ct** y) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(x && y && C > 0 && H >= 2 && W >= 2, HC_ERR_INVALID, "bad arguments");
    if (packing == HC_PACK_SINGLE) {
      // y + rot(y, W) + rot(y, 1) + rot(y, W + 1), all channels' rotations
      // hoisted together, then x 1/4 and one rescale
      HC_CHECK(evk, HC_ERR_INVALID, "single-ciphertext pooling needs Galois keys");
      std::vector<const hc_ct*> xs(x, x + C);
      for (auto* c : xs) {
        check_ct(ctx, c);
        HC_CHECK(c->degree == 1 && c->level >= 1, HC_ERR_DEPTH, "pooling needs a level");
        HC_CHECK(c->level == xs[0]->level, HC_ERR_LEVEL_MISMATCH, "channels at different levels");
      }
      const int nl = xs[0]->level + 1;
      std::vector<std::vector<hc_ct*>> r = rotate_hoisted_batch(ctx, evk, xs, {W, 1, W + 1});
      std::vector<hc_ct*> s0 = new_cts(ctx, C, xs[0]->level, 1, xs[0]->scale), s1 = new_cts(ctx, C, xs[0]->level, 1, 1.0);
      {
        std::vector<BufPtr> keep;
        std::vector<CtRef> d0, d1, xr, r0, r1, r2;
        for (int c = 0; c < C; ++c) {
          s0[c]->scale = xs[c]->scale;
          s1[c]->scale = r[1][c]->scale;
          d0.push_back(s0[c]->ref());
          d1.push_back(s1[c]->ref());
          xr.push_back(xs[c]->ref());
          r0.push_back(r[0][c]->ref());
          r1.push_back(r[1][c]->ref());
          r2.push_back(r[2][c]->ref());
        }
        const CtRef *dd0 = refs_dev(ctx, d0, keep), *dd1 = refs_dev(ctx, d1, keep);
        launch_ew(ctx, 0, dd0, refs_dev(ctx, xr, keep), refs_dev(ctx, r0, keep), C, 2, nl);
        launch_ew(ctx, 0, dd1, refs_dev(ctx, r1, keep), refs_dev(ctx, r2, keep), C, 2, nl);
        launch_ew(ctx, 0, dd0, dd0, dd1, C, 2, nl);
      }
      std::vector<hc_ct*> o = mulc_rs(ctx, std::vector<const hc_ct*>(s0.begin(), s0.end()), 0.25,
                                      (double)ctx->P.chain[xs[0]->level]);
      for (int c = 0; c < C; ++c) y[c] = o[c];
      free_all(s0);
      free_all(s1);
      for (auto& v : r) free_all(v);
      return;
    }
    HC_CHECK(packing == HC_PACK_BATCH, HC_ERR_INVALID, "unknown packing");
    const int Ho = H / 2, Wo = W / 2, nin = H * W * C, nout = Ho * Wo * C;
    std::vector<const hc_ct*> xs(x, x + nin);
    const int level = xs[0]->level;
    for (auto* c : xs) {
      check_ct(ctx, c);
      HC_CHECK(c->level == level && c->degree == 1, HC_ERR_LEVEL_MISMATCH, "inputs at different levels");
      check_scales(c->scale, xs[0]->scale);
    }
    HC_CHECK(level >= 1, HC_ERR_DEPTH, "no level left");
    std::vector<int> idx;
    for (int i = 0; i < Ho; ++i)
      for (int j = 0; j < Wo; ++j)
        for (int c = 0; c < C; ++c) {
          idx.push_back(((2 * i) * W + 2 * j) * C + c);
          idx.push_back(((2 * i + 1) * W + 2 * j) * C + c);
          idx.push_back(((2 * i) * W + 2 * j + 1) * C + c);
          idx.push_back(((2 * i + 1) * W + 2 * j + 1) * C + c);
        }
    std::vector<hc_ct*> s = new_cts(ctx, nout, level, 1, xs[0]->scale);
    {
      std::vector<BufPtr> keep;
      std::vector<CtRef> xr, sr;
      for (auto* c : xs) xr.push_back(c->ref());
      for (auto* c : s) sr.push_back(c->ref());
      launch_sum4(ctx, refs_dev(ctx, sr, keep), refs_dev(ctx, xr, keep), ids_dev(ctx, idx, keep), nout, level + 1);
    }
    std::vector<const hc_ct*> sc(s.begin(), s.end());
    std::vector<hc_ct*> m = mul_const_cts(ctx, sc, 0.25, (double)ctx->P.chain[level]);
    free_all(s);
    std::vector<const hc_ct*> mc(m.begin(), m.end());
    std::vector<hc_ct*> out = new_cts(ctx, nout, level - 1, 1, m[0]->scale / (double)ctx->P.chain[level]);
    rescale_cts(ctx, mc, out);
    free_all(m);
    for (int i = 0; i < nout; ++i) y[i] = out[i];
  });
}

namespace {
// Degree-2 sums of the FC layer: d_r = sum_k x_k (x) w_{r n_in + k}, the
// weights viewed at the activations' level.  Caller frees the results.
std::vector<hc_ct*> fc_tensor_sums(hc_ctx* ctx, const hc_ct* const* x, int n_in, const hc_ct* const* w, int n_out) {
  std::vector<const hc_ct*> xs(x, x + n_in);
  const int level = xs[0]->level;
  for (auto* c : xs) {
    check_ct(ctx, c);
    HC_CHECK(c->level == level && c->degree == 1, HC_ERR_LEVEL_MISMATCH, "inputs at different levels");
    check_scales(c->scale, xs[0]->scale);
  }
  std::vector<const hc_ct*> ws;
  std::vector<hc_ct*> views;
  for (int i = 0; i < n_in * n_out; ++i) {
    check_ct(ctx, w[i]);
    HC_CHECK(w[i]->level >= level && w[i]->degree == 1, HC_ERR_LEVEL_MISMATCH, "weight below the activations");
    check_scales(w[i]->scale, w[0]->scale);
    views.push_back(new hc_ct{ctx, w[i]->buf, w[i]->data, w[i]->stride, level, 1, w[i]->scale});
    ws.push_back(views.back());
  }
  std::vector<int> xi, wi, off{0};
  for (int r = 0; r < n_out; ++r) {
    for (int k = 0; k < n_in; ++k) {
      xi.push_back(k);
      wi.push_back(r * n_in + k);
    }
    off.push_back((int)xi.size());
  }
  std::vector<hc_ct*> d = tensor_acc(ctx, xs, ws, xi, wi, off, level, xs[0]->scale * ws[0]->scale);
  free_all(views);
  return d;
}
}  // namespace

extern "C" int hc_enc_fc(hc_ctx* ctx, const hc_evk* evk, hc_packing packing, const hc_ct* const* x, int n_in,
                         const hc_ct* const* w, const hc_ct* const* bias, int n_out, hc_ct** y) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(packing == HC_PACK_BATCH, HC_ERR_INVALID, "fc supports batch packing");
    HC_CHECK(evk && x && w && y && n_in > 0 && n_out > 0, HC_ERR_INVALID, "bad arguments");
    HC_CHECK(x[0] && x[0]->level >= 1, HC_ERR_DEPTH, "no level left");
    std::vector<hc_ct*> d = fc_tensor_sums(ctx, x, n_in, w, n_out);
    std::vector<const hc_ct*> bs;
    if (bias)
      for (int r = 0; r < n_out; ++r) {
        check_ct(ctx, bias[r]);
        bs.push_back(bias[r]);
      }
    std::vector<hc_ct*> r = relin_rescale(ctx, evk, d, bias ? &bs : nullptr);
    free_all(d);
    for (int i = 0; i < n_out; ++i) y[i] = r[i];
  });
}

extern "C" int hc_relin_rescale_batch(hc_ctx* ctx, const hc_evk* evk, const hc_ct* const* d, int n, hc_ct** outs) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(evk && d && outs && n > 0, HC_ERR_INVALID, "bad arguments");
    std::vector<hc_ct*> in;
    for (int i = 0; i < n; ++i) {
      check_ct(ctx, d[i]);
      HC_CHECK(d[i]->level == d[0]->level, HC_ERR_LEVEL_MISMATCH, "batch mixes levels");
      in.push_back(const_cast<hc_ct*>(d[i]));  // read only
    }
    std::vector<hc_ct*> r = relin_rescale(ctx, evk, in, nullptr);
    for (int i = 0; i < n; ++i) outs[i] = r[i];
  });
}

extern "C" int hc_enc_fc_partial(hc_ctx* ctx, hc_packing packing, const hc_ct* const* x, int n_in,
                                 const hc_ct* const* w, int n_out, hc_ct** y) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(packing == HC_PACK_BATCH, HC_ERR_INVALID, "fc supports batch packing");
    HC_CHECK(x && w && y && n_in > 0 && n_out > 0, HC_ERR_INVALID, "bad arguments");
    HC_CHECK(x[0], HC_ERR_INVALID, "null input");
    std::vector<hc_ct*> d = fc_tensor_sums(ctx, x, n_in, w, n_out);
    for (int i = 0; i < n_out; ++i) y[i] = d[i];
  });
}

// =====================================================================
// Graph capture
// =====================================================================
struct hc_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<void*> arenas;
  // the other captured contexts' streams, and one event per stream plus one
  // for the origin, ordering each launch against work on those streams
  std::vector<cudaStream_t> joined;
  std::vector<cudaEvent_t> order;
};

namespace {
// The contexts of one capture: non-null, distinct, none capturing, every
// stream not the legacy default.  *stream = the first context's stream (the
// capture's origin); *others = the other contexts' streams, each once.
int check_graph_ctxs(hc_ctx* const* ctxs, int n, cudaStream_t* stream, std::vector<cudaStream_t>* others) {
  if (!ctxs || n <= 0) return HC_ERR_INVALID;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || ctxs[i]->stream == nullptr) return HC_ERR_INVALID;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return HC_ERR_INVALID;
  }
  *stream = ctxs[0]->stream;
  others->clear();
  for (int i = 1; i < n; ++i) {
    const cudaStream_t s = ctxs[i]->stream;
    if (s != *stream && std::find(others->begin(), others->end(), s) == others->end()) others->push_back(s);
  }
  return HC_OK;
}
}  // namespace

// Capture on the first context's stream; every other stream joins the
// capture through an event recorded on the origin (a fork), so the contexts'
// work becomes parallel branches of one graph, joined again at the end.
extern "C" int hc_graph_begin(hc_ctx* const* ctxs, int n, size_t arena_bytes) {
  cudaStream_t st;
  std::vector<cudaStream_t> others;
  int rc = check_graph_ctxs(ctxs, n, &st, &others);
  if (rc != HC_OK) return rc;
  return guard(ctxs[0], [&] {
    const size_t words = std::max<size_t>(arena_bytes / 8, 32);
    for (int i = 0; i < n; ++i) HC_CHECK(!ctxs[i]->arena, HC_ERR_INVALID, "context already capturing");
    HC_CUDA(cudaStreamSynchronize(st));
    for (cudaStream_t s : others) HC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i) {
      void* p = nullptr;
      if (cudaMalloc(&p, words * 8) != cudaSuccess) {
        cudaGetLastError();
        for (int k = 0; k < i; ++k) {
          cudaFree(ctxs[k]->arena);
          ctxs[k]->arena = nullptr;
        }
        throw HcError{HC_ERR_OOM, "cannot allocate the capture arena"};
      }
      ctxs[i]->arena = (u64*)p;
      ctxs[i]->arena_words = words;
      ctxs[i]->arena_off = 0;
    }
    hc_ctx* lead = ctxs[0];
    lead->capture_joined.clear();
    lead->capture_events.assign(2 * others.size(), nullptr);
    for (auto& e : lead->capture_events) HC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    HC_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (size_t k = 0; k < others.size(); ++k) {
      if (cudaEventRecord(lead->capture_events[2 * k], st) != cudaSuccess ||
          cudaStreamWaitEvent(others[k], lead->capture_events[2 * k], 0) != cudaSuccess) {
        // undo: join what was forked, end and drop the capture, free the arenas
        for (size_t j = 0; j < lead->capture_joined.size(); ++j) {
          cudaEventRecord(lead->capture_events[2 * j + 1], lead->capture_joined[j]);
          cudaStreamWaitEvent(st, lead->capture_events[2 * j + 1], 0);
        }
        cudaGraph_t gr = nullptr;
        cudaStreamEndCapture(st, &gr);
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        for (cudaEvent_t e : lead->capture_events) cudaEventDestroy(e);
        lead->capture_events.clear();
        lead->capture_joined.clear();
        for (int i = 0; i < n; ++i) {
          cudaFree(ctxs[i]->arena);
          ctxs[i]->arena = nullptr;
        }
        throw HcError{HC_ERR_CUDA, "cannot fork the capture to another context's stream"};
      }
      lead->capture_joined.push_back(others[k]);
    }
  });
}

extern "C" int hc_graph_end(hc_ctx* const* ctxs, int n, hc_graph** out) {
  cudaStream_t st;
  std::vector<cudaStream_t> others;
  int rc = check_graph_ctxs(ctxs, n, &st, &others);
  if (rc != HC_OK) return rc;
  auto* g = new hc_graph();
  g->stream = st;
  for (int i = 0; i < n; ++i) {
    if (ctxs[i]->arena) g->arenas.push_back(ctxs[i]->arena);
    ctxs[i]->arena = nullptr;
    ctxs[i]->arena_words = ctxs[i]->arena_off = 0;
  }
  hc_ctx* lead = ctxs[0];
  // join every forked stream back into the origin and end the capture,
  // whatever happened while capturing (an invalidated capture fails here)
  const std::vector<cudaStream_t>& joined = lead->capture_joined;
  for (size_t k = 0; k < joined.size() && 2 * k + 1 < lead->capture_events.size(); ++k) {
    cudaEventRecord(lead->capture_events[2 * k + 1], joined[k]);
    cudaStreamWaitEvent(st, lead->capture_events[2 * k + 1], 0);
  }
  const cudaError_t e = cudaStreamEndCapture(st, &g->graph);
  for (cudaEvent_t ev : lead->capture_events) cudaEventDestroy(ev);
  lead->capture_events.clear();
  g->joined = lead->capture_joined;
  lead->capture_joined.clear();
  rc = guard(lead, [&] {
    HC_CHECK(e == cudaSuccess && g->graph, HC_ERR_CUDA, std::string("capture failed: ") + cudaGetErrorString(e));
    HC_CHECK(out, HC_ERR_INVALID, "null output");
    HC_CUDA(cudaGraphInstantiate(&g->exec, g->graph, 0));
    g->order.assign(g->joined.size() + 1, nullptr);
    for (auto& ev : g->order) HC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    *out = g;
  });
  if (rc != HC_OK) {
    cudaGetLastError();
    hc_graph_destroy(g);
  }
  return rc;
}

// The graph runs on the origin stream, after the work already issued on the
// other captured contexts' streams, and later work on those streams waits
// for it: each context sees the launch in its own stream order.
extern "C" int hc_graph_launch(hc_graph* g) {
  if (!g || !g->exec || g->order.size() != g->joined.size() + 1) return HC_ERR_INVALID;
  for (size_t k = 0; k < g->joined.size(); ++k)
    if (cudaEventRecord(g->order[k], g->joined[k]) != cudaSuccess ||
        cudaStreamWaitEvent(g->stream, g->order[k], 0) != cudaSuccess)
      return HC_ERR_CUDA;
  if (cudaGraphLaunch(g->exec, g->stream) != cudaSuccess) return HC_ERR_CUDA;
  if (!g->joined.empty()) {
    if (cudaEventRecord(g->order.back(), g->stream) != cudaSuccess) return HC_ERR_CUDA;
    for (cudaStream_t s : g->joined)
      if (cudaStreamWaitEvent(s, g->order.back(), 0) != cudaSuccess) return HC_ERR_CUDA;
  }
  return HC_OK;
}

extern "C" void hc_graph_destroy(hc_graph* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (cudaEvent_t e : g->order)
    if (e) cudaEventDestroy(e);
  for (void* p : g->arenas) cudaFree(p);
  delete g;
}

// =====================================================================
// Batched single-ciphertext convolution
// =====================================================================
namespace {
int conv2d_single_batch(hc_ctx* ctx, const hc_evk* evk, const hc_ct* const* x, int nimg, int W,
                        const hc_ct* const* w, int cout, int kh, int kw, hc_ct** y, bool hoisted) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(evk && nimg >= 0 && (nimg == 0 || (x && w && y)) && W > 0 && cout > 0 && kh > 0 && kw > 0,
             HC_ERR_INVALID, "bad arguments");
    if (nimg == 0) return;
    const int n = ctx->P.n, T = kh * kw;
    std::vector<int> steps;
    for (int p = 0; p < kh; ++p)
      for (int q = 0; q < kw; ++q) steps.push_back(p * W + q);
    std::vector<u64> gs;
    for (int r : steps) {
      const u64 g = galois_elt(ctx->P, r);
      if (g != 1) HC_CHECK(evk->galois.count(g), HC_ERR_NO_KEY, "no Galois key for rotation " + std::to_string(r));
      gs.push_back(g);
    }
    std::map<int, std::vector<int>> groups;  // level -> image indices
    for (int i = 0; i < nimg; ++i) {
      check_ct(ctx, x[i]);
      HC_CHECK(x[i]->degree == 1 && x[i]->level >= 1, HC_ERR_DEPTH, "images need degree 1 and a level to spend");
      groups[x[i]->level].push_back(i);
    }
    for (int i = 0; i < cout * T; ++i) {
      check_ct(ctx, w[i]);
      HC_CHECK(w[i]->degree == 1, HC_ERR_INVALID, "weights need degree 1");
    }
    // one branch per level: the levels' work overlaps on the device
    const std::vector<std::pair<int, std::vector<int>>> glist(groups.begin(), groups.end());
    fork_join(ctx, (int)glist.size(), [&](int branch) {
      const int level = glist[branch].first, nq = level + 1;
      const std::vector<int>& idx = glist[branch].second;
      const int G = (int)idx.size();
      std::vector<BufPtr> keep;
      std::vector<CtRef> xr;
      std::vector<const hc_ct*> xg;
      for (int gi = 0; gi < G; ++gi) {
        const hc_ct* c = x[idx[gi]];
        check_scales(c->scale, x[idx[0]]->scale);
        xr.push_back(c->ref());
        xg.push_back(c);
      }
      // rotated images, step-major: rot[t * G + g]
      std::vector<hc_ct*> rot;
      if (hoisted) {  // one ModUp per image; every step's key switch after it batched
        std::vector<std::vector<hc_ct*>> hr = rotate_hoisted_batch(ctx, evk, xg, steps);
        for (int t = 0; t < T; ++t)
          for (int gi = 0; gi < G; ++gi) rot.push_back(hr[t][gi]);
      } else {
        rot = new_cts(ctx, T * G, level, 1, x[idx[0]]->scale);
        const CtRef* xrd = refs_dev(ctx, xr, keep);
        // kappa_g of every image for every rotation step into one slab, then one
        // key switch over all (step, image) items with each step's Galois key
        int nrot = 0;
        for (int t = 0; t < T; ++t) nrot += gs[t] != 1;
        BufPtr tmp = ctx->buffer(std::max<size_t>(1, 2 * (size_t)nrot * G * nq * n));
        keep.push_back(tmp);
        std::vector<CtRef> t0, t1, o, src;
        std::vector<const u64*> ks;
        std::vector<u64> gitem;  // each (step, image) item's Galois element
        int nr = 0;              // rotation steps placed so far
        for (int t = 0; t < T; ++t) {
          std::vector<CtRef> ot;
          for (int gi = 0; gi < G; ++gi) ot.push_back(rot[t * G + gi]->ref());
          if (gs[t] == 1) {
            launch_ew(ctx, 3, refs_dev(ctx, ot, keep), xrd, nullptr, G, 2, nq);
            continue;
          }
          for (int gi = 0; gi < G; ++gi) {
            u64* base = tmp->ptr + ((size_t)nr * G + gi) * 2 * nq * n;
            t0.push_back(CtRef{base, (u64)nq * n});
            t1.push_back(CtRef{base + (size_t)nq * n, (u64)nq * n});
            src.push_back(xr[gi]);
            o.push_back(ot[gi]);
            ks.push_back(evk->galois.at(gs[t]).buf->ptr);
            gitem.push_back(gs[t]);
          }
          ++nr;
        }
        if (!o.empty()) {  // t0 holds each item's (c0, c1) pair: one automorphism launch for all
          launch_automorph_items(ctx, refs_dev(ctx, t0, keep), refs_dev(ctx, src, keep), (int)o.size(), 2, nq,
                                 upload(ctx, gitem, keep));
          keyswitch_batch_keys(ctx, ks, level, t1, &t0, nullptr, o);
        }
      }
      // weights viewed at this level
      std::vector<hc_ct*> wv;
      std::vector<const hc_ct*> ws;
      for (int i = 0; i < cout * T; ++i) {
        HC_CHECK(w[i]->level >= level, HC_ERR_LEVEL_MISMATCH, "weight below an image's level");
        wv.push_back(new hc_ct{ctx, w[i]->buf, w[i]->data, w[i]->stride, level, 1, w[i]->scale});
        ws.push_back(wv.back());
      }
      std::vector<const hc_ct*> xs(rot.begin(), rot.end());
      std::vector<int> xi, wi, off{0};
      for (int gi = 0; gi < G; ++gi)
        for (int co = 0; co < cout; ++co) {
          for (int t = 0; t < T; ++t) {
            xi.push_back(t * G + gi);
            wi.push_back(co * T + t);
          }
          off.push_back((int)xi.size());
        }
      std::vector<hc_ct*> d = tensor_acc(ctx, xs, ws, xi, wi, off, level, xs[0]->scale * ws[0]->scale);
      std::vector<hc_ct*> r = relin_rescale(ctx, evk, d, nullptr);
      for (int gi = 0; gi < G; ++gi)
        for (int co = 0; co < cout; ++co) y[idx[gi] * cout + co] = r[gi * cout + co];
      free_all(d);
      free_all(rot);
      free_all(wv);
    });
  });
}
}  // namespace

extern "C" int hc_enc_conv2d_single_batch(hc_ctx* ctx, const hc_evk* evk, const hc_ct* const* x, int nimg, int W,
                                          const hc_ct* const* w, int cout, int kh, int kw, hc_ct** y) {
  return conv2d_single_batch(ctx, evk, x, nimg, W, w, cout, kh, kw, y, false);
}

extern "C" int hc_enc_conv2d_single_hoisted_batch(hc_ctx* ctx, const hc_evk* evk, const hc_ct* const* x, int nimg,
                                                  int W, const hc_ct* const* w, int cout, int kh, int kw,
                                                  hc_ct** y) {
  return conv2d_single_batch(ctx, evk, x, nimg, W, w, cout, kh, kw, y, true);
}

// =====================================================================
// FC by rotate-and-sum (single-ciphertext activations)
// =====================================================================
extern "C" int hc_enc_fc_rotsum(hc_ctx* ctx, const hc_evk* evk, const hc_ct* const* x, int C, const hc_ct* const* w,
                                int n_out, int span_log2, hc_ct** y) {
  if (!ctx) return HC_ERR_INVALID;
  return guard(ctx, [&] {
    HC_CHECK(evk && x && w && y && C > 0 && n_out > 0 && span_log2 >= 0 && span_log2 < ctx->P.log_n, HC_ERR_INVALID,
             "bad arguments");
    std::vector<const hc_ct*> xs(x, x + C);
    const int level = xs[0]->level;
    for (auto* c : xs) {
      check_ct(ctx, c);
      HC_CHECK(c->level == level && c->degree == 1, HC_ERR_LEVEL_MISMATCH, "inputs at different levels");
      check_scales(c->scale, xs[0]->scale);
    }
    HC_CHECK(level >= 1, HC_ERR_DEPTH, "no level left");
    std::vector<hc_ct*> views;
    std::vector<const hc_ct*> ws;
    for (int i = 0; i < C * n_out; ++i) {
      check_ct(ctx, w[i]);
      HC_CHECK(w[i]->level >= level && w[i]->degree == 1, HC_ERR_LEVEL_MISMATCH, "weight below the activations");
      views.push_back(new hc_ct{ctx, w[i]->buf, w[i]->data, w[i]->stride, level, 1, w[i]->scale});
      ws.push_back(views.back());
    }
    std::vector<int> xi, wi, off{0};
    for (int r = 0; r < n_out; ++r) {
      for (int c = 0; c < C; ++c) {
        xi.push_back(c);
        wi.push_back(r * C + c);
      }
      off.push_back((int)xi.size());
    }
    std::vector<hc_ct*> d = tensor_acc(ctx, xs, ws, xi, wi, off, level, xs[0]->scale * ws[0]->scale);
    std::vector<hc_ct*> z = relin_rescale(ctx, evk, d, nullptr);
    free_all(d);
    free_all(views);
    const int nq = level;  // limbs after the rescale = level
    // z += rot(z, 2^k): all outputs rotate together, one batched key switch per k
    for (int k = 0; k < span_log2; ++k) {
      std::vector<hc_ct*> rot = rotate_batch(ctx, evk, std::vector<const hc_ct*>(z.begin(), z.end()), 1 << k);
      std::vector<BufPtr> keep;
      std::vector<CtRef> zr, rr;
      for (int r = 0; r < n_out; ++r) {
        check_scales(z[r]->scale, rot[r]->scale);
        zr.push_back(z[r]->ref());
        rr.push_back(rot[r]->ref());
      }
      const CtRef* zd = refs_dev(ctx, zr, keep);
      launch_ew(ctx, 0, zd, zd, refs_dev(ctx, rr, keep), n_out, 2, nq);
      free_all(rot);
    }
    for (int r = 0; r < n_out; ++r) y[r] = z[r];
  });
}
