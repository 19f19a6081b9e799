// Host-side internals of libhecnn: handle layouts and the launchers that the
// C ABI (hc_api.cu) composes.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "hc_device.cuh"
#include "hecnn.h"

// ----------------------------------------------------------- host helpers
namespace hch {
u64 mulmod(u64 a, u64 b, u64 q);
u64 powmod(u64 a, u64 e, u64 q);
u64 invmod(u64 a, u64 q);
u64 shoup_of(u64 w, u64 q);  // floor(w 2^64 / q)
bool is_prime(u64 n);
int gen_primes(int log_n, const int* bits, int n, u64* out);
std::vector<u64> gaussian_cdt(double sigma);
u64 primitive_2n_root(int log_n, u64 q);
int bit_reverse(int x, int bits);
int64_t round_half_away(double x, bool* ok);
// encode / decode (host FFT, FP64)
void encode_coeffs(const double* re, const double* im, size_t n_slots, int log_n, double scale,
                   std::vector<double>& coeffs);
void decode_slots(const std::vector<double>& coeffs, int log_n, double scale, double* re,
                  double* im, size_t n);
// centred CRT lift of residues [limbs][N] to doubles
void crt_centred_to_double(const u64* res, const u64* primes, int nl, int n, std::vector<double>& out);
}  // namespace hch

struct hc_params {
  int log_n = 0, n = 0, L = 0, alpha = 0, dnum = 0;
  std::vector<u64> chain;  // q_0..q_L, p_0..p_{alpha-1}
  double scale = 0, sigma = 0;
  std::vector<u64> cdt;
  bool below_2_60 = false;  // every prime < 2^60: basis conversions use 30-bit halves
  int nchain() const { return (int)chain.size(); }
};

struct hc_ctx;

// A device allocation returned to the context allocator when the last
// handle referencing it goes away.
struct DevBuf {
  hc_ctx* ctx = nullptr;
  u64* ptr = nullptr;
  size_t bytes = 0;
  bool owned = true;  // false: carved from the context's capture arena
  ~DevBuf();
};
using BufPtr = std::shared_ptr<DevBuf>;

// Key-switching constants of one level (offsets into ctx->ks_dev).
struct LevelConsts {
  int dnum = 0;
  // ModUp digit j: hat_inv[i] (+sh) for i < |D_j|, then hat_mod[t][i] for t < ext
  std::vector<int> modup_off;
  // rescale: q_l^{-1} mod q_i (+sh), then N^{-1} q_l^{-1} (+sh), each for i < l
  int rescale_off = -1;
  // ModUp digit j: offset in hc_ctx::modup_slots of the ext slots outside
  // the digit ([0, d0) then [d1, l + 1 + alpha)), one transform launch each
  std::vector<int> modup_slots_off;
};

// Tile and launch-shape choices (set by hc_autotune or hc_tune_set).
struct HcTune {
  // per log N: 0 = 256-thread blocks, 1 = 128 (the default: measured fastest
  // at N = 2^13..2^16 on GB300), 2 = 64 (N >= 2^13)
  int ntt_variant[17] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
  int kp_zmul = 1;           // key product: item groups in the grid's z, times the default
  int modup_split = 1;       // ModUp conversion: output primes split over this many blocks
  int tensor_group = 5;      // tensor accumulation: 0 = per output, g = up to g outputs sharing x loads
  int host_streams = 2;      // host-to-host call: chunks' kernels round-robin over this many streams (1..4)
};

struct hc_ctx {
  hc_params P;
  HcTune tune;
  int device = 0;
  cudaStream_t stream = nullptr;
  hc_allocator alloc{};
  bool user_alloc = false;
  Tables tab{};
  std::vector<void*> owned;  // table allocations
  u64* ks_dev = nullptr;     // flat constant buffer
  std::vector<LevelConsts> lv;
  int moddown_off = -1;      // (P/p_k)^{-1} N^{-1} mod p_k (+sh); p_k^{-1} mod q_i
  int* ext_map = nullptr;    // [level][L+1+alpha] chain index of ext slot
  int* modup_slots = nullptr;  // per (level, digit): ext slots raised by that digit's ModUp
  std::string err;
  uint64_t launches = 0;
  // tracing: events around launches while `prof` is set
  bool prof = false;
  std::map<std::string, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
  std::map<std::string, uint64_t> prof_units;
  std::vector<cudaEvent_t> event_pool;
  // the last host-to-host call: per chunk, ms from the call's start to the
  // start and end of its copies in, its kernels and its copies out
  std::vector<double> host_timeline;
  // capture arena: while set, buffer() bump-allocates here instead of the allocator
  u64* arena = nullptr;
  size_t arena_words = 0, arena_off = 0;
  // graph capture led by this context: the other contexts' streams joined
  // to it (fork events recorded at the start) and the events to destroy
  std::vector<cudaStream_t> capture_joined;
  // side streams of fork_join (created on first use, destroyed with the context)
  std::vector<cudaStream_t> aux_streams;
  // copy-in and copy-out streams of the host-to-host call, then its extra
  // compute streams (created on first use)
  cudaStream_t copy_streams[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaStream_t flag_stream = nullptr;  // reads a finished host call's range-check flags
  std::vector<cudaEvent_t> capture_events;

  u64* alloc_words(size_t words);
  void free_words(u64* p);
  BufPtr buffer(size_t words);
  const int* ext_map_of(int level) const { return ext_map + level * (P.L + 1 + P.alpha); }
  const int* modup_slots_of(int level, int digit) const { return modup_slots + lv[level].modup_slots_off[digit]; }
  const u64* ks(int off) const { return ks_dev + off; }
};

struct hc_pt {
  hc_ctx* ctx;
  BufPtr buf;
  u64* data;  // [level+1][N], NTT form
  int level;
  double scale;
};

// A host-to-host call in flight (hc_mul_relin_rescale_host_eval_async): its
// events, the buffers it still uses and its range-check flags.
struct hc_host_op {
  hc_ctx* ctx = nullptr;
  std::vector<cudaEvent_t> evs;  // every event of the call (destroyed at the end)
  std::vector<cudaEvent_t> tev;  // per chunk: copies in, kernels, copies out (begin, end)
  cudaEvent_t t_start = nullptr;
  cudaEvent_t drained = nullptr;  // the last copy out
  std::vector<BufPtr> keep;
  BufPtr flags;
  int nch = 0;
};

struct hc_ct {
  hc_ctx* ctx;
  BufPtr buf;
  u64* data;  // poly k, limb i at data + k*stride + i*N (NTT form)
  u64 stride;
  int level;
  int degree;
  double scale;
  CtRef ref() const { return CtRef{data, stride}; }
};

struct SwitchKeyDev {
  BufPtr buf;  // [dnum][2][L+1+alpha][N], NTT form, chain order
};

struct hc_secret_key {
  hc_ctx* ctx;
  BufPtr s_ntt;  // [L+1+alpha][N] s in NTT form over the whole chain
  std::vector<int8_t> s_coeff;
};

struct hc_public_key {
  hc_ctx* ctx;
  BufPtr buf;  // [2][L+1][N] (b, a) NTT form
};

struct hc_eval_keys {
  hc_ctx* ctx;
  SwitchKeyDev relin;
  std::map<u64, SwitchKeyDev> galois;
};

// Error plumbing.
struct HcError {
  int code;
  std::string msg;
};
#define HC_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw HcError{HC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define HC_CHECK(cond, code, msg) \
  do {                            \
    if (!(cond)) throw HcError{code, msg}; \
  } while (0)

void check_launch(hc_ctx* ctx);

// Brackets one kernel launch with events when the context is profiling.
struct ProfScope {
  hc_ctx* ctx;
  cudaEvent_t a = nullptr, b = nullptr;
  const char* name;
  uint64_t units;
  ProfScope(hc_ctx* c, const char* n, uint64_t u = 0);
  ~ProfScope();
};

// Writes `words` host words to device memory in stream order: a pageable
// copy normally, kernels carrying the words as parameters while the stream
// is being captured into a graph (so the graph holds the values).
void upload_words(hc_ctx* ctx, u64* dst, const u64* src, size_t words);

// Upload a small host array to fresh device memory owned by `keep`.
template <class T>
T* upload(hc_ctx* ctx, const std::vector<T>& v, std::vector<BufPtr>& keep) {
  if (v.empty()) return nullptr;
  size_t words = (v.size() * sizeof(T) + 7) / 8;
  BufPtr b = ctx->buffer(words);
  std::vector<u64> tmp(words, 0);
  std::memcpy(tmp.data(), v.data(), v.size() * sizeof(T));
  upload_words(ctx, b->ptr, tmp.data(), words);
  keep.push_back(b);
  return reinterpret_cast<T*>(b->ptr);
}

// --------------------------------------------------------------- launchers
// NTT (forward) / inverse NTT of every limb of a LimbSet, `items` items.
// scale = false (inverse only) leaves out the factor N^{-1}: the result is N
// times the inverse transform, for consumers that fold N^{-1} into their
// own constants (the basis conversions of ModUp and ModDown).
void launch_ntt(hc_ctx* ctx, const LimbSet& s, int items, bool inverse, bool scale = true);
// Out-of-place: the first pass reads limb (item, poly, limb) from `in`
// (same poly/limb counts as s), the result lands in s.
void launch_ntt_from(hc_ctx* ctx, const LimbSet& s, const LimbSet* in, int items, bool inverse,
                     bool scale = true);
// Forward NTT of the converted limbs z (2 polys x level limbs per item)
// carrying the fused relinearise + rescale tail (KsrFuse): writes f.out.
void launch_ntt_ksr(hc_ctx* ctx, const LimbSet& z, int items, const KsrFuse& f);
// Inverse NTT into `out` (2 polys x level plain limbs per item) carrying the
// coefficient-form tail of KsrFuse: out holds the relinearised and rescaled
// polynomials in coefficient form (f.out is not used).
void launch_intt_ksr(hc_ctx* ctx, const LimbSet& out, int items, const KsrFuse& f);

// Samplers writing coefficient-form limbs dst + r*N for chain indices ids[r].
void launch_sample_ternary(hc_ctx* ctx, u64 seed, u64 tag, u64* dst, const int* ids, int nl);
void launch_sample_gauss(hc_ctx* ctx, u64 seed, u64 tag, u64* dst, const int* ids, int nl);
void launch_sample_uniform(hc_ctx* ctx, u64 seed, u64 tag, u64* dst, const int* ids, int nl);
void launch_reduce_signed(hc_ctx* ctx, const int64_t* src, u64* dst, const int* ids, int nl);

// Elementwise over `items` cts of `npoly` polys x `nl` limbs (limb i mod q_i):
// op 0: out = a + b, 1: out = a - b, 2: out = a * b (pointwise), 3: out = a (copy)
void launch_ew(hc_ctx* ctx, int op, const CtRef* out, const CtRef* a, const CtRef* b, int items,
               int npoly, int nl);
// out = a * s_i (per-limb scalar, all polys) / out = a + s_i on poly 0 only
void launch_scalar(hc_ctx* ctx, bool add, const CtRef* out, const CtRef* a, int items, int npoly,
                   int nl, const u64* scal_dev);
// Tensor products with lazy 128-bit accumulation:
// out[o] = sum_{t<terms[o]} x[xi[o0+t]] (x) w[wi[o0+t]], o0 = off[o].
// out[z] = a[z] (x) b[z], degree-1 operands, one term per output.
void launch_tensor_pair(hc_ctx* ctx, const CtRef* out, const CtRef* a, const CtRef* b, int items, int nl);
// Grouped form: groups of G (1..5) outputs sharing one x sequence,
//   out[g G + k] = sum_{t in [off[g], off[g+1])} x[xi[t]] (x) w[wi[t G + k]],
// the same words as the per-output form with the x operands loaded once.
void launch_tensor_acc_grouped(hc_ctx* ctx, int G, const CtRef* out, const CtRef* x, const CtRef* w, const int* xi,
                               const int* wi, const int* off, int ngroups, int nl, uint64_t terms);
// `terms` (the sum of the outputs' term counts) only labels the launch's
// work for profiling: one unit per (term, limb).
void launch_tensor_acc(hc_ctx* ctx, const CtRef* out, const CtRef* x, const CtRef* w,
                       const int* xi, const int* wi, const int* off, int nout, int nl, uint64_t terms);
// NTT-domain automorphism: out = kappa_g(a) for `items` refs, npoly polys, nl limbs.
void launch_automorph(hc_ctx* ctx, const CtRef* out, const CtRef* a, int items, int npoly, int nl,
                      u64 g);
// The same with a Galois element per item (gs: device array of `items`).
void launch_automorph_items(hc_ctx* ctx, const CtRef* out, const CtRef* a, int items, int npoly, int nl,
                            const u64* gs);
// ModUp basis conversion of digit j at level `level`: reads coefficient-form
// limbs of x (items), writes the ext limbs outside the digit into ext.
void launch_modup_bconv(hc_ctx* ctx, int level, int j, const u64* xcoef, u64 x_item_stride,
                        u64* ext, u64 ext_item_stride, int items);
// Key product: acc[z][k][slot] = sum_j ext[z][j][slot] * key_j[k][chain(slot)]
// (keys stored in Montgomery form, their Q limbs times P^{-1}: the Q slots of
// acc come out divided by P modulo q_i).
void launch_key_product(hc_ctx* ctx, int level, const u64* ext, u64 ext_item_stride,
                        const u64* key, u64* acc, u64 acc_item_stride, int items);
// ModDown conversion of the P part of acc (coefficient form) into z over
// Q_level, times P^{-1} (folded into the constants).
void launch_moddown_bconv(hc_ctx* ctx, int level, const u64* accp_coef, u64 accp_item_stride,
                          u64* z, u64 z_item_stride, int items);
// out_k = base_k + acc_k - z_k over Q_level (base may be null per k): ModDown
// with P^{-1} already in acc's Q limbs (the keys) and in z (the constants).
void launch_moddown_combine(hc_ctx* ctx, int level, const u64* acc, u64 acc_item_stride, const u64* z,
                            u64 z_item_stride, const CtRef* base0, const CtRef* base1, const CtRef* out,
                            int items, const u64* base0_gs = nullptr);  // base0 read through kappa_{gs[z]}
// Rescale: lift[z][k][i] = centred(last[z][k]) mod q_i, i < level.
void launch_rescale_lift(hc_ctx* ctx, int level, const u64* last, u64* lift, int items, int npoly);
// out[z][k][i] = (in_i - lift_i) * q_level^{-1}.
void launch_rescale_combine(hc_ctx* ctx, int level, const CtRef* in, const u64* lift,
                            const CtRef* out, int items, int npoly);
// Copies limb `slot` of each poly of each item into dst[z][k].
void launch_gather_limb(hc_ctx* ctx, const CtRef* src, int slot, u64* dst, int items, int npoly);
// Validity check: counts residues >= q (writes count to *bad).
void launch_check_range(hc_ctx* ctx, const u64* data, int npoly, int nl, u64 poly_stride,
                        unsigned long long* bad);
// Pool sums: out[o] = (x[i0] + x[i1]) + (x[i2] + x[i3]) with idx[4o..4o+3].
void launch_sum4(hc_ctx* ctx, const CtRef* out, const CtRef* x, const int* idx, int nout, int nl);

// Specialised key-switching launchers (same results as the generic ones).
void launch_modup_bconv_fast(hc_ctx* ctx, int level, int j, const u64* xcoef, u64 x_item_stride, u64* ext,
                             u64 ext_item_stride, int items, int ndig = 1);  // digits j .. j + ndig - 1, all full
void launch_moddown_bconv_fast(hc_ctx* ctx, int level, const u64* accp_coef, u64 accp_item_stride, u64* z,
                               u64 z_item_stride, int items);
void launch_key_product_batched(hc_ctx* ctx, int level, const u64* ext, u64 ext_item_stride, const u64* key,
                                u64* acc, u64 acc_item_stride, int items, const CtRef* digit_src = nullptr,
                                const u64* const* item_keys = nullptr,  // per-item keys override `key`
                                const u64* gs = nullptr,                // per-item Galois element: read kappa_g(ext)
                                int ext_items = 0);                     // item z reads ext item z % ext_items
// Fused relinearise + rescale tail (see hc_kernels.cu).
void launch_ksr_last(hc_ctx* ctx, int level, const u64* acc, u64 acc_item_stride, const CtRef* base0,
                     const CtRef* base1, u64* tl, int items);
// In place over tl: the centred c_l = t_k - z_k[l] mod q_l (z carrying
// P^{-1}) as a signed
// integer per coefficient (coefficient-form tl from the inverse NTT).
void launch_ksr_cl(hc_ctx* ctx, int level, u64* tl, const u64* zq, u64 z_item_stride, int items);
// Constants of the fused tail at `level` (q_l^{-1}, N^{-1} q_l^{-1}, whether c_l needs reducing) into f.
void ksr_constants(hc_ctx* ctx, int level, KsrFuse& f);
