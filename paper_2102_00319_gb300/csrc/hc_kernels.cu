// Pointwise and basis-conversion kernels of libhecnn.  Every kernel maps one
// thread to one coefficient of one limb; grids are (N / 256, limbs, items).
#include <algorithm>

#include "hc_internal.h"

namespace {
constexpr int kT = 256;

inline dim3 grid_for(hc_ctx* ctx, int ylimbs, int items) {
  return dim3((unsigned)((ctx->P.n + kT - 1) / kT), (unsigned)ylimbs, (unsigned)items);
}

// --------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, key bumped
// by the Weyl constants between rounds.
__device__ void philox4x64(u64 c0, u64 c1, u64 c2, u64 c3, u64 k0, u64 k1, u64 out[4]) {
  const u64 M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const u64 W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const u64 lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    const u64 lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    const u64 n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// Word i of stream (seed, tag, lane).
__device__ __forceinline__ u64 stream_word(u64 seed, u64 tag, u64 lane, u64 i) {
  u64 o[4];
  philox4x64(i >> 2, lane, 0, 0, seed, tag, o);
  return o[i & 3];
}

__device__ __forceinline__ u64 signed_res(long long v, u64 q) {
  if (v >= 0) return (u64)v % q;
  u64 m = (u64)(-(v + 1)) % q;
  return q - 1 - m;
}

__global__ void k_ternary(u64 seed, u64 tag, u64* dst, const int* ids, int nl, Tables T) {
  const int n = 1 << T.log_n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long v = (long long)(stream_word(seed, tag, 0, (u64)i) % 3) - 1;
  for (int r = 0; r < nl; ++r) dst[(size_t)r * n + i] = signed_res(v, T.mods[ids[r]].q);
}

struct Cdt {
  u64 t[40];
  int n;
};

__global__ void k_gauss(u64 seed, u64 tag, u64* dst, const int* ids, int nl, Tables T, Cdt cdt) {
  const int n = 1 << T.log_n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u64 w = stream_word(seed, tag, 0, (u64)i), r = w >> 1;
  long long mag = 0;
  for (int k = 0; k < cdt.n; ++k) mag += (r >= cdt.t[k]) ? 1 : 0;
  const long long v = (w & 1) ? -mag : mag;
  for (int l = 0; l < nl; ++l) dst[(size_t)l * n + i] = signed_res(v, T.mods[ids[l]].q);
}

__global__ void k_uniform(u64 seed, u64 tag, u64* dst, const int* ids, Tables T) {
  const int n = 1 << T.log_n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int pid = ids[blockIdx.y];
  u64 o[4];
  philox4x64((u64)i >> 1, (u64)pid, 0, 0, seed, tag, o);
  const int w = 2 * (i & 1);
  dst[(size_t)blockIdx.y * n + i] = reduce128(U128{o[w], o[w + 1]}, T.mods[pid]);
}

__global__ void k_reduce_signed(const long long* src, u64* dst, const int* ids, Tables T) {
  const int n = 1 << T.log_n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[(size_t)blockIdx.y * n + i] = signed_res(src[i], T.mods[ids[blockIdx.y]].q);
}

// ---------------------------------------------------------- elementwise
__global__ void k_ew(int op, const CtRef* out, const CtRef* a, const CtRef* b, int nl, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y / nl, l = blockIdx.y % nl, z = blockIdx.z;
  const size_t off = (size_t)l * n + c;
  const u64 x = a[z].p[k * a[z].stride + off];
  const u64 q = T.mods[l].q;
  u64 r;
  if (op == 3) {
    r = x;
  } else {
    const u64 y = b[z].p[k * b[z].stride + off];
    if (op == 0) r = addm(x, y, q);
    else if (op == 1) r = subm(x, y, q);
    else r = mulm(x, y, T.mods[l]);
  }
  out[z].p[k * out[z].stride + off] = r;
}

// scal: [nl] values then [nl] Shoup companions (for the multiply)
__global__ void k_scalar(bool add, const CtRef* out, const CtRef* a, int nl, const u64* scal, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y / nl, l = blockIdx.y % nl, z = blockIdx.z;
  const size_t off = (size_t)l * n + c;
  const u64 x = a[z].p[k * a[z].stride + off];
  const u64 q = T.mods[l].q;
  u64 r;
  if (add) r = (k == 0) ? addm(x, scal[l], q) : x;
  else r = shoup(x, scal[l], scal[nl + l], q);
  out[z].p[k * out[z].stride + off] = r;
}

// out[o] = sum_t x[xi[off[o]+t]] (x) w[wi[off[o]+t]], degree 2, lazily in 128 bits.
__global__ void k_tensor_acc(const CtRef* out, const CtRef* x, const CtRef* w, const int* xi, const int* wi,
                             const int* off, int nl, int chunk, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  // limb-major grid: every output of one limb runs before the next limb, so
  // the operands shared by many outputs (a conv's weights, overlapping
  // windows) stay in L2 while that limb is processed
  const int o = blockIdx.y, l = blockIdx.z;
  const DMod md = T.mods[l];
  const size_t lo = (size_t)l * n + c;
  // Karatsuba per term: s += (x0 + x1)(w0 + w1), so that the middle sum is
  // s - a0 - a2 (exact: s dominates a0 + a2 term by term); three products
  // per term instead of four
  U128 a0{0, 0}, s{0, 0}, a2{0, 0};
  const int t0 = off[o], t1 = off[o + 1];
  int cnt = 0;
  auto middle = [&]() {  // s - a0 - a2 in 128 bits
    U128 m = s;
    u64 t = m.lo - a0.lo;
    m.hi -= a0.hi + (m.lo < a0.lo);
    m.lo = t;
    t = m.lo - a2.lo;
    m.hi -= a2.hi + (m.lo < a2.lo);
    m.lo = t;
    return m;
  };
  for (int t = t0; t < t1; ++t) {
    const CtRef X = x[xi[t]], Wt = w[wi[t]];
    const u64 x0 = X.p[lo], x1 = X.p[X.stride + lo];
    const u64 w0 = Wt.p[lo], w1 = Wt.p[Wt.stride + lo];
    mac(a0, x0, w0);
    mac(s, x0 + x1, w0 + w1);
    mac(a2, x1, w1);
    if (++cnt == chunk) {
      // fold: keep the three sums' residues, with s carrying r0 + r1 + r2 so
      // that s - a0 - a2 still yields the middle residue
      cnt = 0;
      const u64 r1 = reduce128_est(middle(), md);
      const u64 r0 = reduce128_est(a0, md), r2 = reduce128_est(a2, md);
      a0 = U128{r0, 0};
      a2 = U128{r2, 0};
      s = U128{r0 + r1 + r2, 0};
    }
  }
  const CtRef O = out[o];
  O.p[lo] = reduce128_est(a0, md);
  O.p[O.stride + lo] = reduce128_est(middle(), md);
  O.p[2 * O.stride + lo] = reduce128_est(a2, md);
}

// G outputs that share one sequence of x operands (the output channels of a
// conv position, the classes of an FC layer):
//   out[g G + k] = sum_{t in [off[g], off[g+1])} x[xi[t]] (x) w[wi[t G + k]],
// accumulated like k_tensor_acc (Karatsuba per term, 128-bit sums folded every
// `chunk` terms).  Each x word is loaded once for its G products, which cuts
// the operand loads per term from 4 to 2 + 2/G words.  The operands' limb
// pointers are staged in shared memory a tile of terms at a time by the
// whole block (one group and one limb per block), so the term loop issues
// only independent data loads instead of chains of dependent pointer loads.
template <int G>
__global__ void __launch_bounds__(kT, G >= 4 ? 2 : 3) k_tensor_acc_g(const CtRef* out, const CtRef* x, const CtRef* w,
                                                     const int* xi, const int* wi, const int* off, int chunk,
                                                     Tables T) {
  constexpr int TT = 32;  // terms per staged tile
  __shared__ const u64* s_xp[TT];
  __shared__ u64 s_xs[TT];
  __shared__ const u64* s_wp[TT][G];
  __shared__ u64 s_wstr[TT][G];
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;  // n is a multiple of the block size
  const int g = blockIdx.y, l = blockIdx.z;
  const DMod md = T.mods[l];
  const size_t lofs = (size_t)l * n;
  U128 a0[G], sm[G], a2[G];
#pragma unroll
  for (int k = 0; k < G; ++k) a0[k] = sm[k] = a2[k] = U128{0, 0};
  auto middle = [](const U128& s, const U128& x0, const U128& x2) {  // s - x0 - x2 in 128 bits
    U128 m = s;
    u64 t = m.lo - x0.lo;
    m.hi -= x0.hi + (m.lo < x0.lo);
    m.lo = t;
    t = m.lo - x2.lo;
    m.hi -= x2.hi + (m.lo < x2.lo);
    m.lo = t;
    return m;
  };
  const int t0 = off[g], t1 = off[g + 1];
  int cnt = 0;
  for (int tb = t0; tb < t1; tb += TT) {
    const int nt = min(TT, t1 - tb);
    __syncthreads();  // the previous tile's pointers are no longer read
    for (int i = threadIdx.x; i < nt * (G + 1); i += blockDim.x) {
      const int t = i / (G + 1), k = i - t * (G + 1);
      if (k == 0) {
        const CtRef X = x[xi[tb + t]];
        s_xp[t] = X.p + lofs;
        s_xs[t] = X.stride;
      } else {
        const CtRef Wt = w[wi[(size_t)(tb + t) * G + (k - 1)]];
        s_wp[t][k - 1] = Wt.p + lofs;
        s_wstr[t][k - 1] = Wt.stride;
      }
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      const u64* xp = s_xp[t] + c;
      const u64 x0 = xp[0], x1 = xp[s_xs[t]];
      const u64 xsum = x0 + x1;
#pragma unroll
      for (int k = 0; k < G; ++k) {
        const u64* wp = s_wp[t][k] + c;
        const u64 w0 = wp[0], w1 = wp[s_wstr[t][k]];
        mac(a0[k], x0, w0);
        mac(sm[k], xsum, w0 + w1);
        mac(a2[k], x1, w1);
      }
      if (++cnt == chunk) {
        cnt = 0;
#pragma unroll
        for (int k = 0; k < G; ++k) {
          const u64 r1 = reduce128_est(middle(sm[k], a0[k], a2[k]), md);
          const u64 r0 = reduce128_est(a0[k], md), r2 = reduce128_est(a2[k], md);
          a0[k] = U128{r0, 0};
          a2[k] = U128{r2, 0};
          sm[k] = U128{r0 + r1 + r2, 0};
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < G; ++k) {
    const CtRef O = out[(size_t)g * G + k];
    const size_t lo = lofs + c;
    O.p[lo] = reduce128_est(a0[k], md);
    O.p[O.stride + lo] = reduce128_est(middle(sm[k], a0[k], a2[k]), md);
    O.p[2 * O.stride + lo] = reduce128_est(a2[k], md);
  }
}

// out[z] = a[z] (x) b[z] (one term per output): d0 = a0 b0, d2 = a1 b1 and
// d1 = (a0 + a1)(b0 + b1) - d0 - d2 in 128 bits (three products instead of
// four; a0 + a1 < 2q keeps the product below 2^124 and the difference is the
// exact a0 b1 + a1 b0).
__global__ void k_tensor_pair(const CtRef* out, const CtRef* a, const CtRef* b, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int l = blockIdx.y, z = blockIdx.z;
  const DMod md = T.mods[l];
  const CtRef A = a[z], B = b[z], O = out[z];
  const size_t lo = (size_t)l * n + c;
  const u64 a0 = A.p[lo], a1 = A.p[A.stride + lo], b0 = B.p[lo], b1 = B.p[B.stride + lo];
  const U128 p0{a0 * b0, __umul64hi(a0, b0)}, p2{a1 * b1, __umul64hi(a1, b1)};
  const u64 sa = a0 + a1, sb = b0 + b1;
  U128 p1{sa * sb, __umul64hi(sa, sb)};
  // p1 -= p0 + p2 (no borrow out: the result is a0 b1 + a1 b0 >= 0)
  u64 t = p1.lo - p0.lo;
  p1.hi -= p0.hi + (p1.lo < p0.lo);
  p1.lo = t;
  t = p1.lo - p2.lo;
  p1.hi -= p2.hi + (p1.lo < p2.lo);
  p1.lo = t;
  O.p[lo] = reduce128_est(p0, md);
  O.p[O.stride + lo] = reduce128_est(p1, md);
  O.p[2 * O.stride + lo] = reduce128_est(p2, md);
}

// NTT-domain automorphism: slot k holds a(psi^{e_k}), e_k = 2 brv(k) + 1;
// kappa_g(a)(psi^{e}) = a(psi^{e g}).
// gs (may be null): per-item Galois elements, overriding g.
// The slot of kappa_g's input that lands in slot k of its output, for
// polynomials in NTT form with bit-reversed evaluation order: slot k holds
// the evaluation at psi^e, e = 2 brev(k) + 1, and kappa_g(a)(psi^e) =
// a(psi^{e g}).
__device__ __forceinline__ int automorph_src(int k, u64 g, int logn) {
  const u64 mask = (2ull << logn) - 1;
  const u64 e = 2 * (u64)(__brev((unsigned)k) >> (32 - logn)) + 1;
  const u64 e2 = (e * g) & mask;
  return (int)(__brev((unsigned)((e2 - 1) >> 1)) >> (32 - logn));
}

__global__ void k_automorph(const CtRef* out, const CtRef* a, int nl, u64 g, const u64* gs, Tables T) {
  const int logn = T.log_n, n = 1 << logn;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int poly = blockIdx.y / nl, l = blockIdx.y % nl, z = blockIdx.z;
  const int src = automorph_src(k, gs ? gs[blockIdx.z] : g, logn);
  out[z].p[poly * out[z].stride + (size_t)l * n + k] = a[z].p[poly * a[z].stride + (size_t)l * n + src];
}

// ModUp: v_i = [x_i hat_inv_i]_{q_i}; y_t = sum_i v_i hat_mod[t][i] mod q_t.
__global__ void k_modup_bconv(const u64* xcoef, u64 x_item_stride, u64* ext, u64 ext_item_stride,
                              const u64* cst, int d0, int ns, int next, const int* emap, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int z = blockIdx.z;
  const u64* x = xcoef + (size_t)z * x_item_stride;
  u64* y = ext + (size_t)z * ext_item_stride;
  u64 v[16];
  for (int i = 0; i < ns; ++i) {
    const u64 q = T.mods[emap[d0 + i]].q;
    v[i] = shoup(x[(size_t)(d0 + i) * n + c], cst[i], cst[ns + i], q);
  }
  const u64* hm = cst + 2 * ns;
  for (int t = 0; t < next; ++t) {
    if (t >= d0 && t < d0 + ns) continue;
    const DMod md = T.mods[emap[t]];
    U128 acc{0, 0};
    for (int i = 0; i < ns; ++i) mac(acc, v[i], hm[t * ns + i]);
    y[(size_t)t * n + c] = reduce128(acc, md);
  }
}

// acc[z][k][s] = sum_j ext[z][j][s] * key[j][k][emap[s]].  Switching keys are
// stored in Montgomery form (key 2^64 mod q), so one Montgomery reduction of
// the sum gives the plain residue.  Any digit count: the sum is folded (an
// exact reduction that keeps the factor 2^64) after every 7 terms, so its
// high word stays below q.
__global__ void k_key_product(const u64* ext, u64 ext_item_stride, const u64* key, u64* acc,
                              u64 acc_item_stride, int dnum, int next, int nchain, const int* emap,
                              const u64* const* item_keys, const u64* gs, int ext_items, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int s = blockIdx.y, z = blockIdx.z;
  const int pid = emap[s];
  const DMod md = T.mods[pid];
  // item z reads the raised digits of item z mod ext_items, through kappa_g when gs is given
  const int ce = gs ? automorph_src(c, gs[z], T.log_n) : c;
  const u64* e = ext + (size_t)(z < ext_items ? z : z % ext_items) * ext_item_stride + (size_t)s * n + ce;
  U128 a0{0, 0}, a1{0, 0};
  for (int j = 0; j < dnum; ++j) {
    if (j > 0 && j % 7 == 0) {
      a0 = U128{reduce128(a0, md), 0};
      a1 = U128{reduce128(a1, md), 0};
    }
    const u64 y = e[(size_t)j * next * n];
    const u64* kz = item_keys ? item_keys[z] : key;  // per-item switching key, if given
    const u64* kb = kz + ((size_t)(2 * j) * nchain + pid) * n + c;
    const u64* ka = kz + ((size_t)(2 * j + 1) * nchain + pid) * n + c;
    mac(a0, y, *kb);
    mac(a1, y, *ka);
  }
  u64* o = acc + (size_t)z * acc_item_stride + (size_t)s * n + c;
  o[0] = redc(a0, md);
  o[(size_t)next * n] = redc(a1, md);
}

// ModDown conversion P -> Q_level of both polys, times P^{-1}.
// cst: [alpha] hat_inv, [alpha] hat_inv_sh, [L+1][alpha] hat_mod with
// hat_mod[t][k] = (P/p_k) P^{-1} = p_k^{-1} mod q_t
__global__ void k_moddown_bconv(const u64* src, u64 src_item_stride, u64 src_poly_stride, u64* zq,
                                u64 z_item_stride, const u64* cst, int alpha, int nq, int L,
                                Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y, z = blockIdx.z;
  const u64* x = src + (size_t)z * src_item_stride + (size_t)k * src_poly_stride;
  u64 v[16];
  for (int i = 0; i < alpha; ++i) {
    const u64 q = T.mods[L + 1 + i].q;
    v[i] = shoup(x[(size_t)i * n + c], cst[i], cst[alpha + i], q);
  }
  const u64* hm = cst + 2 * alpha;
  u64* out = zq + (size_t)z * z_item_stride + (size_t)k * nq * n;
  for (int t = 0; t < nq; ++t) {
    U128 acc{0, 0};
    for (int i = 0; i < alpha; ++i) mac(acc, v[i], hm[t * alpha + i]);
    out[(size_t)t * n + c] = reduce128(acc, T.mods[t]);
  }
}

// out_k = base_k + u_k - NTT(z_k): the key product's Q limbs u and the
// conversion z both carry ModDown's P^{-1} already.
// GATHER: base0 is read through item z's automorphism kappa_{gs[z]} (the
// c0 of a hoisted rotation), so it needs no automorphed copy of its own.
template <bool GATHER>
__global__ void k_moddown_combine(const u64* acc, u64 acc_item_stride, u64 acc_poly_stride,
                                  const u64* zq, u64 z_item_stride, const CtRef* base0,
                                  const CtRef* base1, const CtRef* out, int nq, const u64* gs, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y / nq, i = blockIdx.y % nq, z = blockIdx.z;
  const u64 q = T.mods[i].q;
  const size_t li = (size_t)i * n + c;
  const u64 u = acc[(size_t)z * acc_item_stride + (size_t)k * acc_poly_stride + li];
  const u64 zz = zq[(size_t)z * z_item_stride + (size_t)k * nq * n + li];
  u64 r = subm(u, zz, q);
  const CtRef* base = k == 0 ? base0 : base1;
  if (base) {
    size_t bi = li;
    if constexpr (GATHER) {
      if (k == 0) bi = (size_t)i * n + automorph_src(c, gs[z], T.log_n);
    }
    r = addm(r, base[z].p[bi], q);
  }
  out[z].p[(size_t)k * out[z].stride + li] = r;
}

__global__ void k_gather_limb(const CtRef* src, int slot, u64* dst, int npoly, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y, z = blockIdx.z;
  dst[((size_t)z * npoly + k) * n + c] = src[z].p[(size_t)k * src[z].stride + (size_t)slot * n + c];
}

// lift[z][k][i] = centred(last[z][k]) mod q_i
__global__ void k_rescale_lift(const u64* last, u64* lift, int level, int npoly, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int i = blockIdx.y % level, k = blockIdx.y / level, z = blockIdx.z;
  const u64 ql = T.mods[level].q;
  const DMod mi = T.mods[i];
  const u64 r = last[((size_t)z * npoly + k) * n + c];
  u64 v;
  if (r > (ql - 1) / 2) {
    const u64 m = csub(shoup_lazy(ql - r, 1, mi.one_sh, mi.q), mi.q);  // (q_l - r) mod q_i
    v = negm(m, mi.q);
  } else {
    v = csub(shoup_lazy(r, 1, mi.one_sh, mi.q), mi.q);
  }
  lift[(((size_t)z * npoly + k) * level + i) * n + c] = v;
}

// cst: [level] q_l^{-1} mod q_i, [level] Shoup companions
__global__ void k_rescale_combine(const CtRef* in, const u64* lift, const CtRef* out, const u64* cst,
                                  int level, int npoly, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int i = blockIdx.y % level, k = blockIdx.y / level, z = blockIdx.z;
  const u64 q = T.mods[i].q;
  const u64 x = in[z].p[(size_t)k * in[z].stride + (size_t)i * n + c];
  const u64 y = lift[(((size_t)z * npoly + k) * level + i) * n + c];
  out[z].p[(size_t)k * out[z].stride + (size_t)i * n + c] = shoup(subm(x, y, q), cst[i], cst[level + i], q);
}

__global__ void k_check_range(const u64* data, int nl, u64 poly_stride, unsigned long long* bad, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y / nl, l = blockIdx.y % nl;
  if (data[(size_t)k * poly_stride + (size_t)l * n + c] >= T.mods[l].q) atomicAdd(bad, 1ull);
}

__global__ void k_sum4(const CtRef* out, const CtRef* x, const int* idx, int nl, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y / nl, l = blockIdx.y % nl, o = blockIdx.z;
  const u64 q = T.mods[l].q;
  const size_t off = (size_t)l * n + c;
  const int* id = idx + 4 * o;
  const CtRef A = x[id[0]], B = x[id[1]], C = x[id[2]], D = x[id[3]];
  const u64 s1 = addm(A.p[k * A.stride + off], B.p[k * B.stride + off], q);
  const u64 s2 = addm(C.p[k * C.stride + off], D.p[k * D.stride + off], q);
  out[o].p[k * out[o].stride + off] = addm(s1, s2, q);
}

}  // namespace

namespace {
constexpr int kFillWords = 480;  // 3840 bytes of kernel parameters
struct FillBlock {
  u64 w[kFillWords];
};
__global__ void k_fill(u64* dst, FillBlock b, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = b.w[i];
}
}  // namespace

void upload_words(hc_ctx* ctx, u64* dst, const u64* src, size_t words) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  HC_CUDA(cudaStreamIsCapturing(ctx->stream, &st));
  if (st == cudaStreamCaptureStatusNone) {
    HC_CUDA(cudaMemcpyAsync(dst, src, words * sizeof(u64), cudaMemcpyHostToDevice, ctx->stream));
    return;
  }
  for (size_t o = 0; o < words; o += kFillWords) {
    FillBlock b;
    const int n = (int)std::min<size_t>(kFillWords, words - o);
    std::memcpy(b.w, src + o, n * sizeof(u64));
    k_fill<<<1, 128, 0, ctx->stream>>>(dst + o, b, n);
    ctx->launches++;
  }
  HC_CUDA(cudaGetLastError());
}

void check_launch(hc_ctx* ctx) {
  (void)ctx;
  HC_CUDA(cudaGetLastError());
}

#define LAUNCH_DONE(ctx) \
  do {                   \
    (ctx)->launches++;   \
    check_launch(ctx);   \
  } while (0)

void launch_sample_ternary(hc_ctx* ctx, u64 seed, u64 tag, u64* dst, const int* ids, int nl) {
    {
      ProfScope prof_(ctx, "k_ternary");
      k_ternary<<<grid_for(ctx, 1, 1), kT, 0, ctx->stream>>>(seed, tag, dst, ids, nl, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_sample_gauss(hc_ctx* ctx, u64 seed, u64 tag, u64* dst, const int* ids, int nl) {
  Cdt cdt{};
  HC_CHECK(ctx->P.cdt.size() <= 40, HC_ERR_INVALID, "sigma too large");
  cdt.n = (int)ctx->P.cdt.size();
  for (int i = 0; i < cdt.n; ++i) cdt.t[i] = ctx->P.cdt[i];
    {
      ProfScope prof_(ctx, "k_gauss");
      k_gauss<<<grid_for(ctx, 1, 1), kT, 0, ctx->stream>>>(seed, tag, dst, ids, nl, ctx->tab, cdt);
    }
  LAUNCH_DONE(ctx);
}

void launch_sample_uniform(hc_ctx* ctx, u64 seed, u64 tag, u64* dst, const int* ids, int nl) {
    {
      ProfScope prof_(ctx, "k_uniform");
      k_uniform<<<grid_for(ctx, nl, 1), kT, 0, ctx->stream>>>(seed, tag, dst, ids, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_reduce_signed(hc_ctx* ctx, const int64_t* src, u64* dst, const int* ids, int nl) {
    {
      ProfScope prof_(ctx, "k_reduce_signed");
      k_reduce_signed<<<grid_for(ctx, nl, 1), kT, 0, ctx->stream>>>((const long long*)src, dst, ids, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_ew(hc_ctx* ctx, int op, const CtRef* out, const CtRef* a, const CtRef* b, int items,
               int npoly, int nl) {
  if (items <= 0) return;
    {
      ProfScope prof_(ctx, "k_ew", (uint64_t)items * npoly * nl);
      k_ew<<<grid_for(ctx, npoly * nl, items), kT, 0, ctx->stream>>>(op, out, a, b, nl, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_scalar(hc_ctx* ctx, bool add, const CtRef* out, const CtRef* a, int items, int npoly,
                   int nl, const u64* scal_dev) {
  if (items <= 0) return;
    {
      ProfScope prof_(ctx, "k_scalar", (uint64_t)items * npoly * nl);
      k_scalar<<<grid_for(ctx, npoly * nl, items), kT, 0, ctx->stream>>>(add, out, a, nl, scal_dev, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_tensor_pair(hc_ctx* ctx, const CtRef* out, const CtRef* a, const CtRef* b, int items, int nl) {
  if (items <= 0) return;
  HC_CHECK(items <= 65535, HC_ERR_INVALID, "too many outputs in one launch");
  {
    ProfScope prof_(ctx, "k_tensor_pair", (uint64_t)items * nl);
    k_tensor_pair<<<grid_for(ctx, nl, items), kT, 0, ctx->stream>>>(out, a, b, ctx->tab);
  }
  ctx->launches++;
  check_launch(ctx);
}

namespace {
// The fold interval of the lazy 128-bit sums: the Karatsuba sum gains
// (x0 + x1)(w0 + w1) < 4 qmax^2 per term (on top of a folded residue below
// 3 qmax), so fold before 2^128.
int tensor_fold_chunk(hc_ctx* ctx, int nl) {
  u64 qmax = 0;
  for (int i = 0; i < nl; ++i) qmax = ctx->P.chain[i] > qmax ? ctx->P.chain[i] : qmax;
  unsigned __int128 sq = (unsigned __int128)qmax * qmax;
  unsigned __int128 lim = (~(unsigned __int128)0) - ((unsigned __int128)1 << 64);
  unsigned __int128 per = lim / (4 * sq);
  int chunk = per > 1024 ? 1024 : (int)per - 1;
  HC_CHECK(chunk >= 1, HC_ERR_INVALID, "primes too large for lazy accumulation");
  return chunk;
}
}  // namespace

void launch_tensor_acc_grouped(hc_ctx* ctx, int G, const CtRef* out, const CtRef* x, const CtRef* w, const int* xi,
                               const int* wi, const int* off, int ngroups, int nl, uint64_t terms) {
  if (ngroups <= 0) return;
  HC_CHECK(G >= 1 && G <= 5, HC_ERR_INVALID, "tensor group size must be 1..5");
  HC_CHECK(ngroups <= 65535, HC_ERR_INVALID, "too many output groups in one launch");
  HC_CHECK(ctx->P.n % kT == 0, HC_ERR_INVALID, "ring degree below the block size");
  const int chunk = tensor_fold_chunk(ctx, nl);
  const dim3 grid((unsigned)(ctx->P.n / kT), (unsigned)ngroups, (unsigned)nl);
  {
    ProfScope prof_(ctx, "k_tensor_acc", terms * nl);  // units: (term, limb) pairs
    switch (G) {
      case 1: k_tensor_acc_g<1><<<grid, kT, 0, ctx->stream>>>(out, x, w, xi, wi, off, chunk, ctx->tab); break;
      case 2: k_tensor_acc_g<2><<<grid, kT, 0, ctx->stream>>>(out, x, w, xi, wi, off, chunk, ctx->tab); break;
      case 3: k_tensor_acc_g<3><<<grid, kT, 0, ctx->stream>>>(out, x, w, xi, wi, off, chunk, ctx->tab); break;
      case 4: k_tensor_acc_g<4><<<grid, kT, 0, ctx->stream>>>(out, x, w, xi, wi, off, chunk, ctx->tab); break;
      default: k_tensor_acc_g<5><<<grid, kT, 0, ctx->stream>>>(out, x, w, xi, wi, off, chunk, ctx->tab); break;
    }
  }
  LAUNCH_DONE(ctx);
}

void launch_tensor_acc(hc_ctx* ctx, const CtRef* out, const CtRef* x, const CtRef* w, const int* xi,
                       const int* wi, const int* off, int nout, int nl, uint64_t terms) {
  if (nout <= 0) return;
  const int chunk = tensor_fold_chunk(ctx, nl);
  HC_CHECK(nout <= 65535, HC_ERR_INVALID, "too many outputs in one launch");
    {
      ProfScope prof_(ctx, "k_tensor_acc", terms * nl);  // units: (term, limb) pairs
      k_tensor_acc<<<grid_for(ctx, nout, nl), kT, 0, ctx->stream>>>(out, x, w, xi, wi, off, nl, chunk, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_automorph(hc_ctx* ctx, const CtRef* out, const CtRef* a, int items, int npoly, int nl, u64 g) {
  if (items <= 0) return;
    {
      ProfScope prof_(ctx, "k_automorph", (uint64_t)items * npoly * nl);
      k_automorph<<<grid_for(ctx, npoly * nl, items), kT, 0, ctx->stream>>>(out, a, nl, g, nullptr, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_automorph_items(hc_ctx* ctx, const CtRef* out, const CtRef* a, int items, int npoly, int nl,
                            const u64* gs) {
  if (items <= 0) return;
  HC_CHECK(items <= 65535, HC_ERR_INVALID, "too many automorphism items for one launch");
  {
    ProfScope prof_(ctx, "k_automorph", (uint64_t)items * npoly * nl);
    k_automorph<<<grid_for(ctx, npoly * nl, items), kT, 0, ctx->stream>>>(out, a, nl, 1, gs, ctx->tab);
  }
  LAUNCH_DONE(ctx);
}

void launch_modup_bconv(hc_ctx* ctx, int level, int j, const u64* xcoef, u64 x_item_stride, u64* ext,
                        u64 ext_item_stride, int items) {
  const int alpha = ctx->P.alpha;
  const int d0 = j * alpha;
  const int ns = std::min(alpha, level + 1 - d0);
  const int next = level + 1 + alpha;
  HC_CHECK(ns >= 1 && ns <= 16, HC_ERR_INVALID, "bad digit");
    {
      ProfScope prof_(ctx, "k_modup_bconv", (uint64_t)items * (next - ns));
      k_modup_bconv<<<grid_for(ctx, 1, items), kT, 0, ctx->stream>>>(
        xcoef, x_item_stride, ext, ext_item_stride, ctx->ks(ctx->lv[level].modup_off[j]), d0, ns, next,
        ctx->ext_map_of(level), ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_key_product(hc_ctx* ctx, int level, const u64* ext, u64 ext_item_stride, const u64* key,
                        u64* acc, u64 acc_item_stride, int items) {
  const int next = level + 1 + ctx->P.alpha;
    {
      ProfScope prof_(ctx, "k_key_product", (uint64_t)items * next);
      k_key_product<<<grid_for(ctx, next, items), kT, 0, ctx->stream>>>(
        ext, ext_item_stride, key, acc, acc_item_stride, ctx->lv[level].dnum, next, ctx->P.nchain(),
        ctx->ext_map_of(level), nullptr, nullptr, items, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_moddown_bconv(hc_ctx* ctx, int level, const u64* accp_coef, u64 accp_item_stride,
                          u64* z, u64 z_item_stride, int items) {
  const int next = level + 1 + ctx->P.alpha;
    {
      ProfScope prof_(ctx, "k_moddown_bconv", (uint64_t)items * 2 * (level + 1));
      k_moddown_bconv<<<grid_for(ctx, 2, items), kT, 0, ctx->stream>>>(
        accp_coef, accp_item_stride, (u64)next * ctx->P.n, z, z_item_stride, ctx->ks(ctx->moddown_off),
        ctx->P.alpha, level + 1, ctx->P.L, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_moddown_combine(hc_ctx* ctx, int level, const u64* acc, u64 acc_item_stride, const u64* z,
                            u64 z_item_stride, const CtRef* base0, const CtRef* base1, const CtRef* out,
                            int items, const u64* base0_gs) {
  const int nq = level + 1, next = level + 1 + ctx->P.alpha;
    {
      ProfScope prof_(ctx, "k_moddown_combine", (uint64_t)items * 2 * nq);
      if (base0_gs)
        k_moddown_combine<true><<<grid_for(ctx, 2 * nq, items), kT, 0, ctx->stream>>>(
          acc, acc_item_stride, (u64)next * ctx->P.n, z, z_item_stride, base0, base1, out, nq, base0_gs, ctx->tab);
      else
        k_moddown_combine<false><<<grid_for(ctx, 2 * nq, items), kT, 0, ctx->stream>>>(
          acc, acc_item_stride, (u64)next * ctx->P.n, z, z_item_stride, base0, base1, out, nq, nullptr, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_rescale_lift(hc_ctx* ctx, int level, const u64* last, u64* lift, int items, int npoly) {
    {
      ProfScope prof_(ctx, "k_rescale_lift", (uint64_t)items * npoly * level);
      k_rescale_lift<<<grid_for(ctx, npoly * level, items), kT, 0, ctx->stream>>>(last, lift, level, npoly, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_rescale_combine(hc_ctx* ctx, int level, const CtRef* in, const u64* lift, const CtRef* out,
                            int items, int npoly) {
    {
      ProfScope prof_(ctx, "k_rescale_combine", (uint64_t)items * npoly * level);
      k_rescale_combine<<<grid_for(ctx, npoly * level, items), kT, 0, ctx->stream>>>(
        in, lift, out, ctx->ks(ctx->lv[level].rescale_off), level, npoly, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_gather_limb(hc_ctx* ctx, const CtRef* src, int slot, u64* dst, int items, int npoly) {
    {
      ProfScope prof_(ctx, "k_gather_limb", (uint64_t)items * npoly);
      k_gather_limb<<<grid_for(ctx, npoly, items), kT, 0, ctx->stream>>>(src, slot, dst, npoly, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_check_range(hc_ctx* ctx, const u64* data, int npoly, int nl, u64 poly_stride,
                        unsigned long long* bad) {
    {
      ProfScope prof_(ctx, "k_check_range");
      k_check_range<<<grid_for(ctx, npoly * nl, 1), kT, 0, ctx->stream>>>(data, nl, poly_stride, bad, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

void launch_sum4(hc_ctx* ctx, const CtRef* out, const CtRef* x, const int* idx, int nout, int nl) {
  if (nout <= 0) return;
    {
      ProfScope prof_(ctx, "k_sum4", (uint64_t)nout * 2 * nl);
      k_sum4<<<grid_for(ctx, 2 * nl, nout), kT, 0, ctx->stream>>>(out, x, idx, nl, ctx->tab);
    }
  LAUNCH_DONE(ctx);
}

// ===========================================================================
// Specialised key-switching kernels (digit size / digit count known at
// compile time, constants staged in shared memory, key limbs reused across
// the batch) and the fused relinearise + rescale tail.
// ===========================================================================
namespace {

// ModUp: v_i = [x_i hat_inv_i]_{q_i}; y_t = sum_i v_i hat_mod[t][i] mod q_t
// for every ext slot t outside the digit [d0, d0 + NS).
template <int NS>
__global__ void __launch_bounds__(kT) k_modup_bconv_t(const u64* xcoef, u64 x_item_stride, u64* ext,
                                                       u64 ext_item_stride, const u64* cst, int d0, int next,
                                                       const int* emap, DigitGrid dg, Tables T) {
  // digit d0 / alpha + blockIdx.y / split of a run of full digits
  const int dj = blockIdx.y / dg.split;
  d0 += dj * dg.alpha;
  cst += dj * dg.cst_digit_stride;
  ext += dj * dg.ext_digit_stride;
  extern __shared__ u64 sh[];
  u64* hm = sh;                          // [next][NS]
  DMod* md = (DMod*)(sh + next * NS);    // [next]
  for (int e = threadIdx.x; e < next * NS; e += blockDim.x) hm[e] = cst[2 * NS + e];
  for (int t = threadIdx.x; t < next; t += blockDim.x) md[t] = T.mods[emap[t]];
  __syncthreads();
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int z = blockIdx.z;
  const u64* x = xcoef + (size_t)z * x_item_stride;
  u64* y = ext + (size_t)z * ext_item_stride;
  u64 v[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) v[i] = shoup(x[(size_t)(d0 + i) * n + c], cst[i], cst[NS + i], md[d0 + i].q);
  for (int t = 0; t < next; ++t) {
    if (t >= d0 && t < d0 + NS) continue;
    U128 acc{0, 0};
#pragma unroll
    for (int i = 0; i < NS; ++i) mac(acc, v[i], hm[t * NS + i]);
    y[(size_t)t * n + c] = reduce128(acc, md[t]);
  }
}

// Exact sum of up to 8 products v_i h_i with v_i, h_i < 2^60, each operand
// split into 30-bit halves (v = vh 2^30 + vl, vs = vl + vh < 2^31).  Three
// 32 x 32 -> 64-bit multiply-adds per term (Karatsuba): lo = sum vl hl,
// hi = sum vh hh and sm = sum vs hs, each accumulated in 64 bits without
// carry handling.  lo and hi stay below 2^63; sm may wrap, but the cross
// sum sm - lo - hi = sum (vl hh + vh hl) is below 16 (2^30 - 1)^2 < 2^64,
// so it comes out exact modulo 2^64.  The 128-bit value is assembled once.
struct Acc30 {
  u64 lo, hi, sm;
};
struct Half30 {
  uint32_t l, h, s;
};
constexpr uint32_t kMask30 = (1u << 30) - 1;
__device__ __forceinline__ Half30 halves30(u64 v) {
  const uint32_t l = (uint32_t)v & kMask30, h = (uint32_t)(v >> 30);
  return Half30{l, h, l + h};
}
__device__ __forceinline__ uint4 halves30_packed(u64 v) {
  const Half30 x = halves30(v);
  return make_uint4(x.l, x.h, x.s, 0u);
}
__device__ __forceinline__ void mac30(Acc30& a, const Half30& v, uint4 h) {
  a.lo += (u64)v.l * h.x;
  a.hi += (u64)v.h * h.y;
  a.sm += (u64)v.s * h.z;
}
__device__ __forceinline__ void mac30(Acc30& a, const Half30& v, const Half30& h) {
  a.lo += (u64)v.l * h.l;
  a.hi += (u64)v.h * h.h;
  a.sm += (u64)v.s * h.s;
}
// lo + mid 2^30 + hi 2^60 as a 128-bit value, mid = sm - lo - hi.
__device__ __forceinline__ U128 acc30_value(const Acc30& a) {
  const u64 mid = a.sm - a.lo - a.hi;
  const u64 x = a.lo + (mid << 30);
  const u64 c1 = x < a.lo;
  const u64 y = x + (a.hi << 60);
  const u64 c2 = y < x;
  return U128{y, (mid >> 34) + (a.hi >> 4) + c1 + c2};
}

// ModUp conversion as k_modup_bconv_t with every prime below 2^60: the
// constants sit in shared memory as 30-bit halves.
template <int NS>
__global__ void __launch_bounds__(kT) k_modup_bconv_h(const u64* xcoef, u64 x_item_stride, u64* ext,
                                                       u64 ext_item_stride, const u64* cst, int d0, int next,
                                                       const int* emap, DigitGrid dg, Tables T) {
  // digit d0 / alpha + blockIdx.y / split of a run of full digits; part
  // blockIdx.y % split of its output primes
  const int dj = blockIdx.y / dg.split, part = blockIdx.y - dj * dg.split;
  d0 += dj * dg.alpha;
  cst += dj * dg.cst_digit_stride;
  ext += dj * dg.ext_digit_stride;
  extern __shared__ u64 sh[];
  uint4* hm = reinterpret_cast<uint4*>(sh);  // [next][NS] halves, Montgomery form
  DMod* md = (DMod*)(sh + 2 * next * NS);    // [next]
  for (int t = threadIdx.x; t < next; t += blockDim.x) md[t] = T.mods[emap[t]];
  __syncthreads();
  for (int e = threadIdx.x; e < next * NS; e += blockDim.x) {
    const DMod& mt = md[e / NS];
    hm[e] = halves30_packed(shoup(cst[2 * NS + e], mt.r64, mt.r64_sh, mt.q));  // h 2^64 mod q_t
  }
  __syncthreads();
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int z = blockIdx.z;
  const u64* x = xcoef + (size_t)z * x_item_stride;
  u64* y = ext + (size_t)z * ext_item_stride;
  Half30 v[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) v[i] = halves30(shoup(x[(size_t)(d0 + i) * n + c], cst[i], cst[NS + i], md[d0 + i].q));
  // the output primes may be split over dg.split blocks (a tuning choice)
  const int per = (next + dg.split - 1) / dg.split, t_end = min(next, (part + 1) * per);
  for (int t = part * per; t < t_end; ++t) {
    if (t >= d0 && t < d0 + NS) continue;
    Acc30 acc{0, 0, 0};
#pragma unroll
    for (int i = 0; i < NS; ++i) mac30(acc, v[i], hm[t * NS + i]);
    y[(size_t)t * n + c] = redc(acc30_value(acc), md[t]);  // sum < 8 2^60 q_t: high word < q_t
  }
}

// ModDown conversion as k_moddown_bconv_t with every prime below 2^60.
template <int ALPHA>
__global__ void __launch_bounds__(kT) k_moddown_bconv_h(const u64* src, u64 src_item_stride, u64 src_poly_stride,
                                                         u64* zq, u64 z_item_stride, const u64* cst, int nq, int L,
                                                         Tables T) {
  extern __shared__ u64 sh[];
  uint4* hm = reinterpret_cast<uint4*>(sh);  // [nq][ALPHA] halves, Montgomery form
  DMod* md = (DMod*)(sh + 2 * nq * ALPHA);   // [nq]
  for (int t = threadIdx.x; t < nq; t += blockDim.x) md[t] = T.mods[t];
  __syncthreads();
  for (int e = threadIdx.x; e < nq * ALPHA; e += blockDim.x) {
    const DMod& mt = md[e / ALPHA];
    hm[e] = halves30_packed(shoup(cst[2 * ALPHA + e], mt.r64, mt.r64_sh, mt.q));
  }
  __syncthreads();
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y, z = blockIdx.z;
  const u64* x = src + (size_t)z * src_item_stride + (size_t)k * src_poly_stride;
  Half30 v[ALPHA];
#pragma unroll
  for (int i = 0; i < ALPHA; ++i) v[i] = halves30(shoup(x[(size_t)i * n + c], cst[i], cst[ALPHA + i], T.mods[L + 1 + i].q));
  u64* out = zq + (size_t)z * z_item_stride + (size_t)k * nq * n;
  for (int t = 0; t < nq; ++t) {
    Acc30 acc{0, 0, 0};
#pragma unroll
    for (int i = 0; i < ALPHA; ++i) mac30(acc, v[i], hm[t * ALPHA + i]);
    out[(size_t)t * n + c] = redc(acc30_value(acc), md[t]);
  }
}

// ModDown conversion P -> Q_level of both polys (ALPHA special primes), times
// P^{-1} (folded into the constants, as in k_moddown_bconv).
template <int ALPHA>
__global__ void __launch_bounds__(kT) k_moddown_bconv_t(const u64* src, u64 src_item_stride, u64 src_poly_stride,
                                                         u64* zq, u64 z_item_stride, const u64* cst, int nq, int L,
                                                         Tables T) {
  extern __shared__ u64 sh[];
  u64* hm = sh;                          // [nq][ALPHA]
  DMod* md = (DMod*)(sh + nq * ALPHA);   // [nq]
  for (int e = threadIdx.x; e < nq * ALPHA; e += blockDim.x) hm[e] = cst[2 * ALPHA + e];
  for (int t = threadIdx.x; t < nq; t += blockDim.x) md[t] = T.mods[t];
  __syncthreads();
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y, z = blockIdx.z;
  const u64* x = src + (size_t)z * src_item_stride + (size_t)k * src_poly_stride;
  u64 v[ALPHA];
#pragma unroll
  for (int i = 0; i < ALPHA; ++i) v[i] = shoup(x[(size_t)i * n + c], cst[i], cst[ALPHA + i], T.mods[L + 1 + i].q);
  u64* out = zq + (size_t)z * z_item_stride + (size_t)k * nq * n;
  for (int t = 0; t < nq; ++t) {
    U128 acc{0, 0};
#pragma unroll
    for (int i = 0; i < ALPHA; ++i) mac(acc, v[i], hm[t * ALPHA + i]);
    out[(size_t)t * n + c] = reduce128(acc, md[t]);
  }
}

// acc[z][k][s] = sum_j ext[z][j][s] * key[j][k][emap[s]] for all items z:
// the 2 DNUM key words of (s, c) stay in registers across the batch.
// digit_src (optional): the digit's own slots s in [j alpha, j alpha + alpha)
// come from digit_src[z] (NTT-form input) instead of ext.
template <int DNUM, bool HALVES, bool GATHER>
__global__ void __launch_bounds__(kT) k_key_product_t(const u64* ext, u64 ext_item_stride, const u64* key, u64* acc,
                                                       u64 acc_item_stride, int next, int nchain, const int* emap,
                                                       int items, const CtRef* digit_src, int alpha, int nq,
                                                       const u64* const* item_keys, const u64* gs, int ext_items,
                                                       Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int s = blockIdx.y;
  const int pid = emap[s];
  const DMod md = T.mods[pid];
  u64 kb[DNUM], ka[DNUM];
  Half30 hb[DNUM], ha[DNUM];  // (used by the halves form only)
  // the key limbs of this slot: once for all items, or per item when every
  // item carries its own switching key
  auto load_keys = [&](const u64* kbase) {
#pragma unroll
    for (int j = 0; j < DNUM; ++j) {
      kb[j] = kbase[((size_t)(2 * j) * nchain + pid) * n + c];
      ka[j] = kbase[((size_t)(2 * j + 1) * nchain + pid) * n + c];
      if constexpr (HALVES) {
        hb[j] = halves30(kb[j]);
        ha[j] = halves30(ka[j]);
      }
    }
  };
  if (!item_keys) load_keys(key);
  const int own = (digit_src && s < nq) ? s / alpha : -1;  // the digit whose block holds slot s
  for (int z = blockIdx.z; z < items; z += gridDim.z) {
    if (item_keys) load_keys(item_keys[z]);
    // GATHER: item z reads the raised digits of item z mod ext_items,
    // through kappa_g when gs is given; otherwise its own, in place
    const u64* e = ext + (size_t)s * n;
    if constexpr (GATHER) {
      const int ce = gs ? automorph_src(c, gs[z], T.log_n) : c;
      e += (size_t)(z < ext_items ? z : z % ext_items) * ext_item_stride + ce;
    } else {
      e += (size_t)z * ext_item_stride + c;
    }
    u64* o = acc + (size_t)z * acc_item_stride + (size_t)s * n + c;
    if constexpr (HALVES) {
      // every operand below 2^60: 30-bit halves, carry-free partial sums
      Acc30 a0{0, 0, 0}, a1{0, 0, 0};
#pragma unroll
      for (int j = 0; j < DNUM; ++j) {
        const Half30 y = halves30((j == own) ? digit_src[z].p[(size_t)s * n + c] : e[(size_t)j * next * n]);
        mac30(a0, y, hb[j]);
        mac30(a1, y, ha[j]);
      }
      o[0] = redc(acc30_value(a0), md);  // keys in Montgomery form; sum < 8 q^2
      o[(size_t)next * n] = redc(acc30_value(a1), md);
    } else {
      U128 a0{0, 0}, a1{0, 0};
#pragma unroll
      for (int j = 0; j < DNUM; ++j) {
        const u64 y = (j == own) ? digit_src[z].p[(size_t)s * n + c] : e[(size_t)j * next * n];
        mac(a0, y, kb[j]);
        mac(a1, y, ka[j]);
      }
      o[0] = redc(a0, md);
      o[(size_t)next * n] = redc(a1, md);
    }
  }
}

// Fused relinearise + rescale, step 1: t_k = base_k[l] + acc_k[l] (NTT
// form, last limb only; the key product's Q limbs carry P^{-1} already).
__global__ void k_ksr_last(const u64* acc, u64 acc_item_stride, u64 acc_poly_stride, const CtRef* base0,
                           const CtRef* base1, u64* tl, int level, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y, z = blockIdx.z;
  const u64 q = T.mods[level].q;
  const size_t li = (size_t)level * n + c;
  u64 r = acc[(size_t)z * acc_item_stride + (size_t)k * acc_poly_stride + li];
  const CtRef* base = k == 0 ? base0 : base1;
  if (base) r = addm(r, base[z].p[li], q);
  tl[((size_t)z * 2 + k) * n + c] = r;
}

// Step 2 of the fused form: the centred c_l = t_k - z_k[l] mod q_l (z
// carries P^{-1}) stored over t_k as a signed integer (the transform of the
// other limbs lifts it).
__global__ void k_ksr_cl(u64* tl, const u64* zq, u64 z_item_stride, int level, Tables T) {
  const int n = 1 << T.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int k = blockIdx.y, z = blockIdx.z;
  const u64 ql = T.mods[level].q;
  const u64* zk = zq + (size_t)z * z_item_stride + (size_t)k * (level + 1) * n;
  u64* t = tl + ((size_t)z * 2 + k) * n + c;
  const u64 cl = subm(*t, zk[(size_t)level * n + c], ql);
  const bool neg = cl > (ql - 1) / 2;
  *t = neg ? (u64)(-(long long)(ql - cl)) : cl;
}


}  // namespace

void launch_modup_bconv_fast(hc_ctx* ctx, int level, int j, const u64* xcoef, u64 x_item_stride, u64* ext,
                             u64 ext_item_stride, int items, int ndig) {
  const int alpha = ctx->P.alpha;
  const int d0 = j * alpha;
  const int ns = std::min(alpha, level + 1 - d0);
  const int next = level + 1 + alpha;
  HC_CHECK(ndig >= 1 && (ndig == 1 || (j + ndig) * alpha <= level + 1), HC_ERR_INVALID,
           "a multi-digit conversion covers full digits only");
  HC_CHECK(ndig == 1 || ns <= 8, HC_ERR_INVALID, "multi-digit conversions need a specialised kernel");
  const u64* cst = ctx->ks(ctx->lv[level].modup_off[j]);
  // (the halves form stages 16 bytes per constant, the other 8)
  const size_t smem = (size_t)next * ns * 2 * sizeof(u64) + (size_t)next * sizeof(DMod);
  const bool halves_split = ctx->P.below_2_60 && ns <= 8;
  DigitGrid dg;
  dg.split = halves_split ? std::max(1, std::min(ctx->tune.modup_split, next)) : 1;
  dg.alpha = alpha;
  dg.ext_digit_stride = (u64)next * ctx->P.n;        // digit j's raised limbs follow digit j - 1's
  dg.cst_digit_stride = (u64)(2 + next) * alpha;     // a full digit's constants: hat_inv, its Shoup, hat_mod
  const dim3 g = grid_for(ctx, dg.split * ndig, items);
  ProfScope prof_(ctx, "k_modup_bconv", (uint64_t)items * ndig * (next - ns));
  const bool halves = ctx->P.below_2_60;
#define HC_MODUP(NS)                                                                                          \
  case NS:                                                                                                    \
    if (halves)                                                                                               \
      k_modup_bconv_h<NS><<<g, kT, smem, ctx->stream>>>(xcoef, x_item_stride, ext, ext_item_stride, cst, d0, \
                                                         next, ctx->ext_map_of(level), dg, ctx->tab);         \
    else                                                                                                      \
      k_modup_bconv_t<NS><<<g, kT, smem, ctx->stream>>>(xcoef, x_item_stride, ext, ext_item_stride, cst, d0, \
                                                         next, ctx->ext_map_of(level), dg, ctx->tab);         \
    break;
  switch (ns) {
    HC_MODUP(1) HC_MODUP(2) HC_MODUP(3) HC_MODUP(4) HC_MODUP(5) HC_MODUP(6) HC_MODUP(7) HC_MODUP(8)
    default:
      k_modup_bconv<<<g, kT, 0, ctx->stream>>>(xcoef, x_item_stride, ext, ext_item_stride, cst, d0, ns, next,
                                              ctx->ext_map_of(level), ctx->tab);
  }
#undef HC_MODUP
  ctx->launches++;
  check_launch(ctx);
}

void launch_moddown_bconv_fast(hc_ctx* ctx, int level, const u64* accp_coef, u64 accp_item_stride, u64* z,
                               u64 z_item_stride, int items) {
  const int alpha = ctx->P.alpha, nq = level + 1, next = nq + alpha;
  const u64* cst = ctx->ks(ctx->moddown_off);
  const size_t smem = (size_t)nq * alpha * 2 * sizeof(u64) + (size_t)nq * sizeof(DMod);
  const dim3 g = grid_for(ctx, 2, items);
  const u64 ps = (u64)next * ctx->P.n;
  ProfScope prof_(ctx, "k_moddown_bconv", (uint64_t)items * 2 * nq);
  const bool halves = ctx->P.below_2_60;
#define HC_MODDOWN(A)                                                                                          \
  case A:                                                                                                      \
    if (halves)                                                                                                \
      k_moddown_bconv_h<A><<<g, kT, smem, ctx->stream>>>(accp_coef, accp_item_stride, ps, z, z_item_stride,   \
                                                          cst, nq, ctx->P.L, ctx->tab);                        \
    else                                                                                                       \
      k_moddown_bconv_t<A><<<g, kT, smem, ctx->stream>>>(accp_coef, accp_item_stride, ps, z, z_item_stride,   \
                                                          cst, nq, ctx->P.L, ctx->tab);                        \
    break;
  switch (alpha) {
    HC_MODDOWN(1) HC_MODDOWN(2) HC_MODDOWN(3) HC_MODDOWN(4) HC_MODDOWN(5) HC_MODDOWN(6) HC_MODDOWN(7) HC_MODDOWN(8)
    default:
      k_moddown_bconv<<<g, kT, 0, ctx->stream>>>(accp_coef, accp_item_stride, ps, z, z_item_stride, cst, alpha, nq,
                                                ctx->P.L, ctx->tab);
  }
#undef HC_MODDOWN
  ctx->launches++;
  check_launch(ctx);
}

// The four forms of k_key_product_t<D>: 30-bit halves or 64-bit products,
// with or without the gathered (shared, automorphed) digit reads.
template <int D>
void key_product_t_launch(bool halves, bool gather, dim3 g, cudaStream_t st, const u64* ext, u64 ext_is,
                          const u64* key, u64* acc, u64 acc_is, int next, int nchain, const int* emap, int items,
                          const CtRef* digit_src, int alpha, int nq, const u64* const* item_keys, const u64* gs,
                          int ext_items, const Tables& T) {
  if (halves && gather)
    k_key_product_t<D, true, true><<<g, kT, 0, st>>>(ext, ext_is, key, acc, acc_is, next, nchain, emap, items,
                                                     digit_src, alpha, nq, item_keys, gs, ext_items, T);
  else if (halves)
    k_key_product_t<D, true, false><<<g, kT, 0, st>>>(ext, ext_is, key, acc, acc_is, next, nchain, emap, items,
                                                      digit_src, alpha, nq, item_keys, gs, ext_items, T);
  else if (gather)
    k_key_product_t<D, false, true><<<g, kT, 0, st>>>(ext, ext_is, key, acc, acc_is, next, nchain, emap, items,
                                                      digit_src, alpha, nq, item_keys, gs, ext_items, T);
  else
    k_key_product_t<D, false, false><<<g, kT, 0, st>>>(ext, ext_is, key, acc, acc_is, next, nchain, emap, items,
                                                       digit_src, alpha, nq, item_keys, gs, ext_items, T);
}

void launch_key_product_batched(hc_ctx* ctx, int level, const u64* ext, u64 ext_item_stride, const u64* key,
                                u64* acc, u64 acc_item_stride, int items, const CtRef* digit_src,
                                const u64* const* item_keys, const u64* gs, int ext_items) {
  if (ext_items <= 0) ext_items = items;
  HC_CHECK(!(gs && digit_src), HC_ERR_INVALID, "digit sources are not read through an automorphism");
  const bool gather = gs || ext_items != items;
  const int next = level + 1 + ctx->P.alpha, dnum = ctx->lv[level].dnum;
  // a few item groups in z so small batches still fill the GPU
  const int zgroups =
      std::min(items, std::max(1, 2048 / (next * ((ctx->P.n + kT - 1) / kT))) * std::max(1, ctx->tune.kp_zmul));
  const dim3 g = grid_for(ctx, next, zgroups);
  ProfScope prof_(ctx, "k_key_product", (uint64_t)items * next);
  const bool halves = ctx->P.below_2_60;
#define HC_KP(D)                                                                                                \
  case D:                                                                                                       \
    key_product_t_launch<D>(halves, gather, g, ctx->stream, ext, ext_item_stride, key, acc, acc_item_stride,    \
                            next, ctx->P.nchain(), ctx->ext_map_of(level), items, digit_src, ctx->P.alpha,      \
                            level + 1, item_keys, gs, ext_items, ctx->tab);                                     \
    break;
  switch (dnum) {
    HC_KP(1) HC_KP(2) HC_KP(3) HC_KP(4) HC_KP(5) HC_KP(6) HC_KP(7) HC_KP(8)
    default: {
      HC_CHECK(!digit_src, HC_ERR_INVALID, "digit sources need a specialised key product");
      const dim3 g2 = grid_for(ctx, next, items);
      k_key_product<<<g2, kT, 0, ctx->stream>>>(ext, ext_item_stride, key, acc, acc_item_stride, dnum, next,
                                                ctx->P.nchain(), ctx->ext_map_of(level), item_keys, gs, ext_items,
                                                ctx->tab);
    }
  }
#undef HC_KP
  ctx->launches++;
  check_launch(ctx);
}

void launch_ksr_last(hc_ctx* ctx, int level, const u64* acc, u64 acc_item_stride, const CtRef* base0,
                     const CtRef* base1, u64* tl, int items) {
  const int next = level + 1 + ctx->P.alpha;
  ProfScope prof_(ctx, "k_ksr_last", (uint64_t)items * 2);
  k_ksr_last<<<grid_for(ctx, 2, items), kT, 0, ctx->stream>>>(acc, acc_item_stride, (u64)next * ctx->P.n, base0, base1,
                                                             tl, level, ctx->tab);
  ctx->launches++;
  check_launch(ctx);
}

void launch_ksr_cl(hc_ctx* ctx, int level, u64* tl, const u64* zq, u64 z_item_stride, int items) {
  ProfScope prof_(ctx, "k_ksr_cl", (uint64_t)items * 2);
  k_ksr_cl<<<grid_for(ctx, 2, items), kT, 0, ctx->stream>>>(tl, zq, z_item_stride, level, ctx->tab);
  ctx->launches++;
  check_launch(ctx);
}

void ksr_constants(hc_ctx* ctx, int level, KsrFuse& f) {
  f.qlinv = ctx->ks(ctx->lv[level].rescale_off);
  f.nqlinv = f.qlinv + 2 * level;
  f.level = level;
  // |c_l| <= (q_l - 1) / 2 is already reduced modulo every q_i above that bound
  const u64 half = (ctx->P.chain[level] - 1) / 2;
  f.cl_small = 1;
  for (int i = 0; i < level; ++i) f.cl_small &= ctx->P.chain[i] > half ? 1 : 0;
}

