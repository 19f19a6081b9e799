// Device-side modular arithmetic and addressing shared by the kernels of
// libhecnn.  All residues are uint64 words for primes q < 2^61.
//
// Constant multiplications use Shoup's precomputed quotient (V. Shoup, NTL;
// D. Harvey, "Faster arithmetic for number-theoretic transforms", 2014):
// with w' = floor(w 2^64 / q), a w - floor(a w' / 2^64) q lies in [0, 2q)
// for every a < 2^64.  Products of two variable residues are accumulated
// exactly in 128 bits and reduced once, by splitting the 128-bit value as
// hi 2^64 + lo and reducing both halves with Shoup multiplications by the
// constants 2^64 mod q and 1.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef unsigned long long u64;
typedef unsigned int u32;

#define HC_MAX_CHAIN 64

// Per-prime constants.
struct DMod {
  u64 q;
  u64 r64;     // 2^64 mod q
  u64 r64_sh;  // floor(r64 * 2^64 / q)
  u64 one_sh;  // floor(2^64 / q)
  u64 qinv;    // q^{-1} mod 2^64
};

// Read-only tables of one context.
struct Tables {
  const ulonglong2* fwd2;  // [chain][N] (psi^{brv(k)}, Shoup companion)
  const ulonglong2* inv2;  // [chain][N] (psi^{-brv(k)}, Shoup companion)
  const u64* ninv;    // [chain] N^{-1} mod q
  const u64* ninv_sh;
  const DMod* mods;   // [chain]
  int log_n;
};

// A ciphertext (or any group of polynomials) in device memory: poly k, limb
// i at p + k*stride + i*N.
struct CtRef {
  u64* p;
  u64 stride;
};

// The fused tail of relinearise + rescale carried by the forward NTT of the
// converted limbs z_k[i] (i < level, poly k < 2, item z).  ModDown's P^{-1}
// is already in z (conversion constants) and in the key-product
// accumulators acc (the keys' Q limbs), so:
// - first pass, on load: x = z_k[i] + [c_l]_{q_i}, with c_l the centred last
//   limb of the relinearised poly stored as a signed integer in
//   cl[z][k][coefficient];
// - last pass, on store: out_k[i] = (base_k[i] + acc_k[i] - NTT(x)) q_l^{-1},
//   written to the output ciphertexts instead of back into z.
// The same tail in coefficient form is carried by the inverse NTT of
// y = base_k[i] + acc_k[i] (formed on load by the first pass); the last pass
// stores out_k[i] = INTT(y) q_l^{-1} - (z_k[i] + [c_l]_{q_i}) q_l^{-1} into
// the transform's own limbs, with N^{-1} folded into the first constant.
struct KsrFuse {
  const u64* cl;        // [item][2][N] signed centred c_l
  const u64* acc;       // key-product accumulators, NTT form
  u64 acc_item_stride, acc_poly_stride;
  const CtRef* base0;   // (d0, d1) or null
  const CtRef* base1;
  const CtRef* out;     // level-1 outputs
  const u64* qlinv;     // q_l^{-1} mod q_i, then its Shoup companions
  int level;
  int cl_small;         // every q_i (i < level) exceeds |c_l|: [c_l]_{q_i} needs no reduction
  // coefficient-form tail only
  const u64* z;         // z_k[i] at z + item*z_item_stride + k*z_poly_stride + i*N
  u64 z_item_stride, z_poly_stride;
  const u64* nqlinv;    // N^{-1} q_l^{-1} mod q_i, then its Shoup companions
};


// A set of limbs for batched per-limb kernels (NTT, copies): for batch item
// z, poly k < npoly and limb slot l0 <= s < l0 + nlimb the limb lives at
//   (refs ? refs[z].p + k*refs[z].stride : base + z*item_stride + k*poly_stride) + s*N
// and is taken modulo chain prime prime_map ? prime_map[s] : s.
// A ModUp conversion over a run of full digits in one launch: blockIdx.y /
// split picks the digit, blockIdx.y % split the part of its output primes.
struct DigitGrid {
  int split;
  int alpha;
  u64 ext_digit_stride;  // words between two digits' raised limbs
  u64 cst_digit_stride;  // words between two digits' constants
};

struct LimbSet {
  const CtRef* refs;
  u64* base;
  u64 item_stride;
  u64 poly_stride;
  int npoly;
  int nlimb;
  int l0;
  const int* prime_map;
  const int* slot_map;  // optional: limb l lives at slot slot_map[l] instead of l0 + l
  int slot_map_2d;      // with slot_map: poly k's limb l lives at slot_map[k * nlimb + l]
};

__device__ __forceinline__ u64* limb_ptr(const LimbSet& s, int z, int k, int slot, int n) {
  u64* b = s.refs ? s.refs[z].p + (u64)k * s.refs[z].stride
                  : s.base + (u64)z * s.item_stride + (u64)k * s.poly_stride;
  return b + (u64)slot * n;
}

__device__ __forceinline__ int limb_prime(const LimbSet& s, int slot) {
  return s.prime_map ? s.prime_map[slot] : slot;
}

// ------------------------------------------------------------ arithmetic
#ifdef __CUDACC__
__device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }
__device__ __forceinline__ u64 addm(u64 a, u64 b, u64 q) { return csub(a + b, q); }
__device__ __forceinline__ u64 subm(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
__device__ __forceinline__ u64 negm(u64 a, u64 q) { return a ? q - a : 0; }

// a * w mod q in [0, 2q), w < q, wsh = floor(w 2^64 / q).
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wsh, u64 q) {
  return a * w - __umul64hi(a, wsh) * q;
}
__device__ __forceinline__ u64 shoup(u64 a, u64 w, u64 wsh, u64 q) {
  return csub(shoup_lazy(a, w, wsh, q), q);
}

// Estimate of floor(y wsh / 2^64) from three of the four 32 x 32-bit partial
// products: the low x low product and the carries out of the low words are
// dropped, so the estimate is the exact quotient minus 0, 1 or 2.  Integer
// multiplies are the scarce resource on this GPU (wide and high-half forms
// take two issue slots of the one pipe that runs them); this saves about a
// third of a full 64-bit high product (whether that wins depends on the
// kernel's mix of integer and ALU work).
__device__ __forceinline__ u64 mulhi_est(u64 y, u64 wsh) {
  const uint32_t y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
  const uint32_t w0 = (uint32_t)wsh, w1 = (uint32_t)(wsh >> 32);
  return (u64)y1 * w1 + __umulhi(y1, w0) + __umulhi(y0, w1);
}
// a * w mod q in [0, 4q) for any 64-bit a (w < q, wsh as above): Shoup's
// product with the estimated quotient; needs q < 2^62.
__device__ __forceinline__ u64 shoup_lazy4(u64 a, u64 w, u64 wsh, u64 q) {
  return a * w - mulhi_est(a, wsh) * q;
}

struct U128 {
  u64 lo, hi;
};
// acc += a * b exactly (carry through the PTX carry flag).
__device__ __forceinline__ void mac(U128& acc, u64 a, u64 b) {
  asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;"
      : "+l"(acc.lo), "+l"(acc.hi)
      : "l"(a), "l"(b));
}
// Fully reduced value of hi 2^64 + lo.
__device__ __forceinline__ u64 reduce128(U128 x, const DMod& m) {
  u64 t = shoup_lazy(x.hi, m.r64, m.r64_sh, m.q);     // hi 2^64 mod q, [0, 2q)
  u64 r = x.lo - __umul64hi(x.lo, m.one_sh) * m.q;     // lo mod q,      [0, 2q)
  u64 s = t + r;                                       // [0, 4q)
  s = csub(s, 2 * m.q);
  return csub(s, m.q);
}
// The same value with estimated quotients (q < 2^61, so 8q < 2^64): fewer
// integer multiplies and one more conditional subtraction.  Which form is
// faster depends on the kernel's instruction mix; measured per kernel.
__device__ __forceinline__ u64 reduce128_est(U128 x, const DMod& m) {
  u64 t = shoup_lazy4(x.hi, m.r64, m.r64_sh, m.q);     // [0, 4q)
  u64 r = x.lo - mulhi_est(x.lo, m.one_sh) * m.q;      // [0, 4q)
  u64 s = t + r;                                       // [0, 8q)
  s = csub(s, 4 * m.q);
  s = csub(s, 2 * m.q);
  return csub(s, m.q);
}
// Montgomery's reduction ("Modular multiplication without trial division",
// 1985) with R = 2^64: s R^{-1} mod q, fully reduced, for s = hi 2^64 + lo
// with hi < q.  With m = lo q^{-1} mod 2^64 the low words of s and m q agree,
// so s - m q = (hi - floor(m q / 2^64)) 2^64 with the bracket in (-q, q).
// One low and one high 64-bit product: half the multiplier work of
// reduce128.  Callers fold the factor R into a constant operand.
__device__ __forceinline__ u64 redc(U128 s, const DMod& m) {
  const u64 mh = __umul64hi(s.lo * m.qinv, m.q);
  return s.hi >= mh ? s.hi - mh : s.hi - mh + m.q;
}
__device__ __forceinline__ u64 mulm(u64 a, u64 b, const DMod& m) {
  U128 x{a * b, __umul64hi(a, b)};
  return reduce128(x, m);
}
// [c]_q of a signed integer c stored in a word (the centred c_l of the
// fused tail); `small` says |c| < q is known.
__device__ __forceinline__ u64 lift_signed(u64 word, const DMod& md, int small) {
  const long long c = (long long)word;
  const u64 mag = c < 0 ? (u64)(-c) : (u64)c;
  const u64 m = small ? mag : csub(shoup_lazy(mag, 1, md.one_sh, md.q), md.q);
  return c < 0 ? negm(m, md.q) : m;
}
#endif  // __CUDACC__

