// Negacyclic NTT over 64-bit primes, batched over limbs.
//
// Forward: Cooley-Tukey butterflies with the powers psi^{brv(k)} of a
// primitive 2N-th root psi (the negacyclic twist merged into the twiddles,
// Longa & Naehrig, "Speeding up the Number Theoretic Transform for Faster
// Ideal Lattice-Based Cryptography", 2016).  Input in natural order, output
// in bit-reversed order: slot k holds a(psi^{2 brv(k) + 1}).
// Inverse: Gentleman-Sande butterflies with psi^{-brv(k)}, then N^{-1}.
// In stage st (m = 2^st groups, half distance t = N / 2^{st+1}) the pair
// (j, j + t) uses twiddle index m + (j >> (log N - st)).
//
// Butterflies are Harvey's lazy forms (values in [0, 4q) forward, [0, 2q)
// inverse; "Faster arithmetic for number-theoretic transforms", 2014); each
// pass ends fully reduced.
//
// N = 2^n is split as R x C with R = 2^n1 rows and C = 2^n2 columns
// (j = row * C + col).  The first n1 forward stages mix only rows: a
// "column pass" CTA owns all R rows of TC adjacent columns.  The remaining
// n2 stages mix only within a row: a "row pass" CTA owns RP whole rows.
// Inside a pass the stages run in two register rounds: 2^K1 points strided
// by 2^K2 (the K1 long-distance stages), then 2^K2 adjacent points (the K2
// short-distance stages), with one shared-memory exchange between them.
// The inverse runs the rounds and the passes in the opposite order.  Each
// pass reads and writes each limb once.
#include "hc_internal.h"

namespace {

constexpr int kThreads = 256;

// Forward CT stages st0 .. st0+K-1 on 2^K points; point i has global index
// jb + (i << ls); in local stage s the pair distance is 2^{K-1-s} points.
template <int K>
__device__ __forceinline__ void fwd_block(u64 (&x)[1 << K], u64 jb, int ls, int st0, const ulonglong2* tw, u64 q,
                                          int log_n) {
  const u64 q2 = 2 * q;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int st = st0 + s;
    const int half = 1 << (K - 1 - s);
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) {
      if (i & half) continue;
      const u64 j = jb + ((u64)i << ls);
      const ulonglong2 w = __ldg(tw + ((1ull << st) + (j >> (log_n - st))));
      u64 X = x[i];
      X = X >= q2 ? X - q2 : X;
      const u64 T = shoup_lazy(x[i + half], w.x, w.y, q);
      x[i] = X + T;
      x[i + half] = X - T + q2;
    }
  }
}

// Inverse GS stages st_hi, st_hi-1, .. st_hi-K+1 on 2^K points with global
// indices jb + (i << ls); in local stage s the pair distance is 2^s points.
// Inputs and outputs in [0, 2q).
template <int K>
__device__ __forceinline__ void inv_block(u64 (&x)[1 << K], u64 jb, int ls, int st_hi, const ulonglong2* tw, u64 q,
                                          int log_n) {
  const u64 q2 = 2 * q;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int st = st_hi - s;
    const int half = 1 << s;
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) {
      if (i & half) continue;
      const u64 j = jb + ((u64)i << ls);
      const ulonglong2 w = __ldg(tw + ((1ull << st) + (j >> (log_n - st))));
      const u64 U = x[i], V = x[i + half];
      u64 S = U + V;
      S = S >= q2 ? S - q2 : S;
      x[i] = S;
      x[i + half] = shoup_lazy(U - V + q2, w.x, w.y, q);
    }
  }
}

__device__ __forceinline__ u64 reduce4(u64 x, u64 q) {
  x = x >= 2 * q ? x - 2 * q : x;
  return x >= q ? x - q : x;
}

__device__ __forceinline__ void limb_meta(const LimbSet& s, int log_n, u64*& a, int& pid) {
  const int y = blockIdx.y;
  const int k = y / s.nlimb;
  const int slot = s.l0 + y - k * s.nlimb;
  a = limb_ptr(s, blockIdx.z, k, slot, 1 << log_n);
  pid = limb_prime(s, slot);
}

// Column pass: stages 0..n1-1 (forward) over R = 2^(K1+K2) rows of TC = 2^tcl
// columns starting at blockIdx.x * TC.  Shared tile [row][col].
template <bool INV, int K1, int K2>
__global__ void __launch_bounds__(kThreads) k_cols(LimbSet s, Tables T, int n2, int tcl) {
  constexpr int n1 = K1 + K2;
  extern __shared__ u64 sm[];
  const int log_n = T.log_n;
  u64* a;
  int pid;
  limb_meta(s, log_n, a, pid);
  const u64 q = T.mods[pid].q;
  const ulonglong2* tw = (INV ? T.inv2 : T.fwd2) + ((size_t)pid << log_n);
  const int TC = 1 << tcl;
  const int c0 = blockIdx.x * TC;
  if (!INV) {
    // round 1: 2^K1 rows strided by 2^K2 -> stages 0..K1-1
    for (int w = threadIdx.x; w < (TC << K2); w += blockDim.x) {
      const int c = w & (TC - 1), r0 = w >> tcl;
      u64 x[1 << K1];
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) x[i] = a[((size_t)(r0 + (i << K2)) << n2) + c0 + c];
      fwd_block<K1>(x, (u64)r0 << n2, K2 + n2, 0, tw, q, log_n);
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) sm[((r0 + (i << K2)) << tcl) + c] = x[i];
    }
    __syncthreads();
    // round 2: 2^K2 adjacent rows -> stages K1..n1-1
    for (int w = threadIdx.x; w < (TC << K1); w += blockDim.x) {
      const int c = w & (TC - 1), g = w >> tcl;
      u64 x[1 << K2];
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) x[i] = sm[(((g << K2) + i) << tcl) + c];
      fwd_block<K2>(x, (u64)(g << K2) << n2, n2, K1, tw, q, log_n);
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) a[((size_t)((g << K2) + i) << n2) + c0 + c] = reduce4(x[i], q);
    }
  } else {
    // round A: 2^K2 adjacent rows -> stages n1-1 .. K1
    for (int w = threadIdx.x; w < (TC << K1); w += blockDim.x) {
      const int c = w & (TC - 1), g = w >> tcl;
      u64 x[1 << K2];
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) x[i] = a[((size_t)((g << K2) + i) << n2) + c0 + c];
      inv_block<K2>(x, (u64)(g << K2) << n2, n2, n1 - 1, tw, q, log_n);
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) sm[(((g << K2) + i) << tcl) + c] = x[i];
    }
    __syncthreads();
    // round B: 2^K1 rows strided by 2^K2 -> stages K1-1 .. 0, then N^{-1}
    const u64 ni = T.ninv[pid], nis = T.ninv_sh[pid];
    for (int w = threadIdx.x; w < (TC << K2); w += blockDim.x) {
      const int c = w & (TC - 1), r0 = w >> tcl;
      u64 x[1 << K1];
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) x[i] = sm[((r0 + (i << K2)) << tcl) + c];
      inv_block<K1>(x, (u64)r0 << n2, K2 + n2, K1 - 1, tw, q, log_n);
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i)
        a[((size_t)(r0 + (i << K2)) << n2) + c0 + c] = reduce4(shoup_lazy(x[i], ni, nis, q), q);
    }
  }
}

// Row pass: stages n1..log_n-1 (forward) inside RP rows of C = 2^(K1+K2)
// adjacent points.  Shared rows padded by one word per 2^K2 words.
template <bool INV, int K1, int K2>
__global__ void __launch_bounds__(kThreads) k_rows(LimbSet s, Tables T, int n1, int rpl) {
  constexpr int n2 = K1 + K2, C = 1 << n2;
  constexpr int PADW = C + (C >> K2);  // padded row width
  extern __shared__ u64 sm[];
  const int log_n = T.log_n;
  u64* a;
  int pid;
  limb_meta(s, log_n, a, pid);
  const u64 q = T.mods[pid].q;
  const ulonglong2* tw = (INV ? T.inv2 : T.fwd2) + ((size_t)pid << log_n);
  const int RP = 1 << rpl;
  const int row0 = blockIdx.x * RP;
  u64* src = a + ((size_t)row0 << n2);
  auto sidx = [&](int r, int j) { return r * PADW + j + (j >> K2); };
  if (!INV) {
    // round 1: 2^K1 points strided by 2^K2 (straight from global)
    for (int w = threadIdx.x; w < (RP << K2); w += blockDim.x) {
      const int r = w >> K2, r0 = w & ((1 << K2) - 1);
      u64 x[1 << K1];
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) x[i] = src[((size_t)r << n2) + r0 + (i << K2)];
      fwd_block<K1>(x, ((u64)(row0 + r) << n2) + r0, K2, n1, tw, q, log_n);
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) sm[sidx(r, r0 + (i << K2))] = x[i];
    }
    __syncthreads();
    // round 2: 2^K2 adjacent points
    for (int w = threadIdx.x; w < (RP << K1); w += blockDim.x) {
      const int r = w >> K1, g = w & ((1 << K1) - 1);
      u64 x[1 << K2];
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) x[i] = sm[sidx(r, (g << K2) + i)];
      fwd_block<K2>(x, ((u64)(row0 + r) << n2) + (g << K2), 0, n1 + K1, tw, q, log_n);
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) sm[sidx(r, (g << K2) + i)] = reduce4(x[i], q);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (RP << n2); e += blockDim.x) src[e] = sm[sidx(e >> n2, e & (C - 1))];
  } else {
    for (int e = threadIdx.x; e < (RP << n2); e += blockDim.x) sm[sidx(e >> n2, e & (C - 1))] = src[e];
    __syncthreads();
    // round A: 2^K2 adjacent points -> stages log_n-1 .. log_n-K2
    for (int w = threadIdx.x; w < (RP << K1); w += blockDim.x) {
      const int r = w >> K1, g = w & ((1 << K1) - 1);
      u64 x[1 << K2];
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) x[i] = sm[sidx(r, (g << K2) + i)];
      inv_block<K2>(x, ((u64)(row0 + r) << n2) + (g << K2), 0, log_n - 1, tw, q, log_n);
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) sm[sidx(r, (g << K2) + i)] = x[i];
    }
    __syncthreads();
    // round B: 2^K1 points strided by 2^K2 -> stages log_n-K2-1 .. n1 (to global)
    for (int w = threadIdx.x; w < (RP << K2); w += blockDim.x) {
      const int r = w >> K2, r0 = w & ((1 << K2) - 1);
      u64 x[1 << K1];
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) x[i] = sm[sidx(r, r0 + (i << K2))];
      inv_block<K1>(x, ((u64)(row0 + r) << n2) + r0, K2, log_n - 1 - K2, tw, q, log_n);
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) src[((size_t)r << n2) + r0 + (i << K2)] = reduce4(x[i], q);
    }
  }
}

template <bool INV, int K1, int K2>
void launch_cols(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, int n2) {
  constexpr int n1 = K1 + K2;
  // enough (column, offset) work items for every thread in both rounds
  int tcl = 8 - (K1 < K2 ? K1 : K2);
  if (tcl > n2) tcl = n2;
  while (((size_t)1 << (n1 + tcl)) * sizeof(u64) > 48 * 1024) --tcl;
  dim3 grid(1u << (n2 - tcl), ylimbs, items);
  const size_t smem = ((size_t)1 << (n1 + tcl)) * sizeof(u64);
  ProfScope p(ctx, INV ? "ntt_inv_cols" : "ntt_fwd_cols", (uint64_t)ylimbs * items);
  k_cols<INV, K1, K2><<<grid, kThreads, smem, ctx->stream>>>(s, ctx->tab, n2, tcl);
}

template <bool INV, int K1, int K2>
void launch_rows(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, int n1) {
  constexpr int n2 = K1 + K2;
  int rpl = 8 - (K1 < K2 ? K1 : K2);
  if (rpl > n1) rpl = n1;
  const size_t padw = ((size_t)1 << n2) + ((size_t)1 << (n2 - K2));
  while (((size_t)1 << rpl) * padw * sizeof(u64) > 48 * 1024) --rpl;
  dim3 grid(1u << (n1 - rpl), ylimbs, items);
  const size_t smem = ((size_t)1 << rpl) * padw * sizeof(u64);
  ProfScope p(ctx, INV ? "ntt_inv_rows" : "ntt_fwd_rows", (uint64_t)ylimbs * items);
  k_rows<INV, K1, K2><<<grid, kThreads, smem, ctx->stream>>>(s, ctx->tab, n1, rpl);
}

// Stage splits of a pass of n stages into two register rounds.
template <bool INV>
void cols_dispatch(hc_ctx* ctx, const LimbSet& s, int items, int y, int n1, int n2) {
  switch (n1) {
    case 5: launch_cols<INV, 3, 2>(ctx, s, items, y, n2); break;
    case 6: launch_cols<INV, 3, 3>(ctx, s, items, y, n2); break;
    case 7: launch_cols<INV, 4, 3>(ctx, s, items, y, n2); break;
    case 8: launch_cols<INV, 4, 4>(ctx, s, items, y, n2); break;
    default: throw HcError{HC_ERR_INVALID, "unsupported ring degree"};
  }
}

template <bool INV>
void rows_dispatch(hc_ctx* ctx, const LimbSet& s, int items, int y, int n1, int n2) {
  switch (n2) {
    case 5: launch_rows<INV, 3, 2>(ctx, s, items, y, n1); break;
    case 6: launch_rows<INV, 3, 3>(ctx, s, items, y, n1); break;
    case 7: launch_rows<INV, 4, 3>(ctx, s, items, y, n1); break;
    case 8: launch_rows<INV, 4, 4>(ctx, s, items, y, n1); break;
    default: throw HcError{HC_ERR_INVALID, "unsupported ring degree"};
  }
}

}  // namespace

void launch_ntt(hc_ctx* ctx, const LimbSet& s, int items, bool inverse) {
  if (items <= 0 || s.nlimb <= 0 || s.npoly <= 0) return;
  const int log_n = ctx->P.log_n;
  const int n1 = log_n / 2, n2 = log_n - n1;
  const int ylimbs = s.npoly * s.nlimb;
  HC_CHECK(ylimbs <= 65535 && items <= 65535, HC_ERR_INVALID, "NTT batch too large");
  if (!inverse) {
    cols_dispatch<false>(ctx, s, items, ylimbs, n1, n2);
    rows_dispatch<false>(ctx, s, items, ylimbs, n1, n2);
  } else {
    rows_dispatch<true>(ctx, s, items, ylimbs, n1, n2);
    cols_dispatch<true>(ctx, s, items, ylimbs, n1, n2);
  }
  ctx->launches += 2;
  check_launch(ctx);
}
