// Negacyclic NTT over 64-bit primes, batched over limbs.
//
// Forward: Cooley-Tukey butterflies with the powers psi^{brv(k)} of a
// primitive 2N-th root psi (the negacyclic twist merged into the twiddles,
// Longa & Naehrig, "Speeding up the Number Theoretic Transform for Faster
// Ideal Lattice-Based Cryptography", 2016).  Input in natural order, output
// in bit-reversed order: slot k holds a(psi^{2 brv(k) + 1}).
// Inverse: Gentleman-Sande butterflies with psi^{-brv(k)}, then N^{-1}.
//
// N = 2^n is split as R x Cn with R = 2^n1 rows and Cn = 2^n2 columns
// (element j = row * Cn + col).  The first n1 forward stages mix only rows
// (strides >= Cn): a "column pass" CTA owns a tile of all R rows x TC
// adjacent columns in shared memory.  The remaining n2 stages mix only
// within a row: a "row pass" CTA owns RP whole rows.  The inverse runs the
// row pass first.  Each pass reads and writes every limb once.
#include "hc_internal.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void load_limb_meta(const LimbSet& s, const Tables& T, u64*& a, int& pid) {
  const int n = 1 << T.log_n;
  const int y = blockIdx.y;
  const int k = y / s.nlimb;
  const int slot = s.l0 + y % s.nlimb;
  a = limb_ptr(s, blockIdx.z, k, slot, n);
  pid = limb_prime(s, slot);
}

template <bool INV>
__global__ void __launch_bounds__(kThreads) k_cols(LimbSet s, Tables T, int n1, int n2, int tc) {
  extern __shared__ u64 sm[];
  u64* a;
  int pid;
  load_limb_meta(s, T, a, pid);
  const int n = 1 << T.log_n, R = 1 << n1;
  const u64 q = T.mods[pid].q;
  const u64* w = (INV ? T.inv : T.fwd) + (size_t)pid * n;
  const u64* wsh = (INV ? T.inv_sh : T.fwd_sh) + (size_t)pid * n;
  const int c0 = blockIdx.x * tc;
  const int tot = R * tc;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int r = e / tc, c = e - r * tc;
    sm[e] = a[((size_t)r << n2) + c0 + c];
  }
  __syncthreads();
  const int nb = (R >> 1) * tc;
  for (int it = 0; it < n1; ++it) {
    const int st = INV ? (n1 - 1 - it) : it;
    const int m = 1 << st, th = R >> (st + 1);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int bb = b / tc, c = b - bb * tc;
      const int grp = bb / th, off = bb - grp * th;
      const int r = grp * 2 * th + off;
      const u64 W = __ldg(w + m + grp), Ws = __ldg(wsh + m + grp);
      u64* px = sm + r * tc + c;
      u64* py = px + th * tc;
      const u64 U = *px, V = *py;
      if (!INV) {
        const u64 t = shoup(V, W, Ws, q);
        *px = addm(U, t, q);
        *py = subm(U, t, q);
      } else {
        *px = addm(U, V, q);
        *py = shoup(subm(U, V, q), W, Ws, q);
      }
    }
    __syncthreads();
  }
  if (INV) {
    const u64 ni = T.ninv[pid], nis = T.ninv_sh[pid];
    for (int e = threadIdx.x; e < tot; e += blockDim.x) sm[e] = shoup(sm[e], ni, nis, q);
    __syncthreads();
  }
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int r = e / tc, c = e - r * tc;
    a[((size_t)r << n2) + c0 + c] = sm[e];
  }
}

template <bool INV>
__global__ void __launch_bounds__(kThreads) k_rows(LimbSet s, Tables T, int n1, int n2, int rp) {
  extern __shared__ u64 sm[];
  u64* a;
  int pid;
  load_limb_meta(s, T, a, pid);
  const int n = 1 << T.log_n, rowlen = 1 << n2, half = rowlen >> 1;
  const u64 q = T.mods[pid].q;
  const u64* w = (INV ? T.inv : T.fwd) + (size_t)pid * n;
  const u64* wsh = (INV ? T.inv_sh : T.fwd_sh) + (size_t)pid * n;
  const int row0 = blockIdx.x * rp;
  const int tot = rp * rowlen;
  u64* src = a + (size_t)row0 * rowlen;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) sm[e] = src[e];
  __syncthreads();
  const int nb = rp * half;
  for (int it = 0; it < n2; ++it) {
    const int st = INV ? (T.log_n - 1 - it) : (n1 + it);
    const int m = 1 << st, t = n >> (st + 1);
    const int groups_per_row = rowlen / (2 * t);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int row = b / half, bl = b - row * half;
      const int gl = bl / t, off = bl - gl * t;
      const int j = gl * 2 * t + off;
      const int i = (row0 + row) * groups_per_row + gl;
      const u64 W = __ldg(w + m + i), Ws = __ldg(wsh + m + i);
      u64* px = sm + row * rowlen + j;
      u64* py = px + t;
      const u64 U = *px, V = *py;
      if (!INV) {
        const u64 tt = shoup(V, W, Ws, q);
        *px = addm(U, tt, q);
        *py = subm(U, tt, q);
      } else {
        *px = addm(U, V, q);
        *py = shoup(subm(U, V, q), W, Ws, q);
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < tot; e += blockDim.x) src[e] = sm[e];
}

}  // namespace

void launch_ntt(hc_ctx* ctx, const LimbSet& s, int items, bool inverse) {
  if (items <= 0 || s.nlimb <= 0 || s.npoly <= 0) return;
  const int log_n = ctx->P.log_n;
  const int n1 = log_n / 2, n2 = log_n - n1;
  const int R = 1 << n1, Cn = 1 << n2;
  const int tc = Cn < 16 ? Cn : 16;
  int rp = 4096 >> n2;
  if (rp < 1) rp = 1;
  if (rp > R) rp = R;
  const int ylimbs = s.npoly * s.nlimb;
  HC_CHECK(ylimbs <= 65535 && items <= 65535, HC_ERR_INVALID, "NTT batch too large");
  dim3 gc(Cn / tc, ylimbs, items), gr(R / rp, ylimbs, items);
  const size_t smc = (size_t)R * tc * sizeof(u64), smr = (size_t)rp * Cn * sizeof(u64);
  if (!inverse) {
    {
      ProfScope p(ctx, "ntt_fwd_cols", (uint64_t)ylimbs * items);
      k_cols<false><<<gc, kThreads, smc, ctx->stream>>>(s, ctx->tab, n1, n2, tc);
    }
    {
      ProfScope p(ctx, "ntt_fwd_rows", (uint64_t)ylimbs * items);
      k_rows<false><<<gr, kThreads, smr, ctx->stream>>>(s, ctx->tab, n1, n2, rp);
    }
  } else {
    {
      ProfScope p(ctx, "ntt_inv_rows", (uint64_t)ylimbs * items);
      k_rows<true><<<gr, kThreads, smr, ctx->stream>>>(s, ctx->tab, n1, n2, rp);
    }
    {
      ProfScope p(ctx, "ntt_inv_cols", (uint64_t)ylimbs * items);
      k_cols<true><<<gc, kThreads, smc, ctx->stream>>>(s, ctx->tab, n1, n2, tc);
    }
  }
  ctx->launches += 2;
  check_launch(ctx);
}
