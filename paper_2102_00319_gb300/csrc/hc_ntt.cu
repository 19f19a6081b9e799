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
#include <cooperative_groups.h>

#include "hc_internal.h"

namespace {

// Block sizes: 2^8 threads (tiles of 16 columns / rows at N = 2^16) or 2^7
// (tiles of 8); the context's tuning table picks one per ring degree.

// Forward CT stages ST0 .. ST0+K-1 on 2^K points; point i has global index
// jb + (i << LS), where jb has no bits in common with i << LS (so the
// twiddle index splits into a per-stage part from jb and a constant from i).
// In local stage s the pair distance is 2^{K-1-s} points.
template <int K, int LS, int ST0, int LOGN>
__device__ __forceinline__ void fwd_block(u64 (&x)[1 << K], u32 jb, const ulonglong2* tw, u64 q) {
  const u64 q2 = 2 * q;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int st = ST0 + s;
    const int half = 1 << (K - 1 - s);
    const ulonglong2* tws = tw + ((1u << st) + (jb >> (LOGN - st)));
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) {
      if (i & half) continue;
      const ulonglong2 w = __ldg(tws + (((u32)i << LS) >> (LOGN - st)));
      u64 X = x[i];
      X = X >= q2 ? X - q2 : X;
      const u64 T = shoup_lazy(x[i + half], w.x, w.y, q);
      x[i] = X + T;
      x[i + half] = X - T + q2;
    }
  }
}

// Inverse GS stages STH, STH-1, .. STH-K+1 on 2^K points with global indices
// jb + (i << LS) (disjoint bits as above); in local stage s the pair distance
// is 2^s points.  Inputs and outputs in [0, 2q).
template <int K, int LS, int STH, int LOGN>
__device__ __forceinline__ void inv_block(u64 (&x)[1 << K], u32 jb, const ulonglong2* tw, u64 q) {
  const u64 q2 = 2 * q;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int st = STH - s;
    const int half = 1 << s;
    const ulonglong2* tws = tw + ((1u << st) + (jb >> (LOGN - st)));
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) {
      if (i & half) continue;
      const ulonglong2 w = __ldg(tws + (((u32)i << LS) >> (LOGN - st)));
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

template <int LOGN>
__device__ __forceinline__ void limb_meta(const LimbSet& s, u64*& a, int& pid) {
  const int y = blockIdx.y;
  const int k = y / s.nlimb;
  const int l = y - k * s.nlimb;
  const int slot = s.slot_map ? s.slot_map[s.slot_map_2d ? y : l] : s.l0 + l;
  a = limb_ptr(s, blockIdx.z, k, slot, 1 << LOGN);
  pid = limb_prime(s, slot);
}

// The input limb of an out-of-place pass: same (item, poly, limb) position in `in`.
template <int LOGN>
__device__ __forceinline__ const u64* input_limb(const LimbSet& s, const LimbSet& in) {
  const int y = blockIdx.y;
  const int k = y / s.nlimb;
  const int l = y - k * s.nlimb;
  return limb_ptr(in, blockIdx.z, k, in.l0 + l, 1 << LOGN);
}

// Column pass: stages 0..N1-1 (forward) over R = 2^N1 rows (N1 = K1 + K2) of
// TC = 2^TCL columns starting at blockIdx.x * TC.  Shared tile [row][col].
template <bool INV, int LOGN, int K1, int K2, int TCL, bool FUSE, int TL>
__global__ void __launch_bounds__(1 << TL) k_cols(LimbSet s, LimbSet in, int use_in, int scale, KsrFuse f,
                                                  Tables T) {
  constexpr int N1 = K1 + K2, N2 = LOGN - N1, TC = 1 << TCL;
  constexpr u32 kThreads = 1u << TL;
  extern __shared__ u64 sm[];
  u64* a;
  int pid;
  limb_meta<LOGN>(s, a, pid);
  const u64* ain = use_in ? input_limb<LOGN>(s, in) : a;  // first loads (out-of-place pass)
  const u64 q = T.mods[pid].q;
  const ulonglong2* tw = (INV ? T.inv2 : T.fwd2) + ((size_t)pid << LOGN);
  a += blockIdx.x * TC;
  ain += blockIdx.x * TC;
  // fused relinearise + rescale: limb slot (prime) and the c_l row of this block
  const int fslot = blockIdx.y % s.nlimb, fpoly = blockIdx.y / s.nlimb;
  const u64* fcl = FUSE ? f.cl + ((size_t)blockIdx.z * 2 + fpoly) * ((size_t)1 << LOGN) + blockIdx.x * TC : nullptr;
  if (!INV) {
    // first register round: 2^K1 rows strided by 2^K2 -> stages 0..K1-1
    for (u32 w = threadIdx.x; w < (TC << K2); w += kThreads) {
      const u32 c = w & (TC - 1), r0 = w >> TCL;
      u64 x[1 << K1];
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) {
        const u32 e = ((r0 + (i << K2)) << N2) + c;
        if constexpr (FUSE) {
          // z + [c_l]_{q_i} (z carries P^{-1}; c_l centred, its sign carried by the stored integer)
          x[i] = addm(ain[e], lift_signed(fcl[e], T.mods[pid], f.cl_small), q);
        } else {
          x[i] = ain[e];
        }
      }
      fwd_block<K1, K2 + N2, 0, LOGN>(x, r0 << N2, tw, q);
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) sm[((r0 + (i << K2)) << TCL) + c] = x[i];
    }
    __syncthreads();
    // second register round: 2^K2 adjacent rows -> stages K1..N1-1
    for (u32 w = threadIdx.x; w < (TC << K1); w += kThreads) {
      const u32 c = w & (TC - 1), g = w >> TCL;
      u64 x[1 << K2];
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) x[i] = sm[(((g << K2) + i) << TCL) + c];
      fwd_block<K2, N2, K1, LOGN>(x, (g << K2) << N2, tw, q);
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) a[(((g << K2) + i) << N2) + c] = reduce4(x[i], q);
    }
  } else {
    // first inverse round: 2^K2 adjacent rows -> stages N1-1 .. K1
    for (u32 w = threadIdx.x; w < (TC << K1); w += kThreads) {
      const u32 c = w & (TC - 1), g = w >> TCL;
      u64 x[1 << K2];
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) x[i] = ain[(((g << K2) + i) << N2) + c];
      inv_block<K2, N2, N1 - 1, LOGN>(x, (g << K2) << N2, tw, q);
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) sm[(((g << K2) + i) << TCL) + c] = x[i];
    }
    __syncthreads();
    // second inverse round: 2^K1 rows strided by 2^K2 -> stages K1-1 .. 0, then N^{-1}
    const u64 ni = T.ninv[pid], nis = T.ninv_sh[pid];
    // coefficient-form relinearise + rescale tail: z_k[i] and c_l of this block
    const u64* fz = FUSE ? f.z + (size_t)blockIdx.z * f.z_item_stride + (size_t)fpoly * f.z_poly_stride +
                               ((size_t)fslot << LOGN) + blockIdx.x * TC
                         : nullptr;
    for (u32 w = threadIdx.x; w < (TC << K2); w += kThreads) {
      const u32 c = w & (TC - 1), r0 = w >> TCL;
      u64 x[1 << K1];
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) x[i] = sm[((r0 + (i << K2)) << TCL) + c];
      inv_block<K1, K2 + N2, K1 - 1, LOGN>(x, r0 << N2, tw, q);
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) {
        const u32 e = ((r0 + (i << K2)) << N2) + c;
        if constexpr (FUSE) {
          // INTT(y) q_l^{-1} - (z + [c_l]_{q_i}) q_l^{-1}, N^{-1} folded into the first constant
          const int lv = f.level;
          const u64 yv = csub(shoup_lazy(x[i], f.nqlinv[fslot], f.nqlinv[lv + fslot], q), q);
          const u64 w = addm(fz[e], lift_signed(fcl[e], T.mods[pid], f.cl_small), q);
          a[e] = subm(yv, shoup(w, f.qlinv[fslot], f.qlinv[lv + fslot], q), q);
        } else {
          a[e] = reduce4(scale ? shoup_lazy(x[i], ni, nis, q) : x[i], q);
        }
      }
    }
  }
}

// Row pass: stages N1..LOGN-1 (forward) inside RP = 2^RPL rows of C = 2^N2
// adjacent points (N2 = K1 + K2).  Shared rows padded by one word per 2^K2.
template <bool INV, int LOGN, int K1, int K2, int RPL, bool FUSE, int TL>
__global__ void __launch_bounds__(1 << TL) k_rows(LimbSet s, LimbSet in, int use_in, KsrFuse f, Tables T) {
  constexpr u32 kThreads = 1u << TL;
  constexpr int N2 = K1 + K2, N1 = LOGN - N2, C = 1 << N2, RP = 1 << RPL;
  constexpr int PADW = C + (C >> K2);
  extern __shared__ u64 sm[];
  u64* a;
  int pid;
  limb_meta<LOGN>(s, a, pid);
  const u64* ain = use_in ? input_limb<LOGN>(s, in) : a;  // first loads (out-of-place pass)
  const u64 q = T.mods[pid].q;
  const ulonglong2* tw = (INV ? T.inv2 : T.fwd2) + ((size_t)pid << LOGN);
  const u32 row0 = blockIdx.x * RP;
  u64* src = a + ((size_t)row0 << N2);
  const u64* srcin = ain + ((size_t)row0 << N2);
  auto sidx = [](u32 r, u32 j) { return r * PADW + j + (j >> K2); };
  if (!INV) {
    // first register round: 2^K1 points strided by 2^K2 (straight from global)
    for (u32 w = threadIdx.x; w < (RP << K2); w += kThreads) {
      const u32 r = w >> K2, r0 = w & ((1 << K2) - 1);
      u64 x[1 << K1];
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) x[i] = srcin[(r << N2) + r0 + (i << K2)];
      fwd_block<K1, K2, N1, LOGN>(x, ((row0 + r) << N2) + r0, tw, q);
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) sm[sidx(r, r0 + (i << K2))] = x[i];
    }
    __syncthreads();
    // second register round: 2^K2 adjacent points; the results go back through shared
    // memory so that the stores to global memory are row-contiguous across
    // the warp (measured faster than each thread storing its own points)
    for (u32 w = threadIdx.x; w < (RP << K1); w += kThreads) {
      const u32 r = w >> K1, g = w & ((1 << K1) - 1);
      u64 x[1 << K2];
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) x[i] = sm[sidx(r, (g << K2) + i)];
      fwd_block<K2, 0, N1 + K1, LOGN>(x, ((row0 + r) << N2) + (g << K2), tw, q);
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) sm[sidx(r, (g << K2) + i)] = reduce4(x[i], q);
    }
    __syncthreads();
    if constexpr (FUSE) {
      // out_k[i] = (base_k[i] + acc_k[i] - w) q_l^{-1} for the NTT output w (acc carries P^{-1})
      const int slot = blockIdx.y % s.nlimb, k = blockIdx.y / s.nlimb, z = blockIdx.z;
      const size_t li0 = ((size_t)slot << LOGN) + ((size_t)row0 << N2);
      const u64* accp = f.acc + (size_t)z * f.acc_item_stride + (size_t)k * f.acc_poly_stride + li0;
      const CtRef* base = k == 0 ? f.base0 : f.base1;
      const u64* bp = base ? base[z].p + li0 : nullptr;
      u64* op = f.out[z].p + (size_t)k * f.out[z].stride + li0;
      const u64 qv = f.qlinv[slot], qvs = f.qlinv[f.level + slot];
      // four elements per thread per step: their global loads are in flight together
      constexpr u32 kTile = RP << N2, kU = 4;
      static_assert(kTile % (kThreads * kU) == 0, "epilogue tile");
      for (u32 e0 = threadIdx.x; e0 < kTile; e0 += kThreads * kU) {
        u64 av[kU], bv[kU];
#pragma unroll
        for (u32 u = 0; u < kU; ++u) {
          av[u] = accp[e0 + u * kThreads];
          bv[u] = bp ? bp[e0 + u * kThreads] : 0;
        }
#pragma unroll
        for (u32 u = 0; u < kU; ++u) {
          const u32 e = e0 + u * kThreads;
          u64 r = addm(av[u], bv[u], q);
          r = subm(r, sm[sidx(e >> N2, e & (C - 1))], q);
          op[e] = shoup(r, qv, qvs, q);
        }
      }
    } else {
      for (u32 e = threadIdx.x; e < (RP << N2); e += kThreads) src[e] = sm[sidx(e >> N2, e & (C - 1))];
    }
  } else {
    // first inverse round: 2^K2 adjacent points read straight from global memory as
    // 16-byte pairs (a thread's points are contiguous and 16-byte aligned;
    // measured faster than staging the tile through shared memory)
    // -> stages LOGN-1 .. LOGN-K2
    // coefficient-form relinearise + rescale tail: y = base_k[i] + acc_k[i] on load
    const u64* faccp = nullptr;
    const u64* fbp = nullptr;
    if constexpr (FUSE) {
      const int slot = blockIdx.y % s.nlimb, k = blockIdx.y / s.nlimb, z = blockIdx.z;
      const size_t li0 = ((size_t)slot << LOGN) + ((size_t)row0 << N2);
      faccp = f.acc + (size_t)z * f.acc_item_stride + (size_t)k * f.acc_poly_stride + li0;
      const CtRef* base = k == 0 ? f.base0 : f.base1;
      fbp = base ? base[z].p + li0 : nullptr;
    }
    for (u32 w = threadIdx.x; w < (RP << K1); w += kThreads) {
      const u32 r = w >> K1, g = w & ((1 << K1) - 1);
      u64 x[1 << K2];
      if constexpr (FUSE) {
        const u32 o = (r << N2) + (g << K2);
        const ulonglong2* a2 = reinterpret_cast<const ulonglong2*>(faccp + o);
#pragma unroll
        for (int i = 0; i < (1 << K2); i += 2) {
          const ulonglong2 v = a2[i >> 1];
          x[i] = v.x;
          x[i + 1] = v.y;
        }
        if (fbp) {
          const ulonglong2* b2 = reinterpret_cast<const ulonglong2*>(fbp + o);
#pragma unroll
          for (int i = 0; i < (1 << K2); i += 2) {
            const ulonglong2 v = b2[i >> 1];
            x[i] = addm(x[i], v.x, q);
            x[i + 1] = addm(x[i + 1], v.y, q);
          }
        }
      } else {
        const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(srcin + (r << N2) + (g << K2));
#pragma unroll
        for (int i = 0; i < (1 << K2); i += 2) {
          const ulonglong2 v = s2[i >> 1];
          x[i] = v.x;
          x[i + 1] = v.y;
        }
      }
      inv_block<K2, 0, LOGN - 1, LOGN>(x, ((row0 + r) << N2) + (g << K2), tw, q);
#pragma unroll
      for (int i = 0; i < (1 << K2); ++i) sm[sidx(r, (g << K2) + i)] = x[i];
    }
    __syncthreads();
    // second inverse round: 2^K1 points strided by 2^K2 -> stages LOGN-K2-1 .. N1 (to global)
    for (u32 w = threadIdx.x; w < (RP << K2); w += kThreads) {
      const u32 r = w >> K2, r0 = w & ((1 << K2) - 1);
      u64 x[1 << K1];
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) x[i] = sm[sidx(r, r0 + (i << K2))];
      inv_block<K1, K2, LOGN - 1 - K2, LOGN>(x, ((row0 + r) << N2) + r0, tw, q);
#pragma unroll
      for (int i = 0; i < (1 << K1); ++i) src[(r << N2) + r0 + (i << K2)] = reduce4(x[i], q);
    }
  }
}

// ---------------------------------------------------------------------------
// Pipelined passes (tuning variant 5).  The same column and row passes as
// above, with a grid of at most as many CTAs as are resident at once; each
// CTA walks the tiles t = blockIdx.x, + gridDim.x, ... and, while it
// transforms tile t in shared memory, copies tile t + gridDim.x into a
// second buffer with asynchronous 16-byte copies (cp.async), so that the
// loads of one tile overlap the butterflies of the previous one.  The
// butterflies and their twiddle indices are those of k_cols / k_rows, so
// the words are the same.  Plain transforms only (the fused-tail passes
// keep the per-tile kernels).

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// every committed group but the newest one has landed (this thread's copies)
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Tile t of a pass over tiles_x tiles per limb, ylimbs limb rows per item:
// its output and input limbs, the limb's prime and the tile's index in it.
struct PipeTile {
  u64* a;
  const u64* ain;
  int pid;
  int bx;
};

template <int LOGN>
__device__ __forceinline__ PipeTile pipe_tile(const LimbSet& s, const LimbSet& in, int use_in, int t, int tiles_x,
                                              int ylimbs) {
  PipeTile p;
  p.bx = t % tiles_x;
  const int yz = t / tiles_x;
  const int y = yz % ylimbs, z = yz / ylimbs;
  const int k = y / s.nlimb, l = y - k * s.nlimb;
  const int slot = s.slot_map ? s.slot_map[s.slot_map_2d ? y : l] : s.l0 + l;
  p.a = limb_ptr(s, z, k, slot, 1 << LOGN);
  p.pid = limb_prime(s, slot);
  p.ain = use_in ? limb_ptr(in, z, k, in.l0 + l, 1 << LOGN) : p.a;
  return p;
}

// Column pass, pipelined.  Shared tile [row][col] as in k_cols, each group
// of 2^K2 rows shifted by 8 more words, so that the 2^K2-adjacent-row round
// reads whole 128-byte bank lines.
template <bool INV, int LOGN, int K1, int K2, int TCL, int TL>
__global__ void __launch_bounds__(1 << TL) k_cols_pipe(LimbSet s, LimbSet in, int use_in, int scale, int tiles_x,
                                                       int ylimbs, int total, Tables T) {
  constexpr int N1 = K1 + K2, N2 = LOGN - N1, TC = 1 << TCL;
  constexpr u32 kThreads = 1u << TL;
  constexpr int TILE = (1 << (N1 + TCL)) + (8 << K1);
  static_assert(TCL >= 1, "16-byte copies need two columns per row");
  extern __shared__ __align__(16) u64 sm[];
  auto sidx = [](u32 row, u32 c) { return (row << TCL) + c + ((row >> K2) << 3); };
  int t = blockIdx.x;
  if (t >= total) return;
  auto fetch = [&](int tt, u64* buf) {
    const PipeTile p = pipe_tile<LOGN>(s, in, use_in, tt, tiles_x, ylimbs);
    const u64* g = p.ain + p.bx * TC;
    const bool aligned = ((reinterpret_cast<uintptr_t>(g) & 15) == 0);
    for (u32 ch = threadIdx.x; ch < (TILE - (8 << K1)) / 2; ch += kThreads) {
      const u32 row = ch >> (TCL - 1), c = (ch & ((TC >> 1) - 1)) << 1;
      const u64* src = g + ((size_t)row << N2) + c;
      if (aligned) {
        cp_async16(buf + sidx(row, c), src);
      } else {  // plain loads for a limb that does not start on a 16-byte boundary
        buf[sidx(row, c)] = src[0];
        buf[sidx(row, c) + 1] = src[1];
      }
    }
  };
  int cur = 0;
  fetch(t, sm);
  cp_async_commit();
  for (; t < total; t += gridDim.x) {
    if (t + (int)gridDim.x < total) fetch(t + gridDim.x, sm + (cur ^ 1) * TILE);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    u64* buf = sm + cur * TILE;
    const PipeTile p = pipe_tile<LOGN>(s, in, use_in, t, tiles_x, ylimbs);
    const u64 q = T.mods[p.pid].q;
    const ulonglong2* tw = (INV ? T.inv2 : T.fwd2) + ((size_t)p.pid << LOGN);
    u64* a = p.a + p.bx * TC;
    if (!INV) {
      // 2^K1 rows strided by 2^K2 -> stages 0..K1-1, in place
      for (u32 w = threadIdx.x; w < (TC << K2); w += kThreads) {
        const u32 c = w & (TC - 1), r0 = w >> TCL;
        u64 x[1 << K1];
#pragma unroll
        for (int i = 0; i < (1 << K1); ++i) x[i] = buf[sidx(r0 + (i << K2), c)];
        fwd_block<K1, K2 + N2, 0, LOGN>(x, r0 << N2, tw, q);
#pragma unroll
        for (int i = 0; i < (1 << K1); ++i) buf[sidx(r0 + (i << K2), c)] = x[i];
      }
      __syncthreads();
      // 2^K2 adjacent rows -> stages K1..N1-1, to global memory
      for (u32 w = threadIdx.x; w < (TC << K1); w += kThreads) {
        const u32 c = w & (TC - 1), g = w >> TCL;
        u64 x[1 << K2];
#pragma unroll
        for (int i = 0; i < (1 << K2); ++i) x[i] = buf[sidx((g << K2) + i, c)];
        fwd_block<K2, N2, K1, LOGN>(x, (g << K2) << N2, tw, q);
#pragma unroll
        for (int i = 0; i < (1 << K2); ++i) a[(((g << K2) + i) << N2) + c] = reduce4(x[i], q);
      }
    } else {
      // 2^K2 adjacent rows -> stages N1-1 .. K1, in place
      for (u32 w = threadIdx.x; w < (TC << K1); w += kThreads) {
        const u32 c = w & (TC - 1), g = w >> TCL;
        u64 x[1 << K2];
#pragma unroll
        for (int i = 0; i < (1 << K2); ++i) x[i] = buf[sidx((g << K2) + i, c)];
        inv_block<K2, N2, N1 - 1, LOGN>(x, (g << K2) << N2, tw, q);
#pragma unroll
        for (int i = 0; i < (1 << K2); ++i) buf[sidx((g << K2) + i, c)] = x[i];
      }
      __syncthreads();
      // 2^K1 rows strided by 2^K2 -> stages K1-1 .. 0, then N^{-1}, to global memory
      const u64 ni = T.ninv[p.pid], nis = T.ninv_sh[p.pid];
      for (u32 w = threadIdx.x; w < (TC << K2); w += kThreads) {
        const u32 c = w & (TC - 1), r0 = w >> TCL;
        u64 x[1 << K1];
#pragma unroll
        for (int i = 0; i < (1 << K1); ++i) x[i] = buf[sidx(r0 + (i << K2), c)];
        inv_block<K1, K2 + N2, K1 - 1, LOGN>(x, r0 << N2, tw, q);
#pragma unroll
        for (int i = 0; i < (1 << K1); ++i)
          a[((r0 + (i << K2)) << N2) + c] = reduce4(scale ? shoup_lazy(x[i], ni, nis, q) : x[i], q);
      }
    }
    __syncthreads();  // the buffer is refilled two tiles on
    cur ^= 1;
  }
  cp_async_wait_all();
}

// Row pass, pipelined.  Rows padded by two words per 2^K2 (the 16-byte
// copies stay aligned; the strided round reads whole bank lines and the
// adjacent round reads 16-byte pairs without conflicts).
template <bool INV, int LOGN, int K1, int K2, int RPL, int TL>
__global__ void __launch_bounds__(1 << TL) k_rows_pipe(LimbSet s, LimbSet in, int use_in, int tiles_x, int ylimbs,
                                                       int total, Tables T) {
  constexpr u32 kThreads = 1u << TL;
  constexpr int N2 = K1 + K2, N1 = LOGN - N2, C = 1 << N2, RP = 1 << RPL;
  constexpr int PADW = C + (C >> (K2 - 1));
  constexpr int TILE = RP * PADW;
  static_assert(K2 >= 1, "16-byte pairs need two adjacent points");
  extern __shared__ __align__(16) u64 sm[];
  auto sidx = [](u32 r, u32 j) { return r * PADW + j + ((j >> K2) << 1); };
  int t = blockIdx.x;
  if (t >= total) return;
  auto fetch = [&](int tt, u64* buf) {
    const PipeTile p = pipe_tile<LOGN>(s, in, use_in, tt, tiles_x, ylimbs);
    const u64* g = p.ain + ((size_t)p.bx * RP << N2);
    const bool aligned = ((reinterpret_cast<uintptr_t>(g) & 15) == 0);
    for (u32 ch = threadIdx.x; ch < (RP << N2) / 2; ch += kThreads) {
      const u32 e = ch << 1, r = e >> N2, j = e & (C - 1);
      if (aligned) {
        cp_async16(buf + sidx(r, j), g + e);
      } else {
        buf[sidx(r, j)] = g[e];
        buf[sidx(r, j) + 1] = g[e + 1];
      }
    }
  };
  int cur = 0;
  fetch(t, sm);
  cp_async_commit();
  for (; t < total; t += gridDim.x) {
    if (t + (int)gridDim.x < total) fetch(t + gridDim.x, sm + (cur ^ 1) * TILE);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    u64* buf = sm + cur * TILE;
    const PipeTile p = pipe_tile<LOGN>(s, in, use_in, t, tiles_x, ylimbs);
    const u64 q = T.mods[p.pid].q;
    const ulonglong2* tw = (INV ? T.inv2 : T.fwd2) + ((size_t)p.pid << LOGN);
    const u32 row0 = p.bx * RP;
    u64* dst = p.a + ((size_t)row0 << N2);
    if (!INV) {
      // 2^K1 points strided by 2^K2 -> stages N1 .. N1+K1-1, in place
      for (u32 w = threadIdx.x; w < (RP << K2); w += kThreads) {
        const u32 r = w >> K2, r0 = w & ((1 << K2) - 1);
        u64 x[1 << K1];
#pragma unroll
        for (int i = 0; i < (1 << K1); ++i) x[i] = buf[sidx(r, r0 + (i << K2))];
        fwd_block<K1, K2, N1, LOGN>(x, ((row0 + r) << N2) + r0, tw, q);
#pragma unroll
        for (int i = 0; i < (1 << K1); ++i) buf[sidx(r, r0 + (i << K2))] = x[i];
      }
      __syncthreads();
      // 2^K2 adjacent points -> the last K2 stages, reduced, in place
      for (u32 w = threadIdx.x; w < (RP << K1); w += kThreads) {
        const u32 r = w >> K1, g = w & ((1 << K1) - 1);
        ulonglong2* v2 = reinterpret_cast<ulonglong2*>(buf + sidx(r, g << K2));
        u64 x[1 << K2];
#pragma unroll
        for (int i = 0; i < (1 << K2); i += 2) {
          const ulonglong2 v = v2[i >> 1];
          x[i] = v.x;
          x[i + 1] = v.y;
        }
        fwd_block<K2, 0, N1 + K1, LOGN>(x, ((row0 + r) << N2) + (g << K2), tw, q);
#pragma unroll
        for (int i = 0; i < (1 << K2); i += 2) v2[i >> 1] = make_ulonglong2(reduce4(x[i], q), reduce4(x[i + 1], q));
      }
      __syncthreads();
      // row-contiguous 16-byte stores
      const bool aligned = ((reinterpret_cast<uintptr_t>(dst) & 15) == 0);
      for (u32 ch = threadIdx.x; ch < (RP << N2) / 2; ch += kThreads) {
        const u32 e = ch << 1, r = e >> N2, j = e & (C - 1);
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(buf + sidx(r, j));
        if (aligned) {
          *reinterpret_cast<ulonglong2*>(dst + e) = v;
        } else {
          dst[e] = v.x;
          dst[e + 1] = v.y;
        }
      }
    } else {
      // 2^K2 adjacent points -> stages LOGN-1 .. LOGN-K2, in place
      for (u32 w = threadIdx.x; w < (RP << K1); w += kThreads) {
        const u32 r = w >> K1, g = w & ((1 << K1) - 1);
        ulonglong2* v2 = reinterpret_cast<ulonglong2*>(buf + sidx(r, g << K2));
        u64 x[1 << K2];
#pragma unroll
        for (int i = 0; i < (1 << K2); i += 2) {
          const ulonglong2 v = v2[i >> 1];
          x[i] = v.x;
          x[i + 1] = v.y;
        }
        inv_block<K2, 0, LOGN - 1, LOGN>(x, ((row0 + r) << N2) + (g << K2), tw, q);
#pragma unroll
        for (int i = 0; i < (1 << K2); i += 2) v2[i >> 1] = make_ulonglong2(x[i], x[i + 1]);
      }
      __syncthreads();
      // 2^K1 points strided by 2^K2 -> stages LOGN-K2-1 .. N1, to global memory
      for (u32 w = threadIdx.x; w < (RP << K2); w += kThreads) {
        const u32 r = w >> K2, r0 = w & ((1 << K2) - 1);
        u64 x[1 << K1];
#pragma unroll
        for (int i = 0; i < (1 << K1); ++i) x[i] = buf[sidx(r, r0 + (i << K2))];
        inv_block<K1, K2, LOGN - 1 - K2, LOGN>(x, ((row0 + r) << N2) + r0, tw, q);
#pragma unroll
        for (int i = 0; i < (1 << K1); ++i) dst[(r << N2) + r0 + (i << K2)] = reduce4(x[i], q);
      }
    }
    __syncthreads();  // the buffer is refilled two tiles on
    cur ^= 1;
  }
  cp_async_wait_all();
}

// Pass geometry for ring degree 2^LOGN: the column pass takes floor(LOGN/2)
// stages, the row pass the rest; each pass splits into two register rounds.
template <int n>
struct Split {
  static constexpr int K1 = n == 5 ? 3 : (n == 6 ? 3 : 4);
  static constexpr int K2 = n - K1;
  static constexpr int KMIN = K1 < K2 ? K1 : K2;
};

constexpr int cmin(int a, int b) { return a < b ? a : b; }

// tiles: enough (column or row, offset) work items for all 2^TL threads, at
// most 48 KB of shared memory
template <int N1, int N2, int TL>
struct ColTile {
  static constexpr int raw = cmin(TL - Split<N1>::KMIN, N2);
  static constexpr int TCL = (1 << (N1 + raw)) * 8 > 48 * 1024 ? raw - 1 : raw;
};
template <int N1, int N2, int TL>
struct RowTile {
  static constexpr int K2 = Split<N2>::K2;
  static constexpr int PADW = (1 << N2) + (1 << (N2 - K2));
  static constexpr int raw = cmin(TL - Split<N2>::KMIN, N1);
  static constexpr int RPL = (1 << raw) * PADW * 8 > 48 * 1024 ? raw - 1 : raw;
};

template <bool INV, int LOGN, int TL>
void launch_pass_cols_t(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, const LimbSet* in, bool scale,
                        const KsrFuse* fuse) {
  constexpr int N1 = LOGN / 2, N2 = LOGN - N1;
  using Sp = Split<N1>;
  constexpr int TCL = ColTile<N1, N2, TL>::TCL;
  dim3 grid(1u << (N2 - TCL), ylimbs, items);
  const size_t smem = ((size_t)1 << (N1 + TCL)) * sizeof(u64);
  ProfScope p(ctx, INV ? (fuse ? "ntt_inv_cols_ksr" : "ntt_inv_cols") : (fuse ? "ntt_fwd_cols_ksr" : "ntt_fwd_cols"),
              (uint64_t)ylimbs * items);
  if (fuse)
    k_cols<INV, LOGN, Sp::K1, Sp::K2, TCL, true, TL><<<grid, 1 << TL, smem, ctx->stream>>>(s, s, 0, 1, *fuse,
                                                                                         ctx->tab);
  else
    k_cols<INV, LOGN, Sp::K1, Sp::K2, TCL, false, TL><<<grid, 1 << TL, smem, ctx->stream>>>(
        s, in ? *in : s, in ? 1 : 0, scale ? 1 : 0, KsrFuse{}, ctx->tab);
}

template <bool INV, int LOGN, int TL>
void launch_pass_rows_t(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, const LimbSet* in,
                        const KsrFuse* fuse) {
  constexpr int N1 = LOGN / 2, N2 = LOGN - N1;
  using Sp = Split<N2>;
  constexpr int RPL = RowTile<N1, N2, TL>::RPL;
  dim3 grid(1u << (N1 - RPL), ylimbs, items);
  const size_t smem = ((size_t)1 << RPL) * RowTile<N1, N2, TL>::PADW * sizeof(u64);
  ProfScope p(ctx, INV ? (fuse ? "ntt_inv_rows_ksr" : "ntt_inv_rows") : (fuse ? "ntt_fwd_rows_ksr" : "ntt_fwd_rows"),
              (uint64_t)ylimbs * items);
  if (fuse)
    k_rows<INV, LOGN, Sp::K1, Sp::K2, RPL, true, TL><<<grid, 1 << TL, smem, ctx->stream>>>(s, s, 0, *fuse,
                                                                                         ctx->tab);
  else
    k_rows<INV, LOGN, Sp::K1, Sp::K2, RPL, false, TL><<<grid, 1 << TL, smem, ctx->stream>>>(
        s, in ? *in : s, in ? 1 : 0, KsrFuse{}, ctx->tab);
}

// Pipelined passes: 128-thread CTAs, as many as are resident at once (at
// most one per tile).
template <typename K>
int pipe_grid(hc_ctx* ctx, K kern, size_t smem, long long total) {
  int per_sm = 0, sms = 0;
  HC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
  HC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  return (int)std::min<long long>(total, (long long)std::max(1, per_sm) * sms);
}

template <bool INV, int LOGN>
void launch_pass_cols_pipe(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, const LimbSet* in, bool scale) {
  constexpr int TL = 7, N1 = LOGN / 2, N2 = LOGN - N1;
  using Sp = Split<N1>;
  constexpr int TCL = ColTile<N1, N2, TL>::TCL;
  constexpr int TILE = (1 << (N1 + TCL)) + (8 << Sp::K1);
  const int tiles_x = 1 << (N2 - TCL);
  const long long total = (long long)tiles_x * ylimbs * items;
  HC_CHECK(total < (1ll << 31), HC_ERR_INVALID, "NTT batch too large");
  const size_t smem = 2 * (size_t)TILE * sizeof(u64);
  auto kern = k_cols_pipe<INV, LOGN, Sp::K1, Sp::K2, TCL, TL>;
  const int grid = pipe_grid(ctx, kern, smem, total);
  ProfScope p(ctx, INV ? "ntt_inv_cols" : "ntt_fwd_cols", (uint64_t)ylimbs * items);
  kern<<<grid, 1 << TL, smem, ctx->stream>>>(s, in ? *in : s, in ? 1 : 0, scale ? 1 : 0, tiles_x, ylimbs,
                                             (int)total, ctx->tab);
}

template <bool INV, int LOGN>
void launch_pass_rows_pipe(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, const LimbSet* in) {
  constexpr int TL = 7, N1 = LOGN / 2, N2 = LOGN - N1;
  using Sp = Split<N2>;
  constexpr int RPL = RowTile<N1, N2, TL>::RPL;
  constexpr int PADW = (1 << N2) + ((1 << N2) >> (Sp::K2 - 1));
  const int tiles_x = 1 << (N1 - RPL);
  const long long total = (long long)tiles_x * ylimbs * items;
  HC_CHECK(total < (1ll << 31), HC_ERR_INVALID, "NTT batch too large");
  const size_t smem = 2 * ((size_t)1 << RPL) * PADW * sizeof(u64);
  auto kern = k_rows_pipe<INV, LOGN, Sp::K1, Sp::K2, RPL, TL>;
  const int grid = pipe_grid(ctx, kern, smem, total);
  ProfScope p(ctx, INV ? "ntt_inv_rows" : "ntt_fwd_rows", (uint64_t)ylimbs * items);
  kern<<<grid, 1 << TL, smem, ctx->stream>>>(s, in ? *in : s, in ? 1 : 0, tiles_x, ylimbs, (int)total, ctx->tab);
}

// variant 0: 256-thread blocks, 1: 128-thread blocks, 2: 64-thread blocks
// (N >= 2^13 only; smaller rings fall back to 128)
template <bool INV, int LOGN>
void launch_pass_cols(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, const LimbSet* in = nullptr,
                      bool scale = true, const KsrFuse* fuse = nullptr) {
  const int v = ctx->tune.ntt_variant[LOGN];
  if constexpr (LOGN >= 13) {
    if (v == 2) return launch_pass_cols_t<INV, LOGN, 6>(ctx, s, items, ylimbs, in, scale, fuse);
  }
  if (v == 1 || v >= 3)
    launch_pass_cols_t<INV, LOGN, 7>(ctx, s, items, ylimbs, in, scale, fuse);
  else
    launch_pass_cols_t<INV, LOGN, 8>(ctx, s, items, ylimbs, in, scale, fuse);
}

template <bool INV, int LOGN>
void launch_pass_rows(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, const LimbSet* in = nullptr,
                      const KsrFuse* fuse = nullptr) {
  const int v = ctx->tune.ntt_variant[LOGN];
  if constexpr (LOGN >= 13) {
    if (v == 2) return launch_pass_rows_t<INV, LOGN, 6>(ctx, s, items, ylimbs, in, fuse);
  }
  if (v == 1 || v >= 3)
    launch_pass_rows_t<INV, LOGN, 7>(ctx, s, items, ylimbs, in, fuse);
  else
    launch_pass_rows_t<INV, LOGN, 8>(ctx, s, items, ylimbs, in, fuse);
}

// ---------------------------------------------------------------------------
// Single-pass transform: one limb of N = CL 2^LQ points held in the shared
// memory of a cluster of CL CTAs (2^LQ = 16384 words, 128 KiB, per CTA), so
// that each limb is read from and written to global memory once.
//
// Forward (stage st: half distance N / 2^{st+1}): the first C = log2 CL
// stages pair points of different CTAs.  CTA r takes the offsets j in
// [r Q / CL, (r+1) Q / CL) of every CTA's chunk (Q = 2^LQ), loads the CL
// points j + k Q straight from global memory, runs stages 0..C-1 on them in
// registers and stores point k into CTA k's shared memory (distributed
// shared memory) at local index j.  After a cluster barrier every CTA holds
// its contiguous chunk [r Q, (r+1) Q), whose remaining LQ stages stay
// inside it: register rounds of 5 or 4 stages between shared-memory
// exchanges, then a coalesced copy to global memory.
// Inverse: the same in reverse: the chunk's LQ stages first, a cluster
// barrier, then stages C-1..0 across the CTAs with distributed-shared-memory
// loads and the results (times N^{-1} unless the caller folds it) written to
// global memory; a last cluster barrier keeps each CTA's shared memory alive
// until the others have read it.  Cluster barriers are hardware barriers
// (no spin loop).  With CL = 1 (N <= 2^14) the chunk is the whole limb.
// Shared-memory words are padded by one per 16 (index i at i + i / 16), so
// the rounds with contiguous points per thread do not conflict on banks.

__device__ __forceinline__ u32 opad(u32 i) { return i + (i >> 4); }

// Local rounds of the chunk's LQ stages, forward order: round i covers
// stages S0(i) .. S0(i) + K(i) - 1.  WIDE = 1: rounds of up to 5 stages (32
// points per thread, three rounds); WIDE = 0: up to 4 (16 points, four).
template <int LQ, int WIDE>
struct OnePassRounds;
template <>
struct OnePassRounds<14, 1> {
  static constexpr int n = 3;
  static constexpr int s0[4] = {0, 5, 10, 14};
  static constexpr int k[4] = {5, 5, 4, 0};
};
template <>
struct OnePassRounds<14, 0> {
  static constexpr int n = 4;
  static constexpr int s0[4] = {0, 4, 8, 11};
  static constexpr int k[4] = {4, 4, 3, 3};
};
template <>
struct OnePassRounds<13, 1> {
  static constexpr int n = 3;
  static constexpr int s0[4] = {0, 5, 9, 13};
  static constexpr int k[4] = {5, 4, 4, 0};
};
template <>
struct OnePassRounds<13, 0> {
  static constexpr int n = 4;
  static constexpr int s0[4] = {0, 4, 7, 10};
  static constexpr int k[4] = {4, 3, 3, 3};
};

// One register round of local stages S0..S0+K-1 over the CTA's chunk in
// shared memory (forward, or inverse in reverse stage order).  Group g of
// 2^K points: local index ((g >> LS) << (LS + K)) + (g & (2^LS - 1)) + (m << LS),
// LS = LQ - S0 - K; its global index adds r 2^LQ.
template <bool INV, int LOGN, int LQ, int TL, int S0, int K>
__device__ __forceinline__ void onepass_round(u64* sm, u32 r, const ulonglong2* tw, u64 q) {
  if constexpr (K > 0) {
    constexpr int C = LOGN - LQ, LS = LQ - S0 - K;
    constexpr u32 kThreads = 1u << TL;
    constexpr u32 kGroups = 1u << (LQ - K);
    static_assert(kGroups % kThreads == 0 || kGroups < kThreads, "groups per thread");
    for (u32 g = threadIdx.x; g < kGroups; g += kThreads) {
      const u32 lo = g & ((1u << LS) - 1), hi = g >> LS;
      const u32 i0 = (hi << (LS + K)) + lo;
      const u32 jb = (r << LQ) + i0;
      u64 x[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) x[m] = sm[opad(i0 + ((u32)m << LS))];
      if constexpr (!INV)
        fwd_block<K, LS, C + S0, LOGN>(x, jb, tw, q);
      else
        inv_block<K, LS, C + S0 + K - 1, LOGN>(x, jb, tw, q);
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) sm[opad(i0 + ((u32)m << LS))] = x[m];
    }
  }
}

template <bool INV, int LOGN, int LQ, int TL, int WIDE>
__device__ __forceinline__ void onepass_local(u64* sm, u32 r, const ulonglong2* tw, u64 q) {
  using R = OnePassRounds<LQ, WIDE>;
  if constexpr (!INV) {
    onepass_round<false, LOGN, LQ, TL, R::s0[0], R::k[0]>(sm, r, tw, q);
    __syncthreads();
    onepass_round<false, LOGN, LQ, TL, R::s0[1], R::k[1]>(sm, r, tw, q);
    __syncthreads();
    onepass_round<false, LOGN, LQ, TL, R::s0[2], R::k[2]>(sm, r, tw, q);
    if constexpr (R::n > 3) {
      __syncthreads();
      onepass_round<false, LOGN, LQ, TL, R::s0[3], R::k[3]>(sm, r, tw, q);
    }
  } else {
    if constexpr (R::n > 3) {
      onepass_round<true, LOGN, LQ, TL, R::s0[3], R::k[3]>(sm, r, tw, q);
      __syncthreads();
    }
    onepass_round<true, LOGN, LQ, TL, R::s0[2], R::k[2]>(sm, r, tw, q);
    __syncthreads();
    onepass_round<true, LOGN, LQ, TL, R::s0[1], R::k[1]>(sm, r, tw, q);
    __syncthreads();
    onepass_round<true, LOGN, LQ, TL, R::s0[0], R::k[0]>(sm, r, tw, q);
  }
}

// Blocks per SM the launch bounds ask for: one 512-thread CTA with a 2^14
// chunk, three 256-thread CTAs with 2^13 chunks (their shared memory fits).
template <int TL>
constexpr int onepass_min_blocks() {
  return TL >= 9 ? 1 : 3;
}

template <bool INV, int LOGN, int LQ, int TL, int WIDE>
__global__ void __launch_bounds__(1u << TL, onepass_min_blocks<TL>())
    k_ntt_onepass(LimbSet s, LimbSet in, int use_in, int scale, Tables T) {
  namespace cg = cooperative_groups;
  constexpr int C = LOGN - LQ, CL = 1 << C, Q = 1 << LQ;
  constexpr u32 kThreads = 1u << TL;
  constexpr u32 kJ = Q / CL;                         // cross-CTA offsets per CTA
  constexpr u32 kJT = CL > 1 ? kJ / kThreads : 1;    // ... per thread
  static_assert(CL == 1 || kJ % kThreads == 0, "cross-CTA offsets per thread");
  extern __shared__ u64 sm[];
  u64* a;
  int pid;
  limb_meta<LOGN>(s, a, pid);
  const u64* ain = use_in ? input_limb<LOGN>(s, in) : a;
  const u64 q = T.mods[pid].q;
  const ulonglong2* tw = (INV ? T.inv2 : T.fwd2) + ((size_t)pid << LOGN);
  const u32 r = CL > 1 ? cg::this_cluster().block_rank() : 0;
  const u64* src = ain + ((size_t)r << LQ);
  u64* dst = a + ((size_t)r << LQ);
  if constexpr (!INV) {
    if constexpr (CL > 1) {
      cg::cluster_group cl = cg::this_cluster();
      // all of this thread's loads first (kJT offsets x CL points in flight)
      u64 x[kJT][CL];
#pragma unroll
      for (u32 v = 0; v < kJT; ++v)
#pragma unroll
        for (int k = 0; k < CL; ++k) x[v][k] = ain[r * kJ + v * kThreads + threadIdx.x + ((u32)k << LQ)];
#pragma unroll
      for (u32 v = 0; v < kJT; ++v) fwd_block<C, LQ, 0, LOGN>(x[v], r * kJ + v * kThreads + threadIdx.x, tw, q);
      cl.sync();  // every CTA of the cluster has started before remote stores
#pragma unroll
      for (int k = 0; k < CL; ++k) {
        u64* peer = cl.map_shared_rank(sm, k);
#pragma unroll
        for (u32 v = 0; v < kJT; ++v) peer[opad(r * kJ + v * kThreads + threadIdx.x)] = x[v][k];
      }
      cl.sync();  // the chunks are complete (remote stores visible)
    } else {
      for (u32 e = threadIdx.x; e < (u32)Q; e += kThreads) sm[opad(e)] = src[e];
      __syncthreads();
    }
    onepass_local<false, LOGN, LQ, TL, WIDE>(sm, r, tw, q);
    __syncthreads();
    for (u32 e = threadIdx.x; e < (u32)Q; e += kThreads) dst[e] = reduce4(sm[opad(e)], q);
  } else {
    for (u32 e = threadIdx.x; e < (u32)Q; e += kThreads) sm[opad(e)] = src[e];
    __syncthreads();
    onepass_local<true, LOGN, LQ, TL, WIDE>(sm, r, tw, q);
    const u64 ni = T.ninv[pid], nis = T.ninv_sh[pid];
    if constexpr (CL > 1) {
      cg::cluster_group cl = cg::this_cluster();
      cl.sync();  // every chunk's local stages are done
      u64 x[kJT][CL];
#pragma unroll
      for (int k = 0; k < CL; ++k) {
        const u64* peer = cl.map_shared_rank(sm, k);
#pragma unroll
        for (u32 v = 0; v < kJT; ++v) x[v][k] = peer[opad(r * kJ + v * kThreads + threadIdx.x)];
      }
      cl.sync();  // all remote reads are done before any CTA of the cluster exits
#pragma unroll
      for (u32 v = 0; v < kJT; ++v) {
        const u32 j = r * kJ + v * kThreads + threadIdx.x;
        inv_block<C, LQ, C - 1, LOGN>(x[v], j, tw, q);
#pragma unroll
        for (int k = 0; k < CL; ++k)
          a[j + ((u32)k << LQ)] = reduce4(scale ? shoup_lazy(x[v][k], ni, nis, q) : x[v][k], q);
      }
    } else {
      __syncthreads();
      for (u32 e = threadIdx.x; e < (u32)Q; e += kThreads) {
        const u64 v = sm[opad(e)];
        dst[e] = reduce4(scale ? shoup_lazy(v, ni, nis, q) : v, q);
      }
    }
  }
}

// Forms: CHUNK14 = 1: chunks of 2^14 words per 512-thread CTA (one per SM;
// clusters of N / 2^14), rounds of up to 5 stages; CHUNK14 = 0: chunks of
// 2^13 words per 256-thread CTA (three per SM; clusters of N / 2^13, at most
// 8), rounds of up to 4 stages.
template <bool INV, int LOGN, int CHUNK14>
void launch_onepass(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, const LimbSet* in, bool scale) {
  constexpr int LQ = (CHUNK14 && LOGN >= 14) ? 14 : 13;
  constexpr int TL = CHUNK14 ? 9 : 8;
  constexpr int WIDE = CHUNK14 ? 1 : 0;
  constexpr int CL = 1 << (LOGN - LQ);
  static_assert(CL <= 8, "portable cluster size");
  const size_t smem = (size_t)((1 << LQ) + (1 << (LQ - 4))) * sizeof(u64);
  auto kern = k_ntt_onepass<INV, LOGN, LQ, TL, WIDE>;
  static unsigned long long attr_set = 0;  // per instantiation, one bit per device
  if (ctx->device >= 64 || !(attr_set >> ctx->device & 1)) {
    HC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ctx->device < 64) attr_set |= 1ull << ctx->device;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)CL, (unsigned)ylimbs, (unsigned)items);
  lc.blockDim = dim3(1u << TL);
  lc.dynamicSmemBytes = smem;
  lc.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  ProfScope p(ctx, INV ? "ntt_inv_onepass" : "ntt_fwd_onepass", (uint64_t)ylimbs * items);
  HC_CUDA(cudaLaunchKernelEx(&lc, kern, s, in ? *in : s, in ? 1 : 0, scale ? 1 : 0, ctx->tab));
}

template <int LOGN>
void ntt_logn(hc_ctx* ctx, const LimbSet& s, int items, int ylimbs, bool inverse, const LimbSet* in, bool scale,
              const KsrFuse* fuse = nullptr) {
  if constexpr (LOGN >= 13) {
    // variants 3 / 4: plain transforms in one pass, rounds of up to 5 / 4
    // stages (the fused-tail transforms stay two-pass, 128-thread tiles)
    const int v = ctx->tune.ntt_variant[LOGN];
    if (!fuse && (v == 3 || v == 4)) {
      if (inverse) {
        if (v == 3) launch_onepass<true, LOGN, 1>(ctx, s, items, ylimbs, in, scale);
        else launch_onepass<true, LOGN, 0>(ctx, s, items, ylimbs, in, scale);
      } else {
        if (v == 3) launch_onepass<false, LOGN, 1>(ctx, s, items, ylimbs, in, scale);
        else launch_onepass<false, LOGN, 0>(ctx, s, items, ylimbs, in, scale);
      }
      ctx->launches -= 1;  // one launch instead of two (the caller counts two)
      return;
    }
  }
  if constexpr (LOGN >= 13) {
    // variant 5: pipelined two-pass transforms (fused-tail ones as variant 1)
    if (!fuse && ctx->tune.ntt_variant[LOGN] == 5) {
      if (!inverse) {
        launch_pass_cols_pipe<false, LOGN>(ctx, s, items, ylimbs, in, true);
        launch_pass_rows_pipe<false, LOGN>(ctx, s, items, ylimbs, nullptr);
      } else {
        launch_pass_rows_pipe<true, LOGN>(ctx, s, items, ylimbs, in);
        launch_pass_cols_pipe<true, LOGN>(ctx, s, items, ylimbs, nullptr, scale);
      }
      return;
    }
  }
  if (!inverse) {
    launch_pass_cols<false, LOGN>(ctx, s, items, ylimbs, in, true, fuse);
    launch_pass_rows<false, LOGN>(ctx, s, items, ylimbs, nullptr, fuse);
  } else {
    launch_pass_rows<true, LOGN>(ctx, s, items, ylimbs, in, fuse);
    launch_pass_cols<true, LOGN>(ctx, s, items, ylimbs, nullptr, scale, fuse);
  }
}

}  // namespace

void launch_ntt(hc_ctx* ctx, const LimbSet& s, int items, bool inverse, bool scale) {
  launch_ntt_from(ctx, s, nullptr, items, inverse, scale);
}

namespace {
void ntt_dispatch(hc_ctx* ctx, const LimbSet& s, const LimbSet* in, int items, bool inverse, bool scale,
                  const KsrFuse* fuse) {
  if (items <= 0 || s.nlimb <= 0 || s.npoly <= 0) return;
  const int ylimbs = s.npoly * s.nlimb;
  HC_CHECK(ylimbs <= 65535 && items <= 65535, HC_ERR_INVALID, "NTT batch too large");
  switch (ctx->P.log_n) {
    case 10: ntt_logn<10>(ctx, s, items, ylimbs, inverse, in, scale, fuse); break;
    case 11: ntt_logn<11>(ctx, s, items, ylimbs, inverse, in, scale, fuse); break;
    case 12: ntt_logn<12>(ctx, s, items, ylimbs, inverse, in, scale, fuse); break;
    case 13: ntt_logn<13>(ctx, s, items, ylimbs, inverse, in, scale, fuse); break;
    case 14: ntt_logn<14>(ctx, s, items, ylimbs, inverse, in, scale, fuse); break;
    case 15: ntt_logn<15>(ctx, s, items, ylimbs, inverse, in, scale, fuse); break;
    case 16: ntt_logn<16>(ctx, s, items, ylimbs, inverse, in, scale, fuse); break;
    default: throw HcError{HC_ERR_INVALID, "unsupported ring degree"};
  }
  ctx->launches += 2;
  check_launch(ctx);
}
}  // namespace

void launch_ntt_from(hc_ctx* ctx, const LimbSet& s, const LimbSet* in, int items, bool inverse, bool scale) {
  ntt_dispatch(ctx, s, in, items, inverse, scale, nullptr);
}

void launch_ntt_ksr(hc_ctx* ctx, const LimbSet& s, int items, const KsrFuse& fuse) {
  HC_CHECK(s.npoly == 2 && s.l0 == 0 && !s.prime_map && !s.slot_map && !s.refs, HC_ERR_INVALID,
           "fused tail needs plain z limbs");
  ntt_dispatch(ctx, s, nullptr, items, false, true, &fuse);
}

void launch_intt_ksr(hc_ctx* ctx, const LimbSet& out, int items, const KsrFuse& fuse) {
  HC_CHECK(out.npoly == 2 && out.l0 == 0 && !out.prime_map && !out.slot_map && !out.refs && fuse.z &&
               fuse.nqlinv,
           HC_ERR_INVALID, "coefficient-form tail needs plain output limbs and its constants");
  ntt_dispatch(ctx, out, nullptr, items, true, true, &fuse);
}
