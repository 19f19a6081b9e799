// Throughput of the integer-multiply forms that the modular arithmetic is
// built from, and of its units of work (hc_int_mul_rates), measured on the
// context's GPU.  The roofline of the multiplication-dense kernels (NTT
// butterflies: two 64-bit low products and one high product each; the
// tensor accumulation: one low and one high product per 64 x 64 -> 128
// multiply-add) is derived from these rates.  Every thread runs four independent dependency chains so
// that the issue rate of the multiplier, not the chains' latency, limits.
#include "hc_internal.h"

namespace {

constexpr int kProbeIters = 4096;
constexpr int kProbeForms = 9;

template <int KIND>
__global__ void k_probe_chains(u64* out, u64 c, u64 d) {
  u64 x0 = threadIdx.x + 1, x1 = x0 * 3, x2 = x0 * 5, x3 = x0 * 7;
  u32 a0 = (u32)x0, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  const u32 cc = (u32)c, dd = (u32)d;
  // constants outside the timed loop's body: w = c mod d (forms 6, 7) or
  // 2^64 mod d (form 8) with its Shoup companion, floor(2^64 / d) (form 8)
  const unsigned __int128 two64 = (unsigned __int128)1 << 64;
  const u64 w = KIND == 8 ? (u64)(two64 % d) : (KIND >= 6 ? c % d : 0);
  const u64 wsh = KIND >= 6 ? (u64)(((unsigned __int128)w << 64) / d) : 0;
  const u64 onesh = KIND == 8 ? (u64)(two64 / d) : 0;
  const u64 q2 = 2 * d;
#pragma unroll 8
  for (int i = 0; i < kProbeIters; ++i) {
    if constexpr (KIND == 0) {  // 32-bit multiply-add
      a0 = a0 * cc + dd;
      a1 = a1 * cc + dd;
      a2 = a2 * cc + dd;
      a3 = a3 * cc + dd;
    } else if constexpr (KIND == 1) {  // high half of a 32 x 32 product, accumulated
      a0 += __umulhi(a0, cc);
      a1 += __umulhi(a1, cc);
      a2 += __umulhi(a2, cc);
      a3 += __umulhi(a3, cc);
    } else if constexpr (KIND == 2) {  // 32 x 32 -> 64 multiply-add
      x0 += (u64)a0 * cc;
      x1 += (u64)a1 * cc;
      x2 += (u64)a2 * cc;
      x3 += (u64)a3 * cc;
      a0 ^= (u32)x0;
      a1 ^= (u32)x1;
      a2 ^= (u32)x2;
      a3 ^= (u32)x3;
    } else if constexpr (KIND == 3) {  // low 64 bits of a 64 x 64 product, plus an add
      x0 = x0 * c + d;
      x1 = x1 * c + d;
      x2 = x2 * c + d;
      x3 = x3 * c + d;
    } else if constexpr (KIND == 4) {  // high 64 bits of a 64 x 64 product, accumulated
      x0 += __umul64hi(x0, c);
      x1 += __umul64hi(x1, c);
      x2 += __umul64hi(x2, c);
      x3 += __umul64hi(x3, c);
    } else if constexpr (KIND == 5) {  // 64 x 64 -> 128 multiply-accumulate with carry (the tensor sums' step)
      U128 s0{x0, 0}, s1{x1, 0}, s2{x2, 0}, s3{x3, 0};
      mac(s0, s0.lo, c);
      mac(s1, s1.lo, c);
      mac(s2, s2.lo, c);
      mac(s3, s3.lo, c);
      x0 = s0.lo ^ s0.hi;
      x1 = s1.lo ^ s1.hi;
      x2 = s2.lo ^ s2.hi;
      x3 = s3.lo ^ s3.hi;
    } else if constexpr (KIND == 6) {  // lazy Shoup product by a constant (q = d, w = c mod q)
      x0 = shoup_lazy(x0, w, wsh, d);
      x1 = shoup_lazy(x1, w, wsh, d);
      x2 = shoup_lazy(x2, w, wsh, d);
      x3 = shoup_lazy(x3, w, wsh, d);
    } else if constexpr (KIND == 8) {
      // the epilogue a split-integer tensor-core basis conversion would need
      // per output residue: 15 fp32 partial sums (exact integers below 2^22,
      // here from a linear congruential sequence, as a fused kernel would
      // hold them on chip), converted to integers, assembled as
      // sum_s P_s 2^{8 s} in 128 bits and reduced modulo q (= d)
      u64 r[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        U128 y{0, 0};
        u32 st = a0 + 977u * (u32)k + (u32)i;
#pragma unroll
        for (int sft = 0; sft < 15; ++sft) {
          st = st * 1664525u + 1013904223u;
          const u64 v = (u64)__float2uint_rz((float)(st >> 10));
          const int sh = 8 * sft;
          if (sh < 64) {
            const u64 lo = v << sh, hi = sh ? (v >> (64 - sh)) : 0;
            const u64 t = y.lo + lo;
            y.hi += hi + (t < lo);
            y.lo = t;
          } else {
            y.hi += v << (sh - 64);
          }
        }
        const u64 t = shoup_lazy(y.hi & ((1ull << 62) - 1), w, wsh, d);
        u64 z = t + (y.lo - __umul64hi(y.lo, onesh) * d);
        z = z >= 2 * d ? z - 2 * d : z;
        r[k] = z >= d ? z - d : z;
      }
      x0 ^= r[0];
      x1 ^= r[1];
      x2 ^= r[2];
      x3 ^= r[3];
      a0 ^= (u32)r[0];
    } else {  // Harvey's lazy Cooley-Tukey butterfly on two pairs (the NTT's unit of work)
      u64 X = x0 >= q2 ? x0 - q2 : x0, T = shoup_lazy(x1, w, wsh, d);
      x0 = X + T;
      x1 = X - T + q2;
      X = x2 >= q2 ? x2 - q2 : x2;
      T = shoup_lazy(x3, w, wsh, d);
      x2 = X + T;
      x3 = X - T + q2;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 ^ x1 ^ x2 ^ x3 ^ a0 ^ a1 ^ a2 ^ a3;
}

// The multiplier is 0x9e3779b97f4a7c15; the Shoup and butterfly forms use
// the 50-bit prime 2^50 - 2^17 + 1 as their modulus (the chains' values stay
// below 2^64 and the results are discarded: only the instruction stream
// matters).
template <int KIND>
double probe_ops_per_s(hc_ctx* ctx, u64* out, int blocks, int threads, cudaEvent_t e0, cudaEvent_t e1) {
  const u64 c = 0x9e3779b97f4a7c15ull, d = KIND >= 6 ? (1ull << 50) - (1ull << 17) + 1 : 12345;
  k_probe_chains<KIND><<<blocks, threads, 0, ctx->stream>>>(out, c, d);  // warm-up
  HC_CUDA(cudaEventRecord(e0, ctx->stream));
  k_probe_chains<KIND><<<blocks, threads, 0, ctx->stream>>>(out, c, d);
  HC_CUDA(cudaEventRecord(e1, ctx->stream));
  HC_CUDA(cudaEventSynchronize(e1));
  ctx->launches += 2;
  float ms = 0;
  HC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  return (double)blocks * threads * kProbeIters * 4 / (ms * 1e-3);
}

}  // namespace

extern "C" int hc_int_mul_rates(hc_ctx* ctx, double* rates, int cap) {
  if (!ctx) return HC_ERR_INVALID;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  try {
    HC_CHECK(rates && cap >= 2 * kProbeForms, HC_ERR_INVALID, "rates needs 18 entries");
    int sms = 0, khz = 0;
    HC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    HC_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device));
    const int threads = 256, blocks = sms * 8;
    BufPtr buf = ctx->buffer((size_t)blocks * threads);
    HC_CUDA(cudaEventCreate(&e0));
    HC_CUDA(cudaEventCreate(&e1));
    double r[kProbeForms];
    r[0] = probe_ops_per_s<0>(ctx, buf->ptr, blocks, threads, e0, e1);
    r[1] = probe_ops_per_s<1>(ctx, buf->ptr, blocks, threads, e0, e1);
    r[2] = probe_ops_per_s<2>(ctx, buf->ptr, blocks, threads, e0, e1);
    r[3] = probe_ops_per_s<3>(ctx, buf->ptr, blocks, threads, e0, e1);
    r[4] = probe_ops_per_s<4>(ctx, buf->ptr, blocks, threads, e0, e1);
    r[5] = probe_ops_per_s<5>(ctx, buf->ptr, blocks, threads, e0, e1);
    r[6] = probe_ops_per_s<6>(ctx, buf->ptr, blocks, threads, e0, e1);
    r[7] = probe_ops_per_s<7>(ctx, buf->ptr, blocks, threads, e0, e1) / 2;  // two butterflies per chain step
    r[8] = probe_ops_per_s<8>(ctx, buf->ptr, blocks, threads, e0, e1);      // four output residues per step
    HC_CUDA(cudaGetLastError());
    for (int i = 0; i < kProbeForms; ++i) {
      rates[i] = r[i] / sms / (khz * 1e3);  // per SM per clock at the device's maximum clock
      rates[kProbeForms + i] = r[i];        // thread-operations per second
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->err.clear();
    return HC_OK;
  } catch (const HcError& e) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctx->err = e.msg;
    return e.code;
  }
}
