// Throughput of the integer-multiply forms used by the modular arithmetic,
// in thread-operations per SM per clock, on the GPU it runs on.  Each thread
// runs four independent chains so that the pipes, not latencies, limit.
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 intmul_throughput.cu -o intmul && ./intmul
// The 64-bit forms are what Shoup's product costs: two low products and
// one high product per butterfly.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

typedef unsigned long long u64;
constexpr int kIters = 4096;

template <int KIND>
__global__ void chains(u64* out, u64 c, u64 d) {
  u64 x0 = threadIdx.x + 1, x1 = x0 * 3, x2 = x0 * 5, x3 = x0 * 7;
  uint32_t a0 = (uint32_t)x0, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  const uint32_t cc = (uint32_t)c, dd = (uint32_t)d;
#pragma unroll 8
  for (int i = 0; i < kIters; ++i) {
    if (KIND == 0) {  // 32-bit multiply-add
      a0 = a0 * cc + dd; a1 = a1 * cc + dd; a2 = a2 * cc + dd; a3 = a3 * cc + dd;
    } else if (KIND == 1) {  // 32-bit high half
      a0 += __umulhi(a0, cc); a1 += __umulhi(a1, cc); a2 += __umulhi(a2, cc); a3 += __umulhi(a3, cc);
    } else if (KIND == 2) {  // 32 x 32 -> 64 multiply-add
      x0 += (u64)a0 * cc; x1 += (u64)a1 * cc; x2 += (u64)a2 * cc; x3 += (u64)a3 * cc;
      a0 ^= (uint32_t)x0; a1 ^= (uint32_t)x1; a2 ^= (uint32_t)x2; a3 ^= (uint32_t)x3;
    } else if (KIND == 3) {  // 64-bit low product
      x0 = x0 * c + d; x1 = x1 * c + d; x2 = x2 * c + d; x3 = x3 * c + d;
    } else if (KIND == 4) {  // 64-bit high product
      x0 += __umul64hi(x0, c); x1 += __umul64hi(x1, c); x2 += __umul64hi(x2, c); x3 += __umul64hi(x3, c);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 ^ x1 ^ x2 ^ x3 ^ a0 ^ a1 ^ a2 ^ a3;
}

template <int KIND>
double rate(u64* out, int blocks, int threads, int sms, int khz) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  chains<KIND><<<blocks, threads>>>(out, 0x9e3779b97f4a7c15ull, 12345);
  cudaEventRecord(e0);
  chains<KIND><<<blocks, threads>>>(out, 0x9e3779b97f4a7c15ull, 12345);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double ops = (double)blocks * threads * kIters * 4;
  return ops / (ms * 1e-3) / sms / (khz * 1e3);
}

int main() {
  int sms = 0, khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0);
  const int threads = 256, blocks = sms * 8;
  u64* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(u64)) != cudaSuccess) return 1;
  printf("SMs %d, clock attribute %d MHz; ops per SM per clock:\n", sms, khz / 1000);
  const double r0 = rate<0>(out, blocks, threads, sms, khz), r1 = rate<1>(out, blocks, threads, sms, khz),
               r2 = rate<2>(out, blocks, threads, sms, khz), r3 = rate<3>(out, blocks, threads, sms, khz),
               r4 = rate<4>(out, blocks, threads, sms, khz);
  printf("  32-bit multiply-add          %6.1f\n", r0);
  printf("  32-bit high half (+ add)     %6.1f\n", r1);
  printf("  32x32->64 multiply-add (+xor) %5.1f\n", r2);
  printf("  64-bit low product (+ add)   %6.1f\n", r3);
  printf("  64-bit high product (+ add)  %6.1f\n", r4);
  printf("Shoup product in 32-bit multiply-add slots: 2 x %.2f + %.2f = %.2f\n", r0 / r3, r0 / r4,
         2 * r0 / r3 + r0 / r4);
  const cudaError_t e = cudaGetLastError();
  cudaFree(out);
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
