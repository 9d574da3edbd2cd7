// FMA throughput probe: the measured arithmetic peak that the ALU-bound kernels' roofline
// fractions are reported against (measurement support; the paper has no counterpart).
//
// Every thread runs kChains independent multiply-add chains, kUnroll rounds per loop trip, so
// that with a full SM (8 CTAs of 256 threads) the FMA pipes, not dependency latency, bound the
// rate. The chains stay bounded (a <- a m + c with m just above 1); block 0 stores its sums so
// that nothing is dead code.
#include "../../include/phy.h"
#include "launch.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 32;

template <class T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters, T* __restrict__ sink) {
  T a[kChains];
  const T m = (T)1.0000001, c = (T)1e-7;
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (blockIdx.x == 0) sink[threadIdx.x] = s;
}

// Packed pairs: one fma.rn.f32x2 does two FP32 multiply-adds on a 64-bit register pair.
__global__ void __launch_bounds__(kProbeThreads)
    fma2_probe_kernel(int iters, float* __restrict__ sink) {
  unsigned long long a[kChains];
  const float m = 1.0000001f, c = 1e-7f;
  unsigned long long mm, cc;
  asm("mov.b64 %0, {%1, %2};" : "=l"(mm) : "f"(m), "f"(m));
  asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(c), "f"(c));
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    const float x = (float)(threadIdx.x + i) * 1e-3f, y = x + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(x), "f"(y));
  }
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(mm), "l"(cc));
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[i]));
    s += x + y;
  }
  if (blockIdx.x == 0) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" phy_status phy_fma_probe(int32_t kind, int32_t blocks, int32_t iters, void* sink,
                                    double* flops_out, void* stream) {
  if (kind < PHY_PROBE_FP32 || kind > PHY_PROBE_FP64 || blocks < 1 || iters < 1 || !sink)
    return PHY_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double per_thread = (double)iters * kUnroll * kChains * 2.0;
  switch (kind) {
    case PHY_PROBE_FP32:
      fma_probe_kernel<float><<<blocks, kProbeThreads, 0, st>>>(iters, (float*)sink);
      break;
    case PHY_PROBE_FP32X2:
      fma2_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, (float*)sink);
      per_thread *= 2.0;
      break;
    default:
      fma_probe_kernel<double><<<blocks, kProbeThreads, 0, st>>>(iters, (double*)sink);
      break;
  }
  if (flops_out) *flops_out = per_thread * kProbeThreads * (double)blocks;
  return cudaGetLastError() == cudaSuccess ? PHY_OK : PHY_ERR_CUDA;
}
