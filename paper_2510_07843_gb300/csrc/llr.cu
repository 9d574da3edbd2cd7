// Stand-alone max-log demapper: LLRs from equalised symbols and their SINR.
// One thread per (RE, layer). With SINR = mu / e and mu + e = 1: mu = SINR / (1 + SINR), the
// unbiased symbol is x_hat / mu and the effective noise 1 / SINR.
#include "launch.h"

namespace phy {

namespace {

template <int QM>
__global__ void __launch_bounds__(256) llr_kernel(size_t n, const phy_c32* __restrict__ x_hat,
                                                  const float* __restrict__ sinr,
                                                  float* __restrict__ llr, bool f16) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cf x = ld(x_hat + i);
  const float s = sinr[i];
  float out[QM];
  if (s > 0.f && s < 3.0e38f) {
    const float mu = s / (1.f + s);
    const float im = 1.f / mu;
    qam_llr<QM>(im * x, 1.f / s, out);
  } else {
#pragma unroll
    for (int q = 0; q < QM; ++q) out[q] = 0.f;
  }
#pragma unroll
  for (int q = 0; q < QM; q += 2) store_llr_pair(llr, i * QM + q, out[q], out[q + 1], f16);
}

}  // namespace

cudaError_t launch_llr(const Geo& g, const phy_c32* x_hat, const float* sinr, float* llr,
                       cudaStream_t st) {
  const size_t n = (size_t)g.n_cells * g.n_dsym * g.n_sc * g.n_layers;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  switch (g.qm) {
    case 2: llr_kernel<2><<<blocks, threads, 0, st>>>(n, x_hat, sinr, llr, g.llr_f16); break;
    case 4: llr_kernel<4><<<blocks, threads, 0, st>>>(n, x_hat, sinr, llr, g.llr_f16); break;
    case 6: llr_kernel<6><<<blocks, threads, 0, st>>>(n, x_hat, sinr, llr, g.llr_f16); break;
    default: llr_kernel<8><<<blocks, threads, 0, st>>>(n, x_hat, sinr, llr, g.llr_f16); break;
  }
  return cudaGetLastError();
}

}  // namespace phy
