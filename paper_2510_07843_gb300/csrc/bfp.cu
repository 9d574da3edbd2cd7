// Block-floating-point fronthaul decompression: the received grid as it arrives over a split-7
// fronthaul at the software DU the paper targets (the paper prints no format; this is the
// library's reading, the usual shared-exponent block format).
//
// Yc holds one block per (cell, symbol, antenna, PRB), in that order, of 1 + 3w bytes: a parameter
// byte whose low four bits are the exponent e, then the PRB's 24 values I0 Q0 I1 Q1 ... as w-bit
// two's-complement mantissas (1 <= w <= 16), most significant bit first. Value = m 2^e scale.
// Because the blocks follow the grid's own order, block b expands to the 12 complex values
// Y[12 b .. 12 b + 12) of the flat grid: decompression is one linear stream.
//
// The block format and the unpacking helpers are in bfp.cuh.
//
// bfp_decompress_kernel: each warp takes 32 consecutive blocks; its byte range is staged in
// shared memory with coalesced 32-bit loads, each lane unpacks one block into a shared output
// tile, and the warp writes the 32 x 96 contiguous bytes with 16-byte stores. With data_only the
// DMRS symbols are skipped (the fused estimator below reads them from Yc itself).
#include <algorithm>

#include "bfp.cuh"
#include "launch.h"

namespace phy {

namespace {

constexpr int kBfpThreads = 256;
constexpr int kBfpWarps = kBfpThreads / 32;
constexpr int kBfpMaxBlock = 1 + 3 * 16;                  // bytes of a 16-bit block
constexpr int kBfpInWords = (32 * kBfpMaxBlock) / 4 + 4;  // range + misalignment + window slack

__device__ __forceinline__ bool is_dmrs_sym(const Geo& g, int t) {
  return t == g.dmrs0 || (g.n_dmrs == 2 && t == g.dmrs1);
}

__global__ void __launch_bounds__(kBfpThreads)
    bfp_decompress_kernel(Geo g, const uint8_t* __restrict__ yc, long long n_blocks,
                          long long total_bytes, int w, float scale, int data_only,
                          float* __restrict__ Y) {
  __shared__ uint32_t s_in[kBfpWarps][kBfpInWords];
  __shared__ float s_out[kBfpWarps][32 * 24];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = 1 + 3 * w;
  const long long per_sym = (long long)g.n_rx * (g.n_sc / 12);  // blocks per (cell, symbol)
  const uint8_t* in8 = reinterpret_cast<const uint8_t*>(s_in[warp]);
  const long long stride = (long long)gridDim.x * kBfpWarps * 32;
  for (long long b0 = ((long long)blockIdx.x * kBfpWarps + warp) * 32; b0 < n_blocks;
       b0 += stride) {
    const long long b = b0 + lane;
    const bool live =
        b < n_blocks && !(data_only && is_dmrs_sym(g, (int)((b / per_sym) % g.n_sym)));
    if (!__any_sync(0xffffffffu, live)) continue;
    // ---- stage the warp's byte range [b0 nb, b_end nb) as whole 32-bit words
    const long long b_end = min(b0 + 32, n_blocks);
    const long long w0 = (b0 * nb) >> 2, w1 = (b_end * nb + 3) >> 2;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(yc);
    for (long long k = w0 + lane; k < w1; k += 32) {
      uint32_t v;
      if (4 * k + 4 <= total_bytes) {
        v = __ldg(src + k);
      } else {  // the stream's last partial word, byte by byte (little-endian word order)
        v = 0;
        for (int j = 0; j < 4; ++j)
          if (4 * k + j < total_bytes) v |= (uint32_t)__ldg(yc + 4 * k + j) << (8 * j);
      }
      s_in[warp][k - w0] = v;
    }
    __syncwarp();
    // ---- unpack one block per lane
    if (live) {
      const uint8_t* blk = in8 + (b * nb - 4 * w0);
      const float p2 = (float)(1 << (blk[0] & 0xF));
      float* o = &s_out[warp][lane * 24];
#pragma unroll 4
      for (int i = 0; i < 24; ++i) o[i] = bfp_value(bfp_mantissa_padded(blk, w, i), p2, scale);
    }
    __syncwarp();
    // ---- 96 contiguous bytes per block, 16-byte stores over the warp's blocks
    const int nv = (int)(b_end - b0);
    for (int f = lane; f < 6 * nv; f += 32) {
      const int bi = f / 6;
      const long long bb = b0 + bi;
      if (data_only && is_dmrs_sym(g, (int)((bb / per_sym) % g.n_sym))) continue;
      const float4 v = *reinterpret_cast<const float4*>(&s_out[warp][bi * 24 + (f % 6) * 4]);
      *reinterpret_cast<float4*>(Y + bb * 24 + (f % 6) * 4) = v;
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_bfp_decompress(const Geo& g, const uint8_t* yc, int w, float scale,
                                  int data_only, phy_c32* Y, cudaStream_t st) {
  const long long n_blocks = (long long)g.n_cells * g.n_sym * g.n_rx * (g.n_sc / 12);
  const long long total = n_blocks * (1 + 3 * w);
  const long long warps = (n_blocks + 31) / 32;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long want = (warps + kBfpWarps - 1) / kBfpWarps;
  const int grid = (int)std::min<long long>(want, (long long)sms * 8);
  bfp_decompress_kernel<<<grid, kBfpThreads, 0, st>>>(g, yc, n_blocks, total, w, scale,
                                                      data_only, reinterpret_cast<float*>(Y));
  return cudaGetLastError();
}

}  // namespace phy
