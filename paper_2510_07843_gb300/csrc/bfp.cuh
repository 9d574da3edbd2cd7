// Block-floating-point fronthaul blocks: one per (cell, symbol, antenna, PRB), 1 + 3w bytes: a
// parameter byte whose low four bits are the exponent e, then the PRB's 24 values I0 Q0 I1 Q1 ...
// as w-bit two's-complement mantissas (1 <= w <= 16), most significant bit first; the value is
// m 2^e scale. Unpacking helpers shared by the decompressor and the fused LS estimator.
#pragma once

#include "common.cuh"

namespace phy {

// Mantissa i of a block, from bytes that may be read up to two past the bit field (staged copy).
__device__ __forceinline__ int bfp_mantissa_padded(const uint8_t* b, int w, int i) {
  const int o = 8 + i * w;  // bit offset from the block start
  const int by = o >> 3;
  const uint32_t win = ((uint32_t)b[by] << 16) | ((uint32_t)b[by + 1] << 8) | (uint32_t)b[by + 2];
  const uint32_t m = (win >> (24 - (o & 7) - w)) & ((1u << w) - 1u);
  const int sign = 1 << (w - 1);
  return ((int)m ^ sign) - sign;
}

// The same from global memory without reading past the bytes that hold the field.
__device__ __forceinline__ int bfp_mantissa_exact(const uint8_t* b, int w, int i) {
  const int o = 8 + i * w;
  const int by = o >> 3, last = (o + w - 1) >> 3;
  uint32_t win = (uint32_t)__ldg(b + by) << 16;
  if (last > by) win |= (uint32_t)__ldg(b + by + 1) << 8;
  if (last > by + 1) win |= (uint32_t)__ldg(b + by + 2);
  const uint32_t m = (win >> (24 - (o & 7) - w)) & ((1u << w) - 1u);
  const int sign = 1 << (w - 1);
  return ((int)m ^ sign) - sign;
}

// m 2^e scale: m 2^e is exact in FP32 (|m| < 2^15, e <= 15), so the product rounds once.
__device__ __forceinline__ float bfp_value(int m, float p2, float scale) {
  return ((float)m * p2) * scale;
}

// Subcarrier k of grid row (cell, t, r), read straight from the compressed stream.
__device__ __forceinline__ cf bfp_load_re(const Geo& g, const uint8_t* yc, int w, float scale,
                                          int cell, int t, int r, int k) {
  const int nb = 1 + 3 * w, n_prb = g.n_sc / 12;
  const uint8_t* blk =
      yc + ((((size_t)cell * g.n_sym + t) * g.n_rx + r) * n_prb + k / 12) * (size_t)nb;
  const float p2 = (float)(1 << (__ldg(blk) & 0xF));
  const int j = 2 * (k % 12);
  return mk(bfp_value(bfp_mantissa_exact(blk, w, j), p2, scale),
            bfp_value(bfp_mantissa_exact(blk, w, j + 1), p2, scale));
}

}  // namespace phy
