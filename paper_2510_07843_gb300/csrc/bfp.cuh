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

// m 2^e scale: m 2^e is exact in FP32 (|m| < 2^15, e <= 15), so the product rounds once.
__device__ __forceinline__ float bfp_value(int m, float p2, float scale) {
  return ((float)m * p2) * scale;
}

}  // namespace phy
