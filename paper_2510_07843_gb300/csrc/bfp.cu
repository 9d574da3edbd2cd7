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
// The block format and the byte-wise unpacking helpers are in bfp.cuh.
//
// bfp_decompress_kernel: one wave of CTAs striding over the stream; each warp takes 32
// consecutive blocks per iteration: their byte range arrives as coalesced 32-bit loads into
// registers (issued one iteration ahead, so they are in flight while the previous blocks are
// unpacked), is staged in shared memory, each lane unpacks one block into a padded [value][block]
// tile, and the warp writes the 32 x 96 contiguous bytes with 16-byte stores. With data_only the
// DMRS symbols' rows are not written (the fused LS estimator reads them from Yc itself).
#include <algorithm>

#include "bfp.cuh"
#include "launch.h"

namespace phy {

namespace {

constexpr int kBfpThreads = 256;
constexpr int kBfpWarps = kBfpThreads / 32;
constexpr int kBfpMaxBlock = 1 + 3 * 16;                  // bytes of a 16-bit block
constexpr int kBfpInWords = (32 * kBfpMaxBlock) / 4 + 4;  // range + misalignment + window slack
constexpr int kBfpPre = (kBfpInWords + 31) / 32;          // staged words per lane

__device__ __forceinline__ bool is_dmrs_sym(const Geo& g, int t) {
  return t == g.dmrs0 || (g.n_dmrs == 2 && t == g.dmrs1);
}

// One warp-iteration's input: the 32-bit words [w0, w1) of the stream, lane-strided.
__device__ __forceinline__ void bfp_fetch(const uint8_t* __restrict__ yc, long long total_bytes,
                                          long long w0, long long w1, int lane,
                                          uint32_t (&pre)[kBfpPre]) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(yc);
#pragma unroll
  for (int j = 0; j < kBfpPre; ++j) {
    const long long k = w0 + lane + 32 * j;
    uint32_t v = 0;
    if (k < w1) {
      if (4 * k + 4 <= total_bytes) {
        v = __ldg(src + k);
      } else {  // the stream's last partial word, byte by byte (little-endian word order)
        for (int q = 0; q < 4; ++q)
          if (4 * k + q < total_bytes) v |= (uint32_t)__ldg(yc + 4 * k + q) << (8 * q);
      }
    }
    pre[j] = v;
  }
}

// Unpacks the block whose parameter byte is staged byte B0 into out[.][lane]. With the width W
// known at compile time the block is first re-aligned into big-endian 32-bit words v_j (bytes
// B0 + 4j ..), then every mantissa is one funnel shift of a word pair and one arithmetic shift,
// which also sign-extends it. W = 0 selects the byte-wise path for the run-time width w.
template <int W>
__device__ __forceinline__ void bfp_unpack(const uint32_t* s, int B0, int w, float scale,
                                           float (*out)[33], int lane) {
  if constexpr (W == 0) {
    const uint8_t* blk = reinterpret_cast<const uint8_t*>(s) + B0;
    const float p2 = (float)(1 << (blk[0] & 0xF));
#pragma unroll 4
    for (int i = 0; i < 24; ++i)
      out[i][lane] = bfp_value(bfp_mantissa_padded(blk, w, i), p2, scale);
  } else {
    constexpr int kBits = 8 * (1 + 3 * W);
    constexpr int kV = ((kBits - 1) >> 5) + 2;  // aligned words, one spare for the funnel
    const int c = B0 & 3;
    const uint32_t sel = (c << 12) | ((c + 1) << 8) | ((c + 2) << 4) | (c + 3);
    const uint32_t* base = s + (B0 >> 2);
    uint32_t v[kV];
    uint32_t lo = base[0];
#pragma unroll
    for (int j = 0; j < kV; ++j) {
      const uint32_t hi = base[j + 1];
      v[j] = __byte_perm(lo, hi, sel);  // bytes B0+4j .. B0+4j+3, the first most significant
      lo = hi;
    }
    const float p2 = (float)(1 << ((v[0] >> 24) & 0xF));
#pragma unroll
    for (int i = 0; i < 24; ++i) {
      const int o = 8 + i * W;  // bit offset in the block, a constant after unrolling
      const uint32_t f = __funnelshift_l(v[(o >> 5) + 1], v[o >> 5], o & 31);
      out[i][lane] = bfp_value((int)f >> (32 - W), p2, scale);  // top W bits, sign-extended
    }
  }
}

template <int W>
__global__ void __launch_bounds__(kBfpThreads)
    bfp_decompress_kernel(Geo g, const uint8_t* __restrict__ yc, long long n_blocks,
                          long long total_bytes, int w, float scale, int data_only,
                          float* __restrict__ Y) {
  __shared__ uint32_t s_in[kBfpWarps][kBfpPre * 32];
  __shared__ float s_out[kBfpWarps][24][33];  // [value][block], padded: conflict-free both ways
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = 1 + 3 * (W ? W : w);
  const long long per_sym = (long long)g.n_rx * (g.n_sc / 12);  // blocks per (cell, symbol)
  const long long stride = (long long)gridDim.x * kBfpWarps * 32;
  long long b0 = ((long long)blockIdx.x * kBfpWarps + warp) * 32;
  uint32_t pre[kBfpPre];
  if (b0 < n_blocks)
    bfp_fetch(yc, total_bytes, (b0 * nb) >> 2, (min(b0 + 32, n_blocks) * nb + 3) >> 2, lane, pre);
  for (; b0 < n_blocks; b0 += stride) {
    const long long b_end = min(b0 + 32, n_blocks);
    const long long w0 = (b0 * nb) >> 2;
    // ---- stage this iteration's words, then start the next iteration's loads
#pragma unroll
    for (int j = 0; j < kBfpPre; ++j) s_in[warp][lane + 32 * j] = pre[j];
    __syncwarp();
    const long long n0 = b0 + stride;
    if (n0 < n_blocks)
      bfp_fetch(yc, total_bytes, (n0 * nb) >> 2, (min(n0 + 32, n_blocks) * nb + 3) >> 2, lane,
                pre);
    // ---- which of the warp's blocks to write (one division per lane)
    const long long b = b0 + lane;
    const bool dm = data_only && b < b_end && is_dmrs_sym(g, (int)((b / per_sym) % g.n_sym));
    const unsigned skip = __ballot_sync(0xffffffffu, dm);
    const bool live = b < b_end && !dm;
    if (__any_sync(0xffffffffu, live)) {
      // ---- unpack one block per lane
      if (live) bfp_unpack<W>(s_in[warp], (int)(b * nb - 4 * w0), w, scale, s_out[warp], lane);
      __syncwarp();
      // ---- 96 contiguous bytes per block, 16-byte stores over the warp's blocks
      const int nv = (int)(b_end - b0);
      for (int f = lane; f < 6 * nv; f += 32) {
        const int bi = f / 6, v0 = (f % 6) * 4;
        if ((skip >> bi) & 1u) continue;
        const float4 v = make_float4(s_out[warp][v0][bi], s_out[warp][v0 + 1][bi],
                                     s_out[warp][v0 + 2][bi], s_out[warp][v0 + 3][bi]);
        *reinterpret_cast<float4*>(Y + (b0 + bi) * 24 + v0) = v;
      }
    }
    __syncwarp();
  }
}

template <int W>
cudaError_t launch_w(const Geo& g, const uint8_t* yc, long long n_blocks, long long total, int w,
                     float scale, int data_only, phy_c32* Y, int sms, cudaStream_t st) {
  // one wave: as many CTAs as fit on the SMs at once, each striding over the stream
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, bfp_decompress_kernel<W>, kBfpThreads, 0);
  if (e != cudaSuccess) return e;
  const long long want = (n_blocks + 32 * kBfpWarps - 1) / (32 * kBfpWarps);
  const int grid =
      (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * std::max(per_sm, 1)));
  bfp_decompress_kernel<W><<<grid, kBfpThreads, 0, st>>>(g, yc, n_blocks, total, w, scale,
                                                         data_only, reinterpret_cast<float*>(Y));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bfp_decompress(const Geo& g, const uint8_t* yc, int w, float scale,
                                  int data_only, phy_c32* Y, cudaStream_t st) {
  const long long n_blocks = (long long)g.n_cells * g.n_sym * g.n_rx * (g.n_sc / 12);
  const long long total = n_blocks * (1 + 3 * w);
  const int sms = device_sm_count();
  switch (w) {  // the usual fronthaul widths get compile-time bit offsets
    case 8: return launch_w<8>(g, yc, n_blocks, total, w, scale, data_only, Y, sms, st);
    case 9: return launch_w<9>(g, yc, n_blocks, total, w, scale, data_only, Y, sms, st);
    case 12: return launch_w<12>(g, yc, n_blocks, total, w, scale, data_only, Y, sms, st);
    case 14: return launch_w<14>(g, yc, n_blocks, total, w, scale, data_only, Y, sms, st);
    case 16: return launch_w<16>(g, yc, n_blocks, total, w, scale, data_only, Y, sms, st);
    default: return launch_w<0>(g, yc, n_blocks, total, w, scale, data_only, Y, sms, st);
  }
}

}  // namespace phy
