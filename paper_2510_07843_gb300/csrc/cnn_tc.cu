// Learned denoiser forward pass on the tcgen05 tensor cores: BF16 operands, FP32 accumulation.
//
// A 3x3 convolution is a sum over the nine taps of a (positions x C_in) by (C_in x C_out)
// product in which tap (di, dj) reads the input at the position shifted by (di, dj). The
// activations of a group of four 12 x 14 tiles live in shared memory as one matrix, rows =
// positions of the zero-padded 14 x 16 tiles (so that a shift never wraps into another row or
// tile, and reads zeros outside the tile), columns = channels, stored K-major in core matrices
// of 8 rows x 16 bytes with consecutive rows 16 bytes apart. A shift by s rows is then just a
// descriptor start 16 s bytes further on: each tap's operand is read in place by the MMA, with
// no im2col copy. For every 128-row M tile the nine taps (times C_in / 16 K steps) accumulate
// into one TMEM accumulator of C_out columns; the four warps issue the M tiles' MMAs in turn
// (each with descriptors built once and advanced by byte offsets) and commit each tile to its
// own mbarrier, so each tile's epilogue starts as soon as its accumulator is complete; the
// epilogue adds the bias, applies the ReLU,
// rounds to BF16 and writes the interior rows of the next layer's matrix (the padding rows stay
// zero). The last layer adds the FP32 input tile (the residual) and writes FP32 tiles.
//
// Operand rounding follows the bfloat16 form of the network: the weights and every layer's
// input are rounded to nearest BF16; biases, sums and the residual stay FP32.
#include <cuda_bf16.h>

#include "../../include/phy.h"
#include "launch.h"
#include "tc.cuh"

namespace phy {

namespace {

constexpr int kCnnThreads = 128;          // four warps: TMEM lanes 0..127 in the epilogue
constexpr int kTilesPerGroup = 4;
constexpr int kPadR = 16, kPadC = 14;     // padded tile: 14 + 2 rows, 12 + 2 columns
constexpr int kTileRows = 14, kTileCols = 12, kTilePos = kTileRows * kTileCols;
constexpr int kPadPos = kPadR * kPadC;    // 224 positions per padded tile
constexpr int kGroupPos = kTilesPerGroup * kPadPos;  // 896 = 7 M tiles of 128
constexpr int kMTiles = kGroupPos / 128;
constexpr int kGuard = 16;                // zero rows before and after (taps shift <= 15)
constexpr int kRowsP = kGuard + kGroupPos + kGuard;  // 928 rows per activation matrix
constexpr uint32_t kTmemCols = 256;       // 7 M tiles x 32 accumulator columns
constexpr uint32_t kWait = 1u << 22;

static_assert(kGroupPos % 128 == 0 && kRowsP % 8 == 0, "whole M tiles and core matrices");

// Flat parameter layout: per layer W [C_out][C_in][3][3] then b [C_out].
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 2 : 32; }
__host__ __device__ constexpr int cout_of(int l) { return l == 3 ? 2 : 32; }
__host__ __device__ constexpr int woff_of(int l) {
  return l == 0 ? 0 : l == 1 ? 608 : l == 2 ? 9856 : 19104;
}
__host__ __device__ constexpr int boff_of(int l) {
  return l == 0 ? 576 : l == 1 ? 9824 : l == 2 ? 19072 : 19680;
}
// Operand shapes in shared memory: C_in padded to a multiple of 16 (one MMA K step), C_out to
// at least 16 (the smallest N of an M = 128 MMA).
__host__ __device__ constexpr int kin_of(int l) { return l == 0 ? 16 : 32; }
__host__ __device__ constexpr int nout_of(int l) { return l == 3 ? 16 : 32; }

// Shared-memory map (bytes): two 32-channel activation matrices, per layer its nine tap blocks
// of K-major [N rows][K] weights, the biases (FP32), the MMA barrier and the TMEM address.
constexpr size_t kActBytes = (size_t)kRowsP * 32 * 2;  // 59,392
constexpr size_t kOffA = 0, kOffB = kActBytes;
__host__ __device__ constexpr size_t w_bytes(int l) { return (size_t)9 * nout_of(l) * kin_of(l) * 2; }
constexpr size_t kOffW0 = 2 * kActBytes;
constexpr size_t kOffW1 = kOffW0 + w_bytes(0);
constexpr size_t kOffW2 = kOffW1 + w_bytes(1);
constexpr size_t kOffW3 = kOffW2 + w_bytes(2);
constexpr size_t kOffBias = kOffW3 + w_bytes(3);  // 4 x 32 floats
constexpr size_t kOffXres = kOffBias + 4 * 32 * 4;  // the group's FP32 input tiles
constexpr int kGroupIn = kTilesPerGroup * 2 * kTilePos;   // input values of a group
constexpr int kInPerThread = (kGroupIn + kCnnThreads - 1) / kCnnThreads;
constexpr size_t kOffBar = kOffXres + (size_t)kGroupIn * 4;  // one mbarrier per M tile
constexpr size_t kOffMisc = kOffBar + 8 * ((kMTiles + 1) / 2 * 2);
constexpr size_t kSmem = kOffMisc + 16;
static_assert(kSmem <= 227 * 1024, "shared memory map too large");
__host__ __device__ constexpr size_t w_off(int l) {
  return l == 0 ? kOffW0 : l == 1 ? kOffW1 : l == 2 ? kOffW2 : kOffW3;
}

// Byte offset of element (row, k) in a K-major matrix of `rows` rows: 8-element (16-byte) K
// chunks of rows x 16 bytes each, rows 16 bytes apart inside a chunk.
__device__ __forceinline__ uint32_t kmaj(int rows, int row, int k) {
  return (uint32_t)((k >> 3) * rows * 16 + row * 16 + (k & 7) * 2);
}

__device__ __forceinline__ unsigned short bf16_bits(float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  return *reinterpret_cast<const unsigned short*>(&h);
}

// Row of the padded group matrix (guard rows included) holding interior position (i, j) of
// tile t of the group.
__device__ __forceinline__ int act_row(int t, int i, int j) {
  return kGuard + t * kPadPos + (i + 1) * kPadC + (j + 1);
}

// Persistent CTAs (one per SM) over groups of four tiles.
__global__ void __launch_bounds__(kCnnThreads, 1)
    cnn_forward_tc_kernel(int n_tiles, const float* __restrict__ P, const float* __restrict__ x,
                          float* __restrict__ out, unsigned* __restrict__ err,
                          float* __restrict__ acts) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* actA = sm + kOffA;
  unsigned char* actB = sm + kOffB;
  float* bias = reinterpret_cast<float*>(sm + kOffBias);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + kOffMisc);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // both activation matrices zero (their padding and guard rows stay zero from here on)
  for (int i = tid; i < (int)(2 * kActBytes / 16); i += kCnnThreads)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  // weights as per-tap K-major [C_out][C_in] BF16 blocks, zero where padded; biases
#pragma unroll 1
  for (int l = 0; l < 4; ++l) {
    const int N = nout_of(l), K = kin_of(l);
    unsigned char* wl = sm + w_off(l);
    for (int e = tid; e < 9 * N * K; e += kCnnThreads) {
      const int t = e / (N * K), r = e - t * N * K, co = r / K, ci = r - co * K;
      const float v =
          (co < cout_of(l) && ci < cin_of(l)) ? P[woff_of(l) + (co * cin_of(l) + ci) * 9 + t] : 0.f;
      *reinterpret_cast<unsigned short*>(wl + t * N * K * 2 + kmaj(N, co, ci)) = bf16_bits(v);
    }
    for (int c = tid; c < 32; c += kCnnThreads) bias[l * 32 + c] = c < cout_of(l) ? P[boff_of(l) + c] : 0.f;
  }
  if (tid == 0) {
    for (int m = 0; m < kMTiles; ++m) tc::mbar_init(bar + m, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(misc, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = misc[0];
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;

  uint32_t phase = 0;
  bool ok = true;
  const int n_groups = (n_tiles + kTilesPerGroup - 1) / kTilesPerGroup;
  float* xres = reinterpret_cast<float*>(sm + kOffXres);
  // a group's input tiles (contiguous [tile][channel][position]) in registers: the next group's
  // are loaded while this one is computed
  float xin[kInPerThread];
  auto load_group = [&](int grp) {
    const size_t base = (size_t)grp * kGroupIn, total = (size_t)n_tiles * 2 * kTilePos;
#pragma unroll
    for (int u = 0; u < kInPerThread; ++u) {
      const int e = tid + u * kCnnThreads;
      xin[u] = (e < kGroupIn && base + e < total) ? __ldg(x + base + e) : 0.f;
    }
  };
  if ((int)blockIdx.x < n_groups) load_group(blockIdx.x);
  for (int grp = blockIdx.x; grp < n_groups && ok; grp += gridDim.x) {
    const int t0 = grp * kTilesPerGroup;
    // the input tiles, rounded to BF16, as the first layer's 16-channel operand (channels 0, 1),
    // and in FP32 for the residual
#pragma unroll
    for (int u = 0; u < kInPerThread; ++u) {
      const int e = tid + u * kCnnThreads;
      if (e < kGroupIn) {
        const int t = e / (2 * kTilePos), c = (e / kTilePos) & 1, q = e % kTilePos;
        const int i = q / kTileCols, j = q - i * kTileCols;
        *reinterpret_cast<unsigned short*>(actB + kmaj(kRowsP, act_row(t, i, j), c)) =
            bf16_bits(xin[u]);
        xres[e] = xin[u];
      }
    }
    if (grp + (int)gridDim.x < n_groups) load_group(grp + gridDim.x);
#pragma unroll 1
    for (int l = 0; l < 4; ++l) {
      const unsigned char* src = (l & 1) ? actA : actB;
      unsigned char* dst = (l & 1) ? actB : actA;
      tc::fence_proxy_async();  // the operand written above is read by the tensor core
      __syncthreads();
      // lane 0 of each warp issues the MMAs of every fourth M tile (issue is the bottleneck of a
      // run of small N = 32 MMAs from one thread)
      if (lane == 0) {
        tc::fence_after_sync();
        const int N = nout_of(l), K = kin_of(l);
        const uint32_t idesc = tc::instr_desc(tc::kFmtBF16, 128, N);
        const uint32_t lbo_a = kRowsP * 16, lbo_b = N * 16;
        // descriptors built once; each MMA's operands are fixed byte offsets from them
        const uint64_t da0 = tc::smem_desc(tc::smem_u32(src), lbo_a, 128);
        const uint64_t db0 = tc::smem_desc(tc::smem_u32(sm + w_off(l)), lbo_b, 128);
#pragma unroll 1
        for (int m = warp; m < kMTiles; m += kCnnThreads / 32) {
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const int row0 = kGuard + m * 128 + (t / 3 - 1) * kPadC + (t % 3 - 1);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              if (ks < K / 16) {
                const uint64_t da = tc::desc_advance(da0, row0 * 16 + ks * 2 * lbo_a);
                const uint64_t db = tc::desc_advance(db0, t * N * K * 2 + ks * 2 * lbo_b);
                tc::mma<tc::kFmtBF16>(tmem + m * 32, da, db, idesc, (t | ks) != 0 ? 1u : 0u);
              }
            }
          }
          // M tile m's accumulator is complete once every MMA this thread issued so far is:
          // its epilogue starts while the tensor core works on the other tiles
          tc::mma_commit(bar + m);
        }
      }
      // epilogue: this thread's TMEM lane is its row of each M tile
      bool done = true;
#pragma unroll 1
      for (int m = 0; m < kMTiles; ++m) {
        done = __all_sync(0xffffffffu, tc::mbar_wait(bar + m, phase, kWait));  // warp-uniform
        if (!done) break;
        tc::fence_after_sync();
        float v[32];
        tc::tmem_ld32(tmem + lane_base + m * 32, v);
        const int p = m * 128 + 32 * (warp & 3) + lane;  // position in the group
        const int t = p / kPadPos, q = p - t * kPadPos, pr = q / kPadC, pc = q - pr * kPadC;
        if (pr < 1 || pr > kTileRows || pc < 1 || pc > kTileCols) continue;
        const int q0 = (pr - 1) * kTileCols + (pc - 1);
        if (l < 3) {
          // the layer's output as the next layer reads it (BF16), also kept in FP32 for a
          // backward pass when acts is set: acts[l][tile][channel][position]
          float* keep = (acts && t0 + t < n_tiles)
                            ? acts + (size_t)l * n_tiles * 32 * kTilePos +
                                  (size_t)(t0 + t) * 32 * kTilePos + q0
                            : nullptr;
#pragma unroll
          for (int c8 = 0; c8 < 4; ++c8) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const float a = fmaxf(v[c8 * 8 + 2 * h] + bias[l * 32 + c8 * 8 + 2 * h], 0.f);
              const float b = fmaxf(v[c8 * 8 + 2 * h + 1] + bias[l * 32 + c8 * 8 + 2 * h + 1], 0.f);
              const unsigned short ba = bf16_bits(a), bb = bf16_bits(b);
              w[h] = (uint32_t)ba | ((uint32_t)bb << 16);
              if (keep) {
                keep[(size_t)(c8 * 8 + 2 * h) * kTilePos] = __uint_as_float((uint32_t)ba << 16);
                keep[(size_t)(c8 * 8 + 2 * h + 1) * kTilePos] = __uint_as_float((uint32_t)bb << 16);
              }
            }
            *reinterpret_cast<uint4*>(dst + kmaj(kRowsP, kGuard + p, c8 * 8)) =
                make_uint4(w[0], w[1], w[2], w[3]);
          }
        } else if (t0 + t < n_tiles) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const size_t o = ((size_t)(t0 + t) * 2 + c) * kTilePos + q0;
            out[o] = xres[(t * 2 + c) * kTilePos + q0] + (v[c] + bias[3 * 32 + c]);
          }
        }
      }
      if (!done)  // MMAs in flight finish before anything else happens
        for (int m = 0; m < kMTiles; ++m) tc::mbar_wait(bar + m, phase, kWait);
      phase ^= 1u;
      tc::fence_before_sync();  // TMEM reads done before the next layer's MMAs overwrite it
      ok = __syncthreads_and(done);
      if (!ok) break;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (!ok && tid == 0) atomicAdd(err, 1u);
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

size_t cnn_tc_smem_bytes() { return kSmem; }

cudaError_t cnn_forward_tc(int n, const float* P, const float* x, float* out, unsigned* err,
                           cudaStream_t st, float* acts) {
  static bool configured_on[kMaxDevices] = {};
  bool& configured = configured_on[current_device()];
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(cnn_forward_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (n <= 0) return cudaSuccess;
  const int groups = (n + kTilesPerGroup - 1) / kTilesPerGroup;
  const int grid = groups < device_sm_count() ? groups : device_sm_count();
  cnn_forward_tc_kernel<<<grid, kCnnThreads, kSmem, st>>>(n, P, x, out, err, acts);
  return cudaGetLastError();
}

}  // namespace phy
