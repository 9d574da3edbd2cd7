// DMRS least-squares channel estimation (the channel-estimation block named in Sec. III-B).
//
// anchor[cell][d][g][l][r] = (1/L) sum_{i<L} Y[cell][t_d][r][k_i] conj(P[cell][d][l][k_i]),
// k_i = 2 (s_g + i) + (l % 2).
//
// One CTA per (group, DMRS symbol, cell), one thread per receive antenna. The group's 2L
// subcarriers are one contiguous 16L-byte run of each antenna row of Y: each thread loads its
// run once with 16-byte loads into registers; the pilots of the group (all layers) are staged in
// shared memory once per CTA and read as broadcasts. Writes are coalesced over r.
//
// The BFP variant reads the same runs straight from the compressed fronthaul stream (bfp.cuh)
// instead of a decompressed grid, with the decompressor's arithmetic, so its anchors are bitwise
// those of the plain kernel on the decompressed grid. Each warp stages the blocks of its antennas'
// runs (at most four blocks of 1 + 3w bytes per antenna) in shared memory, one antenna row at a
// time with the lanes over the row's 32-bit words (coalesced), and each thread unpacks its own.
#include "batch.cuh"
#include "bfp.cuh"
#include "launch.h"

namespace phy {

namespace {

constexpr int kChestThreads = 64;
constexpr int kChestBfpWords = 52;  // 4 blocks of <= 49 bytes, misalignment and window slack

// Compressed received grid: the stream, its size, mantissa width and scale.
struct BfpGrid {
  const uint8_t* yc;
  long long total;
  int w;
  float scale;
};

// One (group, DMRS symbol, cell) work item; the block's threads are its antennas.
template <int L, bool BFP>
__device__ __forceinline__ void chest_body(const Geo& g, int grp, int d, int cell,
                                           const phy_c32* __restrict__ Y, BfpGrid bfp,
                                           const phy_c32* __restrict__ P,
                                           phy_c32* __restrict__ anchors) {
  __shared__ cf pil[kMaxLayers][2 * L];
  const int r = threadIdx.x;
  const int t = (d == 0) ? g.dmrs0 : g.dmrs1;
  const int s = group_start(g, grp);
  const int k0 = 2 * s;  // first subcarrier of the group's run
  const int nl = g.n_layers;
  const phy_c32* prow = P + (size_t)(cell * g.n_dmrs + d) * nl * g.n_sc + k0;
  // this antenna's run of Y first, so that its loads are in flight with the pilots' ones
  const bool live = r < g.n_rx;
  cf y[2 * L];
  if constexpr (BFP) {
    __shared__ uint32_t s_blk[kChestThreads][kChestBfpWords];
    const int nb = 1 + 3 * bfp.w, n_prb = g.n_sc / 12;
    const int p0 = k0 / 12, p1 = (k0 + 2 * L - 1) / 12;  // PRBs of the run
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(bfp.yc);
    const long long row0 = ((long long)cell * g.n_sym + t) * g.n_rx;
    for (int j = 0; j < 32; ++j) {  // the warp's antennas, one row at a time
      const int rr = warp * 32 + j;
      if (rr >= g.n_rx) break;
      const long long start = ((row0 + rr) * n_prb + p0) * nb;
      const long long w0 = start >> 2, w1 = (start + (long long)(p1 - p0 + 1) * nb + 3) >> 2;
      for (long long k = w0 + lane; k < w1; k += 32) {
        uint32_t v = 0;
        if (4 * k + 4 <= bfp.total) {
          v = __ldg(src + k);
        } else {  // the stream's last partial word
          for (int q = 0; q < 4; ++q)
            if (4 * k + q < bfp.total) v |= (uint32_t)__ldg(bfp.yc + 4 * k + q) << (8 * q);
        }
        s_blk[rr][k - w0] = v;
      }
    }
    __syncwarp();
    if (live) {
      const long long start = ((row0 + r) * n_prb + p0) * nb;
      const uint8_t* run = reinterpret_cast<const uint8_t*>(s_blk[r]) + (start & 3);
#pragma unroll
      for (int i = 0; i < 2 * L; ++i) {
        const int k = k0 + i;
        const uint8_t* blk = run + (k / 12 - p0) * nb;
        const float p2 = (float)(1 << (blk[0] & 0xF));
        const int m = 2 * (k % 12);
        y[i] = mk(bfp_value(bfp_mantissa_padded(blk, bfp.w, m), p2, bfp.scale),
                  bfp_value(bfp_mantissa_padded(blk, bfp.w, m + 1), p2, bfp.scale));
      }
    }
  } else if constexpr (L >= 2) {
    const phy_c32* yrow =
        Y + ((size_t)(cell * g.n_sym + t) * g.n_rx + (live ? r : 0)) * g.n_sc + k0;
    // k0 is even, so the run starts on a 16-byte boundary
    const float4* y4 = reinterpret_cast<const float4*>(yrow);
#pragma unroll
    for (int i = 0; i < L; ++i) {
      const float4 v = __ldg(y4 + i);
      y[2 * i] = mk(v.x, v.y);
      y[2 * i + 1] = mk(v.z, v.w);
    }
  } else {
    const phy_c32* yrow =
        Y + ((size_t)(cell * g.n_sym + t) * g.n_rx + (live ? r : 0)) * g.n_sc + k0;
    y[0] = ld(yrow);
    y[1] = ld(yrow + 1);
  }
  for (int e = threadIdx.x; e < nl * 2 * L; e += blockDim.x) {
    const int l = e / (2 * L), i = e % (2 * L);
    pil[l][i] = ld(prow + (size_t)l * g.n_sc + i);
  }
  __syncthreads();
  if (!live) return;
  phy_c32* out = anchors + (((size_t)(cell * g.n_dmrs + d) * g.G + grp) * nl) * g.n_rx;
  const float inv_l = 1.f / (float)L;
  for (int l = 0; l < nl; ++l) {
    const int c = l & 1;
    cf acc = mk(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < L; ++i) {  // y conj(p); the select keeps y in registers
      const cf yv = c ? y[2 * i + 1] : y[2 * i];
      acc = cfma_cj(pil[l][2 * i + c], yv, acc);
    }
    st(out + (size_t)l * g.n_rx + r, inv_l * acc);
  }
}

template <int L, bool BFP>
__global__ void __launch_bounds__(kChestThreads)
    chest_ls_kernel(Geo g, const phy_c32* __restrict__ Y, BfpGrid bfp,
                    const phy_c32* __restrict__ P, phy_c32* __restrict__ anchors) {
  chest_body<L, BFP>(g, blockIdx.x, blockIdx.y, blockIdx.z, Y, bfp, P, anchors);
}

template <bool BFP>
cudaError_t launch_chest_any(const Geo& g, const phy_c32* Y, BfpGrid bfp, const phy_c32* pilots,
                             phy_c32* anchors, cudaStream_t st) {
  dim3 grid(g.G, g.n_dmrs, g.n_cells);
  const int threads = g.n_rx <= 32 ? 32 : 64;
  switch (g.L) {
    case 1: chest_ls_kernel<1, BFP><<<grid, threads, 0, st>>>(g, Y, bfp, pilots, anchors); break;
    case 2: chest_ls_kernel<2, BFP><<<grid, threads, 0, st>>>(g, Y, bfp, pilots, anchors); break;
    case 4: chest_ls_kernel<4, BFP><<<grid, threads, 0, st>>>(g, Y, bfp, pilots, anchors); break;
    case 8: chest_ls_kernel<8, BFP><<<grid, threads, 0, st>>>(g, Y, bfp, pilots, anchors); break;
    case 16:
      chest_ls_kernel<16, BFP><<<grid, threads, 0, st>>>(g, Y, bfp, pilots, anchors);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Batched LS item: `gp` consecutive groups of one (DMRS symbol, cell), thread (group, antenna);
// the arithmetic per anchor is chest_body's, so both give the same bits. pil: staged pilots
// [group][layer][2L].
template <int L>
__device__ __forceinline__ void chest_multi_body(const Geo& g, int grp0, int gp, int d, int cell,
                                                 const phy_c32* __restrict__ Y,
                                                 const phy_c32* __restrict__ P,
                                                 phy_c32* __restrict__ anchors,
                                                 cf* __restrict__ pil) {
  const int lg = __ffs(kChestBatchThreads / gp) - 1;  // log2 of the padded antenna count
  const int r = threadIdx.x & ((1 << lg) - 1), gi = threadIdx.x >> lg, grp = grp0 + gi;
  const int t = (d == 0) ? g.dmrs0 : g.dmrs1;
  const int nl = g.n_layers;
  const bool live = r < g.n_rx && grp < g.G;
  cf y[2 * L];
  if (live) {
    const int k0 = 2 * group_start(g, grp);  // even: the run starts on a 16-byte boundary
    const phy_c32* yrow = Y + ((size_t)(cell * g.n_sym + t) * g.n_rx + r) * g.n_sc + k0;
    if constexpr (L >= 2) {
      const float4* y4 = reinterpret_cast<const float4*>(yrow);
#pragma unroll
      for (int i = 0; i < L; ++i) {
        const float4 v = __ldg(y4 + i);
        y[2 * i] = mk(v.x, v.y);
        y[2 * i + 1] = mk(v.z, v.w);
      }
    } else {
      y[0] = ld(yrow);
      y[1] = ld(yrow + 1);
    }
  }
  const int ngl = min(gp, g.G - grp0);
  const phy_c32* pbase = P + (size_t)(cell * g.n_dmrs + d) * nl * g.n_sc;
  for (int l = 0; l < nl; ++l) {  // per layer: the chunk's groups, 2L pilots each
    const phy_c32* prow = pbase + (size_t)l * g.n_sc;
    for (int e = threadIdx.x; e < ngl * 2 * L; e += blockDim.x) {
      const int gj = e / (2 * L), i = e % (2 * L);
      pil[(gj * nl + l) * 2 * L + i] = ld(prow + 2 * group_start(g, grp0 + gj) + i);
    }
  }
  __syncthreads();
  if (!live) return;
  phy_c32* out = anchors + (((size_t)(cell * g.n_dmrs + d) * g.G + grp) * nl) * g.n_rx;
  const float inv_l = 1.f / (float)L;
  for (int l = 0; l < nl; ++l) {
    const int c = l & 1;
    const cf* pl = pil + (gi * nl + l) * 2 * L;
    cf acc = mk(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < L; ++i) {
      const cf yv = c ? y[2 * i + 1] : y[2 * i];
      acc = cfma_cj(pl[2 * i + c], yv, acc);
    }
    st(out + (size_t)l * g.n_rx + r, inv_l * acc);
  }
}

// Batched form: CTAs stride over the LS items (group chunk, DMRS symbol, cell) of every job in
// the table; the first item of each job also clears the job's error word for the later stages.
__global__ void __launch_bounds__(kChestBatchThreads)
    chest_batch_kernel(const BatchTable* __restrict__ t) {
  __shared__ Geo sg;
  __shared__ cf pil[kChestBatchPilots];
  __shared__ BatchIndex ix;
  const int n = t->n_items[kBatchChest][0];
  // items strided over the CTAs (a job's items spread over the grid: balanced whatever the mix
  // of light and heavy jobs); a CTA keeps the geometry while consecutive items share a job
  if ((int)blockIdx.x >= n) return;
  batch_index_load(ix, t, kBatchChest, 0);
  __syncthreads();
  int cur = -1;
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    int local;
    const int jb = batch_find(ix, w, local);
    const BatchJob& J = t->job[jb];
    if (jb != cur) {  // uniform over the block
      batch_load_geo(sg, J.g);
      cur = jb;
    }
    __syncthreads();
    const int gp = chest_batch_groups(sg.n_rx), nch = (sg.G + gp - 1) / gp;
    const int grp0 = (local % nch) * gp, d = (local / nch) % sg.n_dmrs;
    const int cell = local / (nch * sg.n_dmrs);
    if (local == 0 && threadIdx.x == 0) *J.err = 0;
    switch (sg.L) {
      case 1: chest_multi_body<1>(sg, grp0, gp, d, cell, J.Y, J.pilots, J.anchors, pil); break;
      case 2: chest_multi_body<2>(sg, grp0, gp, d, cell, J.Y, J.pilots, J.anchors, pil); break;
      case 4: chest_multi_body<4>(sg, grp0, gp, d, cell, J.Y, J.pilots, J.anchors, pil); break;
      default: chest_multi_body<8>(sg, grp0, gp, d, cell, J.Y, J.pilots, J.anchors, pil); break;
    }
    __syncthreads();  // the geometry and the pilot stage are rewritten by the next item
  }
}

}  // namespace

cudaError_t launch_chest_batch(const BatchTable* t, cudaStream_t st) {
  // two waves of CTAs: those that finish early take the next ones
  static int grid_on[kMaxDevices] = {};
  int& grid = grid_on[current_device()];
  if (grid == 0) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chest_batch_kernel,
                                                      kChestBatchThreads, 0) != cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    grid = 2 * device_sm_count() * occ;
  }
  chest_batch_kernel<<<grid, kChestBatchThreads, 0, st>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_chest(const Geo& g, const phy_c32* Y, const phy_c32* pilots, phy_c32* anchors,
                         cudaStream_t st) {
  return launch_chest_any<false>(g, Y, BfpGrid{nullptr, 0, 0, 0.f}, pilots, anchors, st);
}

cudaError_t launch_chest_bfp(const Geo& g, const uint8_t* yc, int w, float scale,
                             const phy_c32* pilots, phy_c32* anchors, cudaStream_t st) {
  const long long total =
      (long long)g.n_cells * g.n_sym * g.n_rx * (g.n_sc / 12) * (long long)(1 + 3 * w);
  return launch_chest_any<true>(g, nullptr, BfpGrid{yc, total, w, scale}, pilots, anchors, st);
}

}  // namespace phy
