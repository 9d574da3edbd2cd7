// Segment kernel on the tcgen05 tensor cores: the corner cross-Gram X = C^H C and the matched
// filter V = C^H y of every RE of a frequency segment, as real GEMMs with FP32 accumulation in
// tensor memory (the paper's covariance-by-FMA step of Fig. 2(b), on the dense unit).
//
// Complex products are embedded in real ones. With the corner-layer columns of C as rows of
// CC = [C ; iC] (row c: (Re C_rc, Im C_rc) interleaved over r; row NXP + c: (-Im, Re)), and y
// likewise interleaved over r:
//   (CC CC_C^T)[c][m]      = Re X[c][m],   (CC CC_C^T)[NXP + c][m] = Im X[c][m]    (M=128, N=NXP)
//   (Yt CC^T)[re][c]       = Re V[c][re],  (Yt CC^T)[re][NXP + c]  = Im V[c][re]   (M=128, N=2NXP)
// with K = 2 x 64 receive antennas (zero-padded). Operands are rounded to TF32, FP16 or BF16
// (round to nearest) when staged; everything after the products stays FP32. The epilogue folds X
// into the per-symbol Gram blocks (as the FP32 kernel does) and V into the matched filter
// b = sum over corners of the interpolation weights times V, per RE, straight from TMEM.
//
// Persistent CTAs of 128 threads loop over (segment, cell) items; tensor memory and the
// mbarrier are set up once per CTA. Thread 0 issues the MMAs; every wait is bounded (a timeout
// bumps an error counter, waits once more and still frees the tensor memory). Operand staging
// keeps 16 global loads in flight per thread, one RE row per thread so a warp's loads coalesce.
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "launch.h"
#include "segment.cuh"
#include "tc.cuh"

namespace phy {

namespace {

constexpr int kTcThreads = 128;
constexpr int kRows = 128;  // UMMA M and rows of every operand tile
constexpr int kK = 128;     // K elements per operand row: (re, im) x 64 antennas
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kWaitIters = 1u << 22;

template <uint32_t FMT>
struct Layout {
  static constexpr int kEs = tc::Elem<FMT>::kBytes;
  static constexpr int kTileBytes = kRows * kK * kEs;
  // no-swizzle K-major core matrices (8 rows x 16 bytes), K-chunk major
  static constexpr uint32_t kLbo = (kRows / 8) * 128;  // next 16-byte K chunk
  static constexpr uint32_t kSbo = 128;                // next 8-row group
  static constexpr int kKSteps = kK * kEs / 32;        // one MMA per 32 bytes of K
  __device__ static uint32_t off(int row, int kel) {
    const int bk = kel * kEs;
    return ((bk >> 4) * (kRows / 8) + (row >> 3)) * 128 + (row & 7) * 16 + (bk & 15);
  }
};

template <uint32_t FMT>
__device__ __forceinline__ void store_pair(unsigned char* p, float a, float b) {
  if constexpr (FMT == tc::kFmtTF32)
    *reinterpret_cast<uint2*>(p) = tc::Elem<FMT>::pack(a, b);
  else
    *reinterpret_cast<uint32_t*>(p) = tc::Elem<FMT>::pack(a, b);
}

constexpr int nxp_of(int nx) { return nx <= 16 ? 16 : (nx + 15) / 16 * 16; }

// CC tile, then one region that holds X in FP32 and afterwards the RE tile, then the barrier.
template <int NL, int NC, uint32_t FMT>
constexpr size_t tc_smem_bytes() {
  constexpr int NXP = nxp_of(NC * NL);
  constexpr size_t xs_bytes = (size_t)NXP * (NXP + 2) * 8;
  constexpr size_t r2 =
      (size_t)Layout<FMT>::kTileBytes > xs_bytes ? Layout<FMT>::kTileBytes : xs_bytes;
  return Layout<FMT>::kTileBytes + ((r2 + 15) & ~(size_t)15) + 16;
}

// Issues one K-loop of MMAs (A and B tiles in the same layout) and commits to the barrier.
template <uint32_t FMT>
__device__ __forceinline__ void gemm_issue(uint32_t tmem, const unsigned char* a,
                                           const unsigned char* b, uint32_t idesc,
                                           uint64_t* bar) {
  using Lay = Layout<FMT>;
  const uint32_t a0 = tc::smem_u32(a), b0 = tc::smem_u32(b);
#pragma unroll 1
  for (int s = 0; s < Lay::kKSteps; ++s) {
    const uint32_t step = (uint32_t)s * 2u * Lay::kLbo;
    tc::mma<FMT>(tmem, tc::smem_desc(a0 + step, Lay::kLbo, Lay::kSbo),
                 tc::smem_desc(b0 + step, Lay::kLbo, Lay::kSbo), idesc, s > 0 ? 1u : 0u);
  }
  tc::mma_commit(bar);
}

// Makes staged shared memory visible to the tensor core and synchronises the CTA.
__device__ __forceinline__ void publish_smem() {
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

template <int NL, int NC, uint32_t FMT>
__global__ void __launch_bounds__(kTcThreads)
    seg_prep_tc_kernel(Geo g, int cell0, int nc, const phy_c32* __restrict__ anchors,
                       const phy_c32* __restrict__ Y, float4* __restrict__ ygg,
                       cf* __restrict__ bvec, unsigned* __restrict__ err) {
  using Lay = Layout<FMT>;
  constexpr int NX = NC * NL;
  constexpr int NXP = nxp_of(NX);
  constexpr int xs = NXP + 2;
  constexpr int NTRI = NL * (NL + 1) / 2;
  static_assert(2 * NXP <= kRows, "corner-layer count too large for one tile");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* cc = smem;
  unsigned char* r2 = smem + Lay::kTileBytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + tc_smem_bytes<NL, NC, FMT>() - 16);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  cf* Xs = reinterpret_cast<cf*>(r2);
  unsigned char* yt = r2;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nr = g.n_rx, nl = g.n_layers, nds = g.n_dsym;

  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(slot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t tmem_warp = tmem + ((uint32_t)(32 * warp) << 16);
  uint32_t phase = 0;
  bool fail = false;

  const int n_work = g.n_seg * nc;
  for (int w = blockIdx.x; w < n_work && !fail; w += gridDim.x) {
    const int j = w % g.n_seg, lc = w / g.n_seg, cell = cell0 + lc;
    int lo, hi;
    segment_range(g, j, lo, hi);
    const int W = hi - lo, nre = W * nds;

    // ---- CC = [C ; iC]
    {
      const int g1 = seg_g1(g, j);
#pragma unroll 8
      for (int it = 0; it < NXP * 64 / kTcThreads; ++it) {
        const int e = tid + it * kTcThreads;
        const int r = e & 63, c = e >> 6;
        const int corner = c / NL, l = c % NL;
        cf v = mk(0.f, 0.f);
        if (c < NX && l < nl && r < nr) {
          const int d = corner >> 1, grp = (corner & 1) ? g1 : j;
          v = ld(anchors + ((((size_t)cell * g.n_dmrs + d) * g.G + grp) * nl + l) * nr + r);
        }
        store_pair<FMT>(cc + Lay::off(c, 2 * r), v.x, v.y);
        store_pair<FMT>(cc + Lay::off(NXP + c, 2 * r), -v.y, v.x);
      }
    }
    publish_smem();

    // ---- X = C^H C
    if (tid == 0) gemm_issue<FMT>(tmem, cc, cc, tc::instr_desc(FMT, kRows, NXP), bar);
    fail = !tc::mbar_wait(bar, phase, kWaitIters);
    phase ^= 1;
    fail = __syncthreads_or(fail);
    if (fail) break;
    tc::fence_after_sync();
    {
      const int row = 32 * warp + lane;
#pragma unroll
      for (int c0 = 0; c0 < NXP; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem_warp + c0, v);
        if (row < 2 * NXP) {
          const int c = row % NXP, part = row / NXP;
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (c0 + q < NXP) reinterpret_cast<float*>(Xs + c * xs + c0 + q)[part] = v[q];
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    auto Xget = [&](int i, int k) -> cf { return Xs[i * xs + k]; };
    form_gram_blocks<NL, kTcThreads>(g, Xget,
                                     ygg + (((size_t)lc * g.n_seg + j) * nds) * NTRI * 2, tid);
    __syncthreads();  // Xs shares its space with the RE tiles below

    // ---- matched filter, 128 REs per tile, one RE row per thread
    const int ntile = (nre + kRows - 1) / kRows;
    for (int t = 0; t < ntile; ++t) {
      const int re = kRows * t + tid;
      const bool valid = re < nre;
      const int jj = valid ? re / W : 0, kk = valid ? re - jj * W : 0, k = lo + kk;
      {
        const phy_c32* yp = Y + ((size_t)cell * g.n_sym + g.dsym[jj]) * nr * g.n_sc + k;
#pragma unroll 1
        for (int r0 = 0; r0 < 64; r0 += 16) {
          cf v[16];
#pragma unroll
          for (int q = 0; q < 16; ++q)
            v[q] = (valid && r0 + q < nr) ? ld(yp + (size_t)(r0 + q) * g.n_sc) : mk(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < 16; ++q) store_pair<FMT>(yt + Lay::off(tid, 2 * (r0 + q)), v[q].x, v[q].y);
        }
      }
      publish_smem();
      if (tid == 0) gemm_issue<FMT>(tmem, yt, cc, tc::instr_desc(FMT, kRows, 2 * NXP), bar);
      fail = !tc::mbar_wait(bar, phase, kWaitIters);
      phase ^= 1;
      fail = __syncthreads_or(fail);
      if (fail) break;
      tc::fence_after_sync();
      // this thread's TMEM lane is its RE row
      const int jr = 32 * warp + lane;
      const int re2 = kRows * t + jr;
      const bool valid2 = re2 < nre;
      const int jj2 = valid2 ? re2 / W : 0, kk2 = valid2 ? re2 - jj2 * W : 0, k2 = lo + kk2;
      const float t1 = g.tw[jj2], t0 = 1.f - t1;
      const float be0 = seg_beta(g, j, k2, 0), be1 = seg_beta(g, j, k2, 1);
      float bre[NL], bim[NL];
#pragma unroll
      for (int l = 0; l < NL; ++l) bre[l] = bim[l] = 0.f;
#pragma unroll
      for (int part = 0; part < 2; ++part) {
#pragma unroll
        for (int c0 = 0; c0 < NXP; c0 += 32) {
          float v[32];
          tc::tmem_ld32(tmem_warp + part * NXP + c0, v);
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int c = c0 + q;
            if (c < NX) {
              const int corner = c / NL, l = c % NL;
              const float be = (l & 1) ? be1 : be0;
              const float wt = ((corner >> 1) ? t1 : t0) * ((corner & 1) ? be : 1.f - be);
              if (part == 0)
                bre[l] = fmaf(wt, v[q], bre[l]);
              else
                bim[l] = fmaf(wt, v[q], bim[l]);
            }
          }
        }
      }
      if (valid2) {
        float4* bo =
            reinterpret_cast<float4*>(bvec + ((size_t)(lc * nds + jj2) * g.n_sc + k2) * NL);
#pragma unroll
        for (int l = 0; l < NL; l += 2)
          bo[l / 2] = make_float4(bre[l], bim[l], bre[l + 1], bim[l + 1]);
      }
      tc::fence_before_sync();
      __syncthreads();  // TMEM and the tile are free for the next round
    }
  }
  if (fail) {
    if (tid == 0) atomicAdd(err, 1u);
    tc::mbar_wait(bar, phase ^ 1, kWaitIters);  // give in-flight MMAs a second chance to land
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

int g_num_sms = 0;

template <int NL, int NC, uint32_t FMT>
cudaError_t launch_one(const Geo& g, int c0, int nc, const phy_c32* anchors, const phy_c32* Y,
                       float4* ygg, cf* bvec, unsigned* err, cudaStream_t st) {
  constexpr size_t smem = tc_smem_bytes<NL, NC, FMT>();
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(seg_prep_tc_kernel<NL, NC, FMT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // all of the unified L1/shared storage as shared memory, so that several CTAs fit
    e = cudaFuncSetAttribute(seg_prep_tc_kernel<NL, NC, FMT>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev)) !=
        cudaSuccess)
      return e;
    // The occupancy query answers 1 for kernels that allocate tensor memory, although several
    // such CTAs do share an SM; size the persistent grid from shared and tensor memory instead
    // (CTAs beyond what fits would only wait for a slot).
    int smem_sm = 0;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
        cudaSuccess)
      return e;
    const int b = smem_sm / (int)(smem + 1024);
    blocks_per_sm = std::max(1, std::min(b, (int)(512 / kTmemCols)));
    if (std::getenv("PHY_DEBUG"))
      std::fprintf(stderr, "seg_prep_tc<%d,%d,%u>: smem %zu, occupancy %d, SMs %d, blocks/SM %d\n",
                   NL, NC, FMT, smem, b, g_num_sms, blocks_per_sm);
  }
  const int n_work = g.n_seg * nc;
  const int grid = std::min(n_work, blocks_per_sm * g_num_sms);
  seg_prep_tc_kernel<NL, NC, FMT><<<grid, kTcThreads, smem, st>>>(g, c0, nc, anchors, Y, ygg,
                                                                 bvec, err);
  return cudaGetLastError();
}

template <int NL, uint32_t FMT>
cudaError_t launch_nc(const Geo& g, int c0, int nc, const phy_c32* anchors, const phy_c32* Y,
                      float4* ygg, cf* bvec, unsigned* err, cudaStream_t st) {
  if (g.n_dmrs == 2) return launch_one<NL, 4, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
  return launch_one<NL, 2, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
}

template <uint32_t FMT>
cudaError_t launch_fmt(const Geo& g, int NL, int c0, int nc, const phy_c32* anchors,
                       const phy_c32* Y, float4* ygg, cf* bvec, unsigned* err, cudaStream_t st) {
  switch (NL) {
    case 2: return launch_nc<2, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
    case 4: return launch_nc<4, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
    case 8: return launch_nc<8, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
    default: return launch_nc<16, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
  }
}

}  // namespace

cudaError_t launch_seg_prep_tc(const Geo& g, int NL, int c0, int nc, const phy_c32* anchors,
                               const phy_c32* Y, float4* ygg, cf* bvec, unsigned* err,
                               cudaStream_t st) {
  switch (g.prec) {
    case PHY_PREC_TC_TF32:
      return launch_fmt<tc::kFmtTF32>(g, NL, c0, nc, anchors, Y, ygg, bvec, err, st);
    case PHY_PREC_TC_BF16:
      return launch_fmt<tc::kFmtBF16>(g, NL, c0, nc, anchors, Y, ygg, bvec, err, st);
    default:
      return launch_fmt<tc::kFmtF16>(g, NL, c0, nc, anchors, Y, ygg, bvec, err, st);
  }
}

}  // namespace phy
