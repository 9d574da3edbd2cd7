// LMMSE detection on FP32 CUDA cores in two kernels: per-segment Gram blocks and matched filter,
// then a flat one-thread-per-RE solve.
//
// With linear interpolation every RE's channel is a weighted sum of the four "corner" anchor
// matrices of its frequency segment (anchors j and j+1 of both DMRS symbols): column l of
// H(k, t) is sum_{d,g} tau_d(t) w_g(k, comb(l)) C_{d,g}[:, l]. The Gram matrix of every RE of a
// segment is therefore a quadratic form in one corner cross-Gram X = C^H C
// (C = [C_00 C_01 C_10 C_11], n_rx x 4 n_layers) computed once per segment: the paper's
// covariance-by-FMA step (Fig. 2(b)) done once per segment instead of once per RE, exact up to
// rounding. Per data symbol the time weights fold X into Y_gg'(t) = H_g(t)^H H_g'(t),
// g, g' in {0, 1}; per RE, A = sum_{g,g'} D_g Y_gg' D_g' + s2 I with D_g diagonal frequency
// weights. The matched filter uses the time-interpolated anchors: b = D_0 H_0^H y + D_1 H_1^H y.
//
//  seg_prep_fp32_kernel: one CTA per (segment, cell). Corners to shared memory, X (lower 4x4
//    tiles), the four Y_gg' blocks per data symbol (lower triangle, 4-tuples) to the workspace,
//    and the matched filter per symbol from a shared-memory Y tile (cp.async double buffer).
//  re_solve_fp32_kernel: one thread per data RE. Builds A from the 4-tuples (bulk-copied to
//    shared memory), solves (solver.cuh; with 9..16 layers the per-thread L21/T block in tensor
//    memory), SINR, unbiasing, max-log LLRs, stores staged through shared memory.
// The two kernels run per chunk of cells so that the intermediates stay small (L2-sized).
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "batch.cuh"
#include "launch.h"
#include "segment.cuh"
#include "refactor64.cuh"
#include "solver.cuh"
#include "tc.cuh"

namespace phy {

namespace {

constexpr int kPrepThreads = 256;
constexpr int kSolveThreads = 128;
constexpr size_t kChunkBudget = 256ull << 20;  // preferred intermediates per chunk of cells

// Intermediates budget per chunk; the environment variable PHY_CHUNK_MB overrides it (tuning).
size_t chunk_budget() {
  static const size_t v = [] {
    const char* e = std::getenv("PHY_CHUNK_MB");
    const long mb = e ? std::atol(e) : 0;
    return mb > 0 ? (size_t)mb << 20 : kChunkBudget;
  }();
  return v;
}

int nl_class(int nl) { return nl <= 2 ? 2 : nl <= 4 ? 4 : nl <= 8 ? 8 : 16; }

// Shared memory of the FP32 segment kernel (cf units): the corner anchors C [rx][corner-layer],
// two received-grid tiles [rx][subcarrier] (the data symbols of one round), and a region that
// first holds X and then the round's interpolated channels Hg [symbol][rx][comb group, layer].
struct PrepLayout {
  int NC, NX, xs, yw, hs;
  int off_C, off_Y, off_X, total;
};

__host__ __device__ inline PrepLayout prep_layout(int NL, int n_dmrs, int n_rx, int wmax) {
  PrepLayout f;
  f.NC = 2 * n_dmrs;
  f.NX = f.NC * NL;
  f.xs = f.NX + 2;                     // keeps 16-byte row alignment, spreads banks
  f.yw = ((wmax + 3) & ~3) + 2;        // room for whole 4-subcarrier quads, even (16-byte rows)
  f.hs = 2 * NL + 2;
  f.off_C = 0;
  f.off_Y = f.off_C + n_rx * f.xs;
  f.off_X = f.off_Y + 2 * n_rx * f.yw;
  const int xr = f.NX * f.xs, hr = 2 * n_rx * f.hs;
  f.total = f.off_X + (xr > hr ? xr : hr);
  return f;
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// One CTA per (segment, cell). X = C^H C from the corner anchors and the per-symbol Gram blocks,
// then the matched filter b = sum_g w_g (tau_0 C_0g + tau_1 C_1g)^H y per RE, two data symbols
// per round: 128 threads per symbol, each group of four lanes one 4-RE x (2 layers x 2 comb
// groups) register tile with the antennas split four ways (a shuffle reduction at the end).
// The received-grid tiles of the next round load (cp.async) while this round computes.
// Work item (segment j, cell lc of the chunk that starts at cell cell0).
template <int NL>
__device__ __forceinline__ void seg_prep_body(const Geo& g, int wmax, int cell0, int j, int lc,
                                              const phy_c32* __restrict__ anchors,
                                              const phy_c32* __restrict__ Y,
                                              float4* __restrict__ ygg, cf* __restrict__ bvec) {
  constexpr int NT = kPrepThreads;
  constexpr int NTRI = NL * (NL + 1) / 2;
  constexpr int LP = NL / 2;  // layer pairs
  static_assert(NT == 256, "two symbols of 128 threads per round");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  const int tid = threadIdx.x;
  const int cell = cell0 + lc;
  const int nr = g.n_rx, nl = g.n_layers, nds = g.n_dsym;
  const PrepLayout f = prep_layout(NL, g.n_dmrs, nr, wmax);
  cf* Cs = sm + f.off_C;
  cf* Xs = sm + f.off_X;
  int lo, hi;
  segment_range(g, j, lo, hi);
  const int W = hi - lo;
  const int nrounds = (nds + 1) / 2;

  // the two tiles of the current round
  auto tile = [&](int buf) { return sm + f.off_Y + buf * nr * f.yw; };
  auto load_round = [&](int n) {
    for (int s2 = 0; s2 < 2; ++s2) {
      const int jj = 2 * n + s2;
      if (jj >= nds) break;
      const phy_c32* ysym = Y + ((size_t)cell * g.n_sym + g.dsym[jj]) * nr * g.n_sc + lo;
      cf* dst = tile(s2);
      // row r, subcarrier pair p from the flat index without an integer division (exact:
      // the flat index is below 2^12)
      if ((lo & 1) == 0) {  // subcarrier pairs (a trailing odd one pairs with padding)
        const int wp = (W + 1) / 2;
        const float inv = 1.f / (float)wp;
        for (int e = tid; e < nr * wp; e += NT) {
          const int r = (int)(((float)e + 0.5f) * inv), kk = 2 * (e - r * wp);
          if (kk + 1 < W)
            cp_async16(dst + r * f.yw + kk, ysym + (size_t)r * g.n_sc + kk);
          else
            cp_async8(dst + r * f.yw + kk, ysym + (size_t)r * g.n_sc + kk);
        }
      } else {
        const float inv = 1.f / (float)W;
        for (int e = tid; e < nr * W; e += NT) {
          const int r = (int)(((float)e + 0.5f) * inv), kk = e - r * W;
          cp_async8(dst + r * f.yw + kk, ysym + (size_t)r * g.n_sc + kk);
        }
      }
    }
    cp_async_commit();
  };
  // ---- corners (asynchronous copies, transposed to [rx][corner-layer]), then round 0's tiles
  {
    const int g1 = seg_g1(g, j), warp = tid >> 5, lane = tid & 31;
    for (int cl = warp; cl < f.NC * NL; cl += NT / 32) {  // (corner, layer) per warp
      const int corner = cl / NL, l = cl % NL;
      const int d = corner >> 1, grp = (corner & 1) ? g1 : j;
      const phy_c32* src = anchors + ((((size_t)cell * g.n_dmrs + d) * g.G + grp) * nl + l) * nr;
      for (int r = lane; r < nr; r += 32) {
        cf* dst = Cs + r * f.xs + cl;
        if (l < nl)
          cp_async8(dst, src + r);
        else
          *dst = mk(0.f, 0.f);
      }
    }
    cp_async_commit();
  }
  load_round(0);  // overlaps the Gram work below
  cp_async_wait<1>();  // the corners
  __syncthreads();
  // ---- X = C^H C, lower 4x4 tiles
  {
    const int nt4 = f.NX / 4;
    const int n_lt = nt4 * (nt4 + 1) / 2;
    for (int t = tid; t < n_lt; t += NT) {
      int ti, tj;
      tri_decode(t, ti, tj);
      cf acc[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = mk(0.f, 0.f);
      for (int r = 0; r < nr; ++r) {
        const float4* row = reinterpret_cast<const float4*>(Cs + r * f.xs);
        const float4 a01 = row[2 * ti], a23 = row[2 * ti + 1];
        const float4 b01 = row[2 * tj], b23 = row[2 * tj + 1];
        const cf a[4] = {mk(a01.x, a01.y), mk(a01.z, a01.w), mk(a23.x, a23.y), mk(a23.z, a23.w)};
        const cf b[4] = {mk(b01.x, b01.y), mk(b01.z, b01.w), mk(b23.x, b23.y), mk(b23.z, b23.w)};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = cfma_cj(a[p], b[q], acc[p][q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) Xs[(4 * ti + p) * f.xs + 4 * tj + q] = acc[p][q];
    }
  }
  __syncthreads();
  // ---- Y_gg'(t), lower triangle, as 4-tuples (Y00, Y01, Y10, Y11) per (l, m)
  {
    auto Xget = [&](int i, int k) -> cf {
      if ((i >> 2) >= (k >> 2)) return Xs[i * f.xs + k];
      const cf v = Xs[k * f.xs + i];
      return mk(v.x, -v.y);
    };
    form_gram_blocks<NL, NT>(g, Xget, ygg + (((size_t)lc * g.n_seg + j) * nds) * NTRI * 2, tid);
  }
  __syncthreads();  // the X region now takes the rounds' interpolated channels
  cf* Hs = Xs;

  // ---- matched filter, two data symbols per round
  const int ks = tid & 3, slot = (tid & 127) >> 2, half = tid >> 7;
  const int nitems = ((W + 3) / 4) * LP;
  const int c1off = g.n_dmrs == 2 ? 2 * NL : 0;  // DMRS-1 corners (the DMRS-0 ones if single)
  for (int n = 0; n < nrounds; ++n) {
    // Hg(t) = C_0g + t1(t) (C_1g - C_0g) for the round's two symbols, while its tiles land
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const float t1 = g.tw[min(2 * n + s2, nds - 1)];
      for (int e = tid; e < nr * 2 * NL; e += NT) {
        const int r = e / (2 * NL), col = e % (2 * NL);  // 2 NL is a power of two
        const cf c0 = Cs[r * f.xs + col], c1 = Cs[r * f.xs + c1off + col];
        Hs[(s2 * nr + r) * f.hs + col] =
            mk(fmaf(t1, c1.x - c0.x, c0.x), fmaf(t1, c1.y - c0.y, c0.y));
      }
    }
    cp_async_wait<0>();
    __syncthreads();
    const int jj = 2 * n + half;
    if (jj < nds) {
      const cf* yt = tile(half);
      const cf* hg = Hs + half * nr * f.hs;
      cf* bout = bvec + ((size_t)(lc * nds + jj) * g.n_sc + lo) * NL;
      for (int it = slot; it < nitems; it += 32) {
        const int kq = it / LP, l0 = 2 * (it % LP), kk0 = 4 * kq;
        cf acc[2][2][4];  // [comb group][layer][RE]
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][b][q] = mk(0.f, 0.f);
#pragma unroll 4
        for (int r = ks; r < nr; r += 4) {
          const float4* yr = reinterpret_cast<const float4*>(yt + r * f.yw + kk0);
          const float4 y01 = yr[0], y23 = yr[1];
          const cf y[4] = {mk(y01.x, y01.y), mk(y01.z, y01.w), mk(y23.x, y23.y), mk(y23.z, y23.w)};
          const cf* hr = hg + r * f.hs + l0;
#pragma unroll
          for (int gg = 0; gg < 2; ++gg) {
            // interpolated channel of layers l0, l0 + 1 on comb group gg at this symbol
            const float4 hv = *reinterpret_cast<const float4*>(hr + gg * NL);
            const cf h[2] = {mk(hv.x, hv.y), mk(hv.z, hv.w)};
#pragma unroll
            for (int li = 0; li < 2; ++li)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[gg][li][q] = cfma_cj(h[li], y[q], acc[gg][li][q]);
          }
        }
        // sum the four antenna subsets: the four lanes of this item (same trip count, so the
        // mask names exactly the lanes that take part)
        const unsigned quad = 0xFu << (tid & 28);
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int m = 1; m < 4; m <<= 1) {
                acc[a][b][q].x += __shfl_xor_sync(quad, acc[a][b][q].x, m);
                acc[a][b][q].y += __shfl_xor_sync(quad, acc[a][b][q].y, m);
              }
        // lane ks writes RE kk0 + ks: b = (1 - beta) V_g0 + beta V_g1 for layers l0, l0 + 1
        const int kk = kk0 + ks;
        if (kk < W) {
          cf v[2];
#pragma unroll
          for (int li = 0; li < 2; ++li) {
            const float be = seg_beta(g, j, lo + kk, (l0 + li) & 1);
            cf z0 = acc[0][li][0], z1 = acc[1][li][0];
#pragma unroll
            for (int q = 1; q < 4; ++q)
              if (ks == q) {
                z0 = acc[0][li][q];
                z1 = acc[1][li][q];
              }
            v[li] = (1.f - be) * z0 + be * z1;
          }
          *reinterpret_cast<float4*>(bout + (size_t)kk * NL + l0) =
              make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        }
      }
    }
    __syncthreads();  // this round's tiles and channels are free
    if (n + 1 < nrounds) load_round(n + 1);
  }
}

template <int NL>
__global__ void __launch_bounds__(kPrepThreads)
    seg_prep_fp32_kernel(Geo g, int wmax, int cell0, const phy_c32* __restrict__ anchors,
                         const phy_c32* __restrict__ Y, float4* __restrict__ ygg,
                         cf* __restrict__ bvec) {
  seg_prep_body<NL>(g, wmax, cell0, blockIdx.x, blockIdx.y, anchors, Y, ygg, bvec);
}

// Thread-private scratch in shared memory, interleaved by thread (conflict-free) over the W
// threads of a solve CTA.
template <int W>
struct SmemScratch {
  cf* base;  // this thread's slot 0
  __device__ __forceinline__ void st(int e, cf v) const { base[e * W] = v; }
  __device__ __forceinline__ cf ld(int e) const { return base[e * W]; }
};



// The solver's 8x8 L21/T matrix of one thread in that scratch, entry (i, j) at slot 8 i + j.
template <int W>
struct SmemRows {
  SmemScratch<W> s;
  __device__ __forceinline__ void st_row(int i, const cf (&r)[8]) const {
#pragma unroll
    for (int j = 0; j < 8; ++j) s.st(kScrL21 + 8 * i + j, r[j]);
  }
  __device__ __forceinline__ void ld_row(int i, cf (&r)[8]) const {
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = s.ld(kScrL21 + 8 * i + j);
  }
  __device__ __forceinline__ void ld_col(int c, cf (&r)[8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = s.ld(kScrL21 + 8 * i + c);
  }
  __device__ __forceinline__ void sync_st() const {}
};

// The same matrix in tensor memory: the thread's own TMEM lane (lane quarter of its warp),
// 128 columns, entry (i, j) in columns 16 i + 2 j (real) and 16 i + 2 j + 1 (imaginary). Loads
// and stores are warp-collective (each access first reconverges the warp); a row is one
// 16-column access, a column eight 2-column ones.
struct TmemRows {
  uint32_t base;  // TMEM address of column 0 at the warp's first lane
  __device__ __forceinline__ void st_row(int i, const cf (&r)[8]) const {
    float v[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[2 * j] = r[j].x;
      v[2 * j + 1] = r[j].y;
    }
    __syncwarp();
    tc::tmem_st16(base + 16u * i, v);
  }
  __device__ __forceinline__ void ld_row(int i, cf (&r)[8]) const {
    float v[16];
    __syncwarp();
    tc::tmem_ld16(base + 16u * i, v);
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = mk(v[2 * j], v[2 * j + 1]);
  }
  __device__ __forceinline__ void ld_col(int c, cf (&r)[8]) const {
    float v[16];
    __syncwarp();
    tc::tmem_ld2x8(base + 2u * c, v);
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = mk(v[2 * i], v[2 * i + 1]);
  }
  __device__ __forceinline__ void sync_st() const {
    __syncwarp();
    tc::tmem_wait_st();
  }
};

// Gram-block bytes of one (segment, data symbol): NTRI 4-tuples of complex values.
constexpr uint32_t gram_block_bytes(int NL) { return (uint32_t)(NL * (NL + 1) / 2) * 32u; }

// The single-job solve with 9..16 layers and 128-RE CTAs keeps the solver's L21/T matrices in
// tensor memory (128 columns per CTA; this kernel issues no MMAs), which leaves shared memory to
// the Gram blocks and one 8-vector per thread: three CTAs (12 warps) fit an SM where the
// shared-memory form fits two. 64-RE CTAs keep the shared-memory form, and so does the batched
// solve: its persistent CTAs would hold tensor memory on every SM for the whole launch, while
// the other layer classes' tensor-core kernels, running next to it on forked streams, need 512
// columns of an SM at once (measured: a mixed serving batch lost more time waiting for those
// allocations than the faster solve gained).
constexpr bool solve_uses_tmem(int NL, int W) { return NL == 16 && W == 128; }
constexpr uint32_t kSolveTmemCols = 128;
constexpr int kSolveCarveoutSlack = 2;  // percent above the exact need
constexpr int solve_min_ctas(bool tm) { return tm ? 3 : 1; }

// The solve kernel's CTA width W (REs per CTA) is a tile shape the autotuner picks: 128 or 64;
// tm selects the tensor-memory form.
constexpr size_t solve_scratch_bytes(int NL, int W, bool tm) {
  return NL != 16 ? 0 : tm ? (size_t)8 * W * sizeof(cf) : (size_t)kScrSlots * W * sizeof(cf);
}

// 9..16 layers: after the solve, shared memory holds every thread's x and d in RE-major tables
// padded to 17 entries per RE, and one ok byte per RE (the transposed epilogue's input).
constexpr size_t solve_stage_bytes(int W = kSolveThreads) {
  return (size_t)W * 17 * (sizeof(cf) + sizeof(float)) + W;
}

// Shared memory of the solve kernel: scratch and the Gram blocks of up to max_segs segments (for
// 9..16 layers at least the epilogue's tables), then the mbarrier and the tensor-memory address
// in the last 16 bytes, which the tables never reach.
__host__ __device__ constexpr size_t solve_smem_bytes(int NL, int QM, int max_segs,
                                                      int W = kSolveThreads, bool tm = false) {
  const size_t main = solve_scratch_bytes(NL, W, tm) + (size_t)max_segs * gram_block_bytes(NL);
  const size_t stage = NL == 16 ? solve_stage_bytes(W) : 0;
  return (main > stage ? main : stage) + 16;
}

// One layer's LLR record (QM values at element index idx, a multiple of QM) to the output:
// FP32 in 16-byte pieces when QM is a multiple of 4 (the record is then 16-byte aligned), else in
// pairs; binary16 (rounded to nearest, saturating at +-65504) as one 16- or 8-byte piece for
// QM = 8 or 4, else in pairs.
template <int QM>
__device__ __forceinline__ void store_llr_record(float* base, size_t idx, const float (&v)[QM],
                                                 bool f16) {
  if (f16) {
    const float m = 65504.f;
    uint32_t w[QM / 2];
#pragma unroll
    for (int q = 0; q < QM; q += 2) {
      const __half2 h = __floats2half2_rn(fminf(fmaxf(v[q], -m), m), fminf(fmaxf(v[q + 1], -m), m));
      w[q / 2] = *reinterpret_cast<const uint32_t*>(&h);
    }
    __half* hb = reinterpret_cast<__half*>(base) + idx;
    if constexpr (QM == 8) {
      *reinterpret_cast<uint4*>(hb) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (QM == 4) {
      *reinterpret_cast<uint2*>(hb) = make_uint2(w[0], w[1]);
    } else {
#pragma unroll
      for (int q = 0; q < QM / 2; ++q) reinterpret_cast<uint32_t*>(hb)[q] = w[q];
    }
  } else if constexpr (QM % 4 == 0) {
#pragma unroll
    for (int q = 0; q < QM; q += 4)
      *reinterpret_cast<float4*>(base + idx + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < QM; q += 2)
      *reinterpret_cast<float2*>(base + idx + q) = make_float2(v[q], v[q + 1]);
  }
}

// LLRs of one layer (unbiased symbol xt; the layer's SINR gives the noise scale), or zeros when
// !ok, stored as the record of layer index li.
template <int QM>
__device__ __forceinline__ void demap_store(float* llr, size_t li, cf xt, float sinr, bool ok,
                                            bool f16) {
  float v[QM];
  if (ok) {
    qam_llr_scaled<QM>(xt, sinr * qam_inv_nrm2<QM>(), v);
  } else {
#pragma unroll
    for (int q = 0; q < QM; ++q) v[q] = 0.f;
  }
  store_llr_record<QM>(llr, li * QM, v, f16);
}
// As demap_store for a compile-time QM, or for QM = 0 the run-time qm.
template <int QM>
__device__ __forceinline__ void demap_store_q(int qm, float* llr, size_t li, cf xt, float sinr,
                                              bool ok, bool f16) {
  if constexpr (QM > 0) {
    demap_store<QM>(llr, li, xt, sinr, ok, f16);
  } else {
    switch (qm) {
      case 2: demap_store<2>(llr, li, xt, sinr, ok, f16); break;
      case 4: demap_store<4>(llr, li, xt, sinr, ok, f16); break;
      case 6: demap_store<6>(llr, li, xt, sinr, ok, f16); break;
      default: demap_store<8>(llr, li, xt, sinr, ok, f16); break;
    }
  }
}

// One CTA per (128 subcarriers, data symbol, cell), one thread per RE. Thread 0 brings the
// Gram-block 4-tuples of the segments the CTA spans into shared memory with bulk copies
// (TMA engine, completion counted on an mbarrier); meanwhile every thread loads its matched
// filter. A barrier timeout, here or in the segment kernel before (its error word), marks the
// CTA's REs with flag bit 3 and leaves their outputs unwritten. With 9..16 layers the SINR,
// unbiasing and demapping run transposed, one (RE, layer) item per thread and step, so that a
// warp's stores cover one contiguous stretch of each output: per-thread stores of whole records
// (512 B apart) would keep each warp waiting on the store path.
// Work item (128 subcarriers from k0 = bx 128, data symbol jj, cell lc of the chunk starting at
// cell0). The barrier `bar` is initialised and its phase `parity` is the one this item's copies
// complete; `tmem` is the CTA's tensor-memory allocation in the tensor-memory form TM. QM = 0
// takes the modulation from g.qm. Returns false if the Gram-block copies did not land even after
// a timeout's second wait (the barrier is then unusable for a later item).
template <int NL, int QM, int W = kSolveThreads, bool TM = false>
__device__ __forceinline__ bool re_solve_body(
    const Geo& g, int cell0, int bx, int jj, int lc, uint64_t* bar, uint32_t parity, uint32_t tmem,
    const float4* __restrict__ ygg, const cf* __restrict__ bvec,
    const float* __restrict__ sigma2, const phy_c32* __restrict__ anchors,
    const phy_c32* __restrict__ Y, phy_c32* __restrict__ x_hat, float* __restrict__ sinr_out,
    float* __restrict__ llr_out, uint8_t* __restrict__ flags_out,
    const unsigned* __restrict__ prep_err) {
  constexpr int NTRI = NL * (NL + 1) / 2;
  constexpr uint32_t kBlk = gram_block_bytes(NL);
  extern __shared__ __align__(128) unsigned char solve_smem[];
  float4* ys = reinterpret_cast<float4*>(solve_smem + solve_scratch_bytes(NL, W, TM));
  const int nl = g.n_layers, nds = g.n_dsym;
  const int qm = QM > 0 ? QM : g.qm;
  const int cell = cell0 + lc;
  const int k0 = bx * W;
  const int k = k0 + threadIdx.x;
  const bool live = k < g.n_sc;
  const int s0 = seg_of(g, k0), s1 = seg_of(g, min(k0 + W, g.n_sc) - 1);
  const int nseg = s1 - s0 + 1;  // <= max_segs (host-computed bound)
  if (threadIdx.x == 0) {
    tc::mbar_arrive_expect_tx(bar, (uint32_t)nseg * kBlk);
    for (int s = 0; s < nseg; ++s)
      tc::bulk_g2s(ys + (size_t)s * NTRI * 2,
                   ygg + (((size_t)lc * g.n_seg + s0 + s) * nds + jj) * NTRI * 2, kBlk, bar);
  }
  const size_t re = ((size_t)lc * nds + jj) * g.n_sc + (live ? k : k0);
  cf b[NL], x[NL];
  float dd[NL];
  bool fin = true;
  if (live) {
    const float4* bp = reinterpret_cast<const float4*>(bvec + re * NL);
#pragma unroll
    for (int l = 0; l < NL; l += 2) {
      const float4 v = __ldg(bp + l / 2);
      b[l] = mk(v.x, v.y);
      b[l + 1] = mk(v.z, v.w);
    }
  }
  bool arrived = tc::mbar_wait(bar, parity, g.wait_solve);
  // after a timeout, let the copies in flight land before the CTA can end
  const bool landed = arrived || tc::mbar_wait(bar, parity, kWaitSolveDefault);
  // one decision for the CTA (it has barriers below); a timed-out Gram/matched-filter kernel
  // (its error word) voids every RE as a wait timeout here would
  arrived = __syncthreads_and(arrived && (threadIdx.x != 0 || *prep_err == 0));
  const size_t ridx = ((size_t)cell * nds + jj) * g.n_sc + (live ? k : k0);
  if (!arrived) {
    if (live) flags_out[ridx] = 8;
    return __syncthreads_and(landed);
  }
  if (NL != 16 && !live) return true;
  const int j = seg_of(g, live ? k : k0);
  const float s2 = sigma2[cell];
  const int kc = live ? k : k0;
  const float be0 = seg_beta(g, j, kc, 0), be1 = seg_beta(g, j, kc, 1);
  const float4* yp = ys + (size_t)(j - s0) * NTRI * 2;
  // weight products w_g(comb l) w_g'(comb m) for the four comb pairs (cl, cm), built once
  float cw[2][2][4];
#pragma unroll
  for (int cl = 0; cl < 2; ++cl)
#pragma unroll
    for (int cm = 0; cm < 2; ++cm) {
      const float bl = cl ? be1 : be0, bm = cm ? be1 : be0;
      cw[cl][cm][0] = (1.f - bl) * (1.f - bm);
      cw[cl][cm][1] = (1.f - bl) * bm;
      cw[cl][cm][2] = bl * (1.f - bm);
      cw[cl][cm][3] = bl * bm;
    }
  auto getA = [&](int l, int m) -> cf {
    if (l >= nl || m >= nl) return (l == m) ? mk(1.f, 0.f) : mk(0.f, 0.f);
    const int e = tri(l, m);
    const float4 p = yp[2 * e], q = yp[2 * e + 1];
    // comb parities are compile-time except in the solver's rolled row loop (a select there)
    const bool ol = l & 1, om = m & 1;
    const float c00 = ol ? (om ? cw[1][1][0] : cw[1][0][0]) : (om ? cw[0][1][0] : cw[0][0][0]);
    const float c01 = ol ? (om ? cw[1][1][1] : cw[1][0][1]) : (om ? cw[0][1][1] : cw[0][0][1]);
    const float c10 = ol ? (om ? cw[1][1][2] : cw[1][0][2]) : (om ? cw[0][1][2] : cw[0][0][2]);
    const float c11 = ol ? (om ? cw[1][1][3] : cw[1][0][3]) : (om ? cw[0][1][3] : cw[0][0][3]);
    cf a;
    a.x = fmaf(c00, p.x, fmaf(c01, p.z, fmaf(c10, q.x, c11 * q.z)));
    a.y = fmaf(c00, p.y, fmaf(c01, p.w, fmaf(c10, q.y, c11 * q.w)));
    if (l == m) {
      a.x += s2;
      a.y = 0.f;
    }
    return a;
  };
  bool ok = false;
  // every thread of a warp takes part in the 9..16-layer solve (its tensor-memory accesses are
  // warp-collective); a thread past the carrier's end solves its block's first RE and discards it
  if (live || NL == 16) {
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      if (l >= nl || !live) b[l] = mk(0.f, 0.f);
      fin = fin && finite_cf(b[l]);
    }
    SolveInfo si;
    if constexpr (NL == 16) {
      // a runtime row of A: its entries (l, 0..7) are consecutive in the packed triangle, and
      // the comb parity of l picks the weight products once for the row
      auto rowA = [&](int l, cf (&row)[8]) {
        const float4* e0 = yp + 2 * tri(l, 0);
        const bool ol = l & 1, lv = l < nl;
        float ce[4], co[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ce[q] = ol ? cw[1][0][q] : cw[0][0][q];
          co[q] = ol ? cw[1][1][q] : cw[0][1][q];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float* c = (k & 1) ? co : ce;
          const float4 p = e0[2 * k], q = e0[2 * k + 1];
          cf a;
          a.x = fmaf(c[0], p.x, fmaf(c[1], p.z, fmaf(c[2], q.x, c[3] * q.z)));
          a.y = fmaf(c[0], p.y, fmaf(c[1], p.w, fmaf(c[2], q.y, c[3] * q.w)));
          row[k] = (lv && k < nl) ? a : mk(0.f, 0.f);  // l >= 8 > k: never on the diagonal
        }
      };
      cf* sb = reinterpret_cast<cf*>(solve_smem) + threadIdx.x;
      if constexpr (TM) {
        // the warp's lane quarter of the allocation: lane field 32 (warp mod 4) << 16
        const TmemRows rows{tmem + (((threadIdx.x >> 5) & 3u) << 21)};
        si = solve16(getA, rowA, SmemScratch<W>{sb}, rows, b, x, dd);
      } else {
        si = solve16(getA, rowA, SmemScratch<W>{sb + kScrV * W}, SmemRows<W>{SmemScratch<W>{sb}},
                     b, x, dd);
      }
    } else {
      si = solve_small<NL>(getA, b, x, dd);
    }
    fin = fin && si.fin;
    ok = si.ok && fin;
    uint8_t flag = 0;
    if (!fin) flag |= 4;
    if (!si.ok || si.pmin < g.pivot_min * si.pmax) flag |= 1;
    if (live && g.refactor && (flag & 1) && fin) {
      Refactor64Out r64;
      refactor_fp64(g, anchors, Y, cell, jj, k, j, s2, &r64);
      if (r64.ok) {
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          if (l < nl) {
            x[l] = r64.x[l];
            dd[l] = r64.d[l];
          }
        }
        ok = true;
        flag |= 2;
      }
    }
    if (live) flags_out[ridx] = flag;
  }
  if constexpr (NL == 16) {
    // Outputs leave in (RE, layer) order: once every thread is past the solve, each stages its
    // x and d in a padded RE-major table (stride 17: few bank conflicts both ways); then the
    // CTA's threads take the (RE, layer) items of its 128 REs in turn, consecutive lanes on
    // consecutive items, so every lane's LLR record (QM values), SINR and x_hat land right after
    // its neighbour's: the stores of a warp cover one contiguous stretch of each output.
    constexpr int kXs = NL + 1;
    cf* xs = reinterpret_cast<cf*>(solve_smem);
    float* ds = reinterpret_cast<float*>(solve_smem + (size_t)W * kXs * sizeof(cf));
    unsigned char* oks = reinterpret_cast<unsigned char*>(ds + W * kXs);
    __syncthreads();  // the scratch and the Gram blocks are dead from here on
    const int r = threadIdx.x;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      xs[r * kXs + l] = x[l];
      ds[r * kXs + l] = dd[l];
    }
    oks[r] = ok ? 1 : 0;
    __syncthreads();
    const int nlive = min(W, g.n_sc - k0);
    const size_t r0 = ((size_t)cell * nds + jj) * g.n_sc + k0;
#pragma unroll 2
    for (int it = threadIdx.x; it < nlive * nl; it += W) {
      const int re = nl == 16 ? (it >> 4) : it / nl, l = it - re * nl;
      const cf xl = xs[re * kXs + l];
      const bool okr = oks[re] != 0;
      const LayerOut o = layer_stats(s2, ds[re * kXs + l]);
      const size_t li = (r0 + re) * nl + l;
      if (llr_out) demap_store_q<QM>(qm, llr_out, li, o.inv_mu * xl, o.sinr, okr, g.llr_f16);
      if (sinr_out) sinr_out[li] = okr ? o.sinr : 0.f;
      if (x_hat) st(x_hat + li, okr ? xl : mk(0.f, 0.f));
    }
  } else {
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      if (l >= nl) continue;
      const LayerOut o = layer_stats(s2, dd[l]);
      const size_t li = ridx * nl + l;
      if (ok) {
        if (x_hat) st(x_hat + li, x[l]);
        if (sinr_out) sinr_out[li] = o.sinr;
        if (llr_out) demap_store_q<QM>(qm, llr_out, li, o.inv_mu * x[l], o.sinr, true, g.llr_f16);
      } else {
        if (x_hat) st(x_hat + li, mk(0.f, 0.f));
        if (sinr_out) sinr_out[li] = 0.f;
        if (llr_out) demap_store_q<QM>(qm, llr_out, li, mk(0.f, 0.f), 1.f, false, g.llr_f16);
      }
    }
  }
  return true;
}

// The CTA's tensor memory for the solver (the TM form): warp 0 allocates kSolveTmemCols
// columns into *slot before the CTA's first barrier, and releases them after its last one.
template <bool kTm>
__device__ __forceinline__ uint32_t solve_tmem_acquire(uint32_t* slot) {
  if constexpr (kTm) {
    if (threadIdx.x < 32) tc::tmem_alloc(slot, kSolveTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    return *slot;
  } else {
    __syncthreads();
    return 0;
  }
}
template <bool kTm>
__device__ __forceinline__ void solve_tmem_release(uint32_t tmem) {
  if constexpr (kTm) {
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
      tc::fence_after_sync();
      tc::tmem_dealloc(tmem, kSolveTmemCols);
    }
  }
}

template <int NL, int QM, int W>
__global__ void __launch_bounds__(W, solve_min_ctas(solve_uses_tmem(NL, W)))
    re_solve_fp32_kernel(Geo g, int cell0, int max_segs, const float4* __restrict__ ygg,
                         const cf* __restrict__ bvec, const float* __restrict__ sigma2,
                         const phy_c32* __restrict__ anchors, const phy_c32* __restrict__ Y,
                         phy_c32* __restrict__ x_hat, float* __restrict__ sinr_out,
                         float* __restrict__ llr_out, uint8_t* __restrict__ flags_out,
                         const unsigned* __restrict__ prep_err) {
  extern __shared__ __align__(128) unsigned char solve_smem[];
  constexpr bool kTm = solve_uses_tmem(NL, W);
  unsigned char* top = solve_smem + solve_smem_bytes(NL, QM, max_segs, W, kTm);
  uint64_t* bar = reinterpret_cast<uint64_t*>(top - 16);
  if (threadIdx.x == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_fence_init();
  }
  const uint32_t tmem = solve_tmem_acquire<kTm>(reinterpret_cast<uint32_t*>(top - 8));
  re_solve_body<NL, QM, W, kTm>(g, cell0, blockIdx.x, blockIdx.y, blockIdx.z, bar, 0, tmem, ygg, bvec,
                           sigma2, anchors, Y, x_hat, sinr_out, llr_out, flags_out, prep_err);
  solve_tmem_release<kTm>(tmem);
}

// ---------------------------------------------------------------- direct form, up to 4 layers
// With up to four layers the cover is at most 2 and the anchors change every 2L <= 4
// subcarriers, so a segment's corner cross-Gram is shared by too few REs to pay for a CTA. Here
// one thread takes one RE (subcarrier k, data symbol t) of one cell: per antenna it interpolates
// its channel row from the four corner anchors of its segment (frequency per comb, then time)
// and accumulates A = H^H H and b = H^H y directly, the plain definition. The solve, SINR, LLRs
// and the FP64 re-computation are those of the solve kernel. QM = 0 takes the modulation from
// g.qm.
//
// A CTA takes 128 consecutive subcarriers of one symbol. Their segments span at most
// 127 / (2L) + 3 anchor groups, so the CTA stages those groups' anchors in shared memory,
// kDirectRc antennas at a time, as [DMRS][layer][antenna][group]: a warp's 32 subcarriers read
// equal (broadcast) or consecutive groups, one wavefront per load, where reading the anchors from
// global memory touched one cache line per distinct segment. Global reads of the stage run over
// antennas (contiguous in the anchor layout).
constexpr int kDirectThreads = 128;
constexpr int kDirectRc = 16;  // antennas per staged chunk
// Anchor groups a CTA can need, for the smallest cover of the class (L >= NL / 2), odd so that
// the staging stores (stride: one antenna row of groups) spread over the banks.
template <int NL>
__host__ __device__ constexpr int direct_groups() {
  return (127 / NL + 3) | 1;
}
template <int NL>
__host__ __device__ constexpr int direct_stage_elems() {
  return 2 * NL * kDirectRc * direct_groups<NL>();
}

template <int NL, int QM>
__device__ __forceinline__ void direct_cta(const Geo& g, int k0, int t, int cell,
                                           const phy_c32* __restrict__ anchors,
                                           const phy_c32* __restrict__ Y,
                                           const float* __restrict__ sigma2,
                                           phy_c32* __restrict__ x_hat,
                                           float* __restrict__ sinr_out,
                                           float* __restrict__ llr_out,
                                           uint8_t* __restrict__ flags_out,
                                           cf* __restrict__ stage) {
  static_assert(NL <= 4, "the direct form keeps its sums in registers");
  constexpr int NTRI = NL * (NL + 1) / 2;
  constexpr int NGP = direct_groups<NL>();
  const int nr = g.n_rx, nl = g.n_layers, nds = g.n_dsym, nd = g.n_dmrs;
  const int qm = QM > 0 ? QM : g.qm;
  const int k = k0 + (int)threadIdx.x;
  const bool live = k < g.n_sc;
  const int kc = live ? k : g.n_sc - 1;
  const int j = seg_of(g, kc), g1 = seg_g1(g, j);
  // groups [gA, gB] cover every segment pair of the CTA's subcarriers (seg_of is monotone)
  const int gA = seg_of(g, k0);
  const int gB = seg_g1(g, seg_of(g, min(k0 + kDirectThreads - 1, g.n_sc - 1)));
  const int ng = gB - gA + 1;  // <= NGP since L >= NL / 2 (host-checked)
  const int lj = j - gA, lg1 = g1 - gA;
  const float bw[2] = {seg_beta(g, j, kc, 0), seg_beta(g, j, kc, 1)};
  const float tau = nd == 2 ? g.tw[t] : 0.f;
  cf A[NTRI], bv[NL];
#pragma unroll
  for (int e = 0; e < NTRI; ++e) A[e] = mk(0.f, 0.f);
#pragma unroll
  for (int l = 0; l < NL; ++l) bv[l] = mk(0.f, 0.f);
  const phy_c32* acell = anchors + (size_t)cell * nd * g.G * nl * nr;  // [d][group][l][r]
  const phy_c32* yk = Y + (((size_t)cell * g.n_sym + g.dsym[t]) * nr) * g.n_sc + kc;
  // this thread's received values of a chunk of antennas (zero past the last antenna)
  auto load_y = [&](int r0, cf(&dst)[kDirectRc]) {
#pragma unroll
    for (int rr = 0; rr < kDirectRc; ++rr)
      dst[rr] = (live && r0 + rr < nr) ? ld(yk + (size_t)(r0 + rr) * g.n_sc) : mk(0.f, 0.f);
  };
  // staging threads: 16 antennas (lanes of a half-warp) x 8 (DMRS, group) rows at a time
  constexpr int kQ = kDirectThreads / kDirectRc;
  const int rr_t = (int)threadIdx.x % kDirectRc, qs = (int)threadIdx.x / kDirectRc;
  cf yv[kDirectRc];
  load_y(0, yv);
  for (int r0 = 0; r0 < nr; r0 += kDirectRc) {
    const int rc = min(kDirectRc, nr - r0);
    __syncthreads();  // every thread is done with the previous chunk
    if (rr_t < rc) {
      for (int q = qs; q < nd * ng; q += kQ) {
        const int d = q >= ng ? 1 : 0, gl = q - d * ng;  // nd <= 2
        const phy_c32* src = acell + ((size_t)(d * g.G + gA + gl) * nl) * nr + r0 + rr_t;
        cf* dst = stage + ((d * NL) * kDirectRc + rr_t) * NGP + gl;
#pragma unroll
        for (int l = 0; l < NL; ++l)
          if (l < nl) dst[l * kDirectRc * NGP] = ld(src + (size_t)l * nr);
      }
    }
    __syncthreads();
    cf yn[kDirectRc];
    load_y(r0 + kDirectRc, yn);  // the next chunk's values load while this one is consumed
    if (live) {
#pragma unroll
      for (int rr = 0; rr < kDirectRc; ++rr) {
        if (rr < rc) {
          cf h[NL];
#pragma unroll
          for (int l = 0; l < NL; ++l) {
            h[l] = mk(0.f, 0.f);
            if (l < nl) {
              const float w1 = bw[l & 1], w0 = 1.f - w1;
              const cf* s0 = stage + (l * kDirectRc + rr) * NGP;
              const cf c0 = s0[lj], c1 = s0[lg1];
              cf v = mk(fmaf(w1, c1.x, w0 * c0.x), fmaf(w1, c1.y, w0 * c0.y));
              if (nd == 2) {
                const cf* s1 = s0 + NL * kDirectRc * NGP;
                const cf e0 = s1[lj], e1 = s1[lg1];
                const cf u = mk(fmaf(w1, e1.x, w0 * e0.x), fmaf(w1, e1.y, w0 * e0.y));
                v = mk(fmaf(tau, u.x - v.x, v.x), fmaf(tau, u.y - v.y, v.y));
              }
              h[l] = v;
            }
          }
          const cf y = yv[rr];
#pragma unroll
          for (int l = 0; l < NL; ++l) {
#pragma unroll
            for (int m = 0; m <= l; ++m) A[tri(l, m)] = cfma_cj(h[l], h[m], A[tri(l, m)]);
            bv[l] = cfma_cj(h[l], y, bv[l]);
          }
        }
      }
    }
#pragma unroll
    for (int rr = 0; rr < kDirectRc; ++rr) yv[rr] = yn[rr];
  }
  if (!live) return;
  const float s2 = sigma2[cell];
  auto getA = [&](int l, int m) -> cf {
    if (l >= nl || m >= nl) return (l == m) ? mk(1.f, 0.f) : mk(0.f, 0.f);
    // A holds sum conj(h_l) h_m: entry (l, m) of H^H H
    cf a = A[tri(l, m)];
    if (l == m) {
      a.x += s2;
      a.y = 0.f;
    }
    return a;
  };
  cf b[NL], x[NL];
  float dd[NL];
  bool fin = true;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    b[l] = l < nl ? bv[l] : mk(0.f, 0.f);
    fin = fin && finite_cf(b[l]);
  }
  const SolveInfo si = solve_small<NL>(getA, b, x, dd);
  fin = fin && si.fin;
  bool ok = si.ok && fin;
  uint8_t flag = 0;
  if (!fin) flag |= 4;
  if (!si.ok || si.pmin < g.pivot_min * si.pmax) flag |= 1;
  if (g.refactor && (flag & 1) && fin) {
    Refactor64Out r64;
    refactor_fp64(g, anchors, Y, cell, t, k, j, s2, &r64);
    if (r64.ok) {
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        if (l < nl) {
          x[l] = r64.x[l];
          dd[l] = r64.d[l];
        }
      }
      ok = true;
      flag |= 2;
    }
  }
  const size_t ridx = ((size_t)cell * nds + t) * g.n_sc + k;
  flags_out[ridx] = flag;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    if (l >= nl) continue;
    const LayerOut o = layer_stats(s2, dd[l]);
    const size_t li = ridx * nl + l;
    if (x_hat) st(x_hat + li, ok ? x[l] : mk(0.f, 0.f));
    if (sinr_out) sinr_out[li] = ok ? o.sinr : 0.f;
    if (llr_out)
      demap_store_q<QM>(qm, llr_out, li, ok ? o.inv_mu * x[l] : mk(0.f, 0.f), o.sinr, ok,
                        g.llr_f16);
  }
}

template <int NL, int QM>
__global__ void __launch_bounds__(kDirectThreads)
    direct_fp32_kernel(Geo g, const phy_c32* __restrict__ anchors, const phy_c32* __restrict__ Y,
                       const float* __restrict__ sigma2, phy_c32* __restrict__ x_hat,
                       float* __restrict__ sinr_out, float* __restrict__ llr_out,
                       uint8_t* __restrict__ flags_out) {
  __shared__ cf stage[direct_stage_elems<NL>()];
  direct_cta<NL, QM>(g, blockIdx.x * kDirectThreads, blockIdx.y, blockIdx.z, anchors, Y, sigma2,
                     x_hat, sinr_out, llr_out, flags_out, stage);
}

// Batched direct form: CTAs stride over the (128 subcarriers, data symbol, cell) items of the
// class's jobs.
template <int NL>
__global__ void __launch_bounds__(kDirectThreads)
    direct_batch_kernel(const BatchTable* __restrict__ t) {
  __shared__ Geo sg;
  __shared__ cf stage[direct_stage_elems<NL>()];
  __shared__ BatchIndex ix;
  constexpr int cls = batch_class(NL);
  const int n = t->n_items[kBatchDirect][cls];
  // items strided over the CTAs (a job's items spread over the grid: balanced whatever the mix
  // of light and heavy jobs); a CTA keeps the geometry while consecutive items share a job
  if ((int)blockIdx.x >= n) return;
  batch_index_load(ix, t, kBatchDirect, cls);
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
    const int nb = (sg.n_sc + kDirectThreads - 1) / kDirectThreads;
    const int k0 = (local % nb) * kDirectThreads;
    const int jj = (local / nb) % sg.n_dsym, cell = local / (nb * sg.n_dsym);
    direct_cta<NL, 0>(sg, k0, jj, cell, J.anchors, J.Y, J.sigma2, J.x_hat, J.sinr, J.llr,
                      J.flags, stage);
    __syncthreads();
  }
}

// Batched forms (one launch per layer class serves every job of that class in the table).
// Segment stage: CTAs stride over the (segment, cell) items of the class's jobs.
template <int NL>
__global__ void __launch_bounds__(kPrepThreads)
    seg_prep_batch_kernel(const BatchTable* __restrict__ t) {
  __shared__ Geo sg;
  __shared__ BatchIndex ix;
  constexpr int cls = batch_class(NL);
  const int n = t->n_items[kBatchSeg][cls];
  if ((int)blockIdx.x >= n) return;
  batch_index_load(ix, t, kBatchSeg, cls);
  __syncthreads();
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    int local;
    const BatchJob& J = t->job[batch_find(ix, w, local)];
    batch_load_geo(sg, J.g);
    __syncthreads();
    seg_prep_body<NL>(sg, J.wmax, 0, local % sg.n_seg, local / sg.n_seg, J.anchors, J.Y, J.ygg,
                      J.bvec);
    __syncthreads();
  }
}

// Solve stage: CTAs stride over the (128 subcarriers, data symbol, cell) items of the class's
// jobs; one mbarrier per CTA counts every item's Gram-block copies, item i completing phase
// i mod 2. The modulation is each job's own (run-time QM).
template <int NL>
__global__ void __launch_bounds__(kSolveThreads)
    re_solve_batch_kernel(const BatchTable* __restrict__ t, int smem_bytes) {
  extern __shared__ __align__(128) unsigned char solve_smem[];
  __shared__ Geo sg;
  __shared__ BatchIndex ix;
  constexpr int cls = batch_class(NL);
  const int n = t->n_items[kBatchSolve][cls];
  if ((int)blockIdx.x >= n) return;
  uint64_t* bar = reinterpret_cast<uint64_t*>(solve_smem + smem_bytes - 16);
  if (threadIdx.x == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_fence_init();
  }
  batch_index_load(ix, t, kBatchSolve, cls);
  __syncthreads();
  uint32_t it = 0;
  for (int w = blockIdx.x; w < n; w += gridDim.x, ++it) {
    int local;
    const BatchJob& J = t->job[batch_find(ix, w, local)];
    batch_load_geo(sg, J.g);
    // the previous item's generic accesses to shared memory come before this item's bulk copies
    if (threadIdx.x == 0) tc::fence_proxy_async();
    __syncthreads();
    const int nb = (sg.n_sc + kSolveThreads - 1) / kSolveThreads;
    const int bx = local % nb, jj = (local / nb) % sg.n_dsym, lc = local / (nb * sg.n_dsym);
    const bool usable = re_solve_body<NL, 0>(sg, 0, bx, jj, lc, bar, it & 1, 0, J.ygg, J.bvec,
                                             J.sigma2, J.anchors, J.Y, J.x_hat, J.sinr, J.llr,
                                             J.flags, J.err);
    if (!__syncthreads_and(usable)) break;  // copies still in flight: the barrier is unusable
  }
}

struct Sizes {
  int NL, ntri;
  size_t ygg_per_cell, b_per_cell;
  int chunk;  // cells per chunk
};

Sizes sizes(const Geo& g, int chunk) {
  Sizes s;
  s.NL = nl_class(g.n_layers);
  s.ntri = s.NL * (s.NL + 1) / 2;
  s.ygg_per_cell = (size_t)g.n_seg * g.n_dsym * s.ntri * 32;
  s.b_per_cell = (size_t)g.n_dsym * g.n_sc * s.NL * 8;
  s.chunk = chunk;
  return s;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Most frequency segments any block of w consecutive subcarriers touches.
int max_segments_per_block(const Geo& g, int w = kSolveThreads) {
  if (g.G == 1) return 1;
  auto seg = [&](int k) {
    int j = (k - g.L) / (2 * g.L);
    if (k < g.L) j = 0;
    return std::min(j, g.n_seg - 1);
  };
  int best = 1;
  for (int k0 = 0; k0 < g.n_sc; k0 += w)
    best = std::max(best, seg(std::min(k0 + w, g.n_sc) - 1) - seg(k0) + 1);
  return best;
}

// error counter of the tensor-core kernels, then the two intermediates for `chunk` cells
size_t scratch_bytes(const Sizes& s, int chunk) {
  return 256 + align256(s.ygg_per_cell * chunk) + align256(s.b_per_cell * chunk);
}

// Shared-memory carveout (percent of the SM's maximum) that holds min_ctas CTAs of `smem` bytes
// (plus the 1 KB the runtime reserves per CTA): the rest of the SM's on-chip memory stays L1
// cache, which holds the register spills of the 12-warp form. Shared-memory-bound forms take all.
int solve_carveout(size_t smem, int min_ctas) {
  if (min_ctas <= 1) return 100;
  static int per_sm[kMaxDevices] = {};
  int& cap = per_sm[current_device()];
  if (cap == 0 && (cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                          current_device()) != cudaSuccess ||
                   cap <= 0))
    cap = 228 * 1024;
  const size_t need = (size_t)min_ctas * (smem + 1024);
  return std::min(100, (int)((100 * need + cap - 1) / cap) + kSolveCarveoutSlack);
}

template <int NL, int QM, int W>
cudaError_t launch_solve_w(const Geo& g, int c0, int nc, const float4* ygg, const cf* bvec,
                           const float* sigma2, const phy_c32* anchors, const phy_c32* Y,
                           phy_c32* x_hat, float* sinr, float* llr, uint8_t* flags,
                           const unsigned* err, cudaStream_t st) {
  const int max_segs = max_segments_per_block(g, W);
  const size_t smem = solve_smem_bytes(NL, QM, max_segs, W, solve_uses_tmem(NL, W));
  static size_t configured_on[kMaxDevices] = {};
  size_t& configured = configured_on[current_device()];
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(re_solve_fp32_kernel<NL, QM, W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(re_solve_fp32_kernel<NL, QM, W>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             solve_carveout(smem, solve_min_ctas(solve_uses_tmem(NL, W))));
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  dim3 grid((g.n_sc + W - 1) / W, g.n_dsym, nc);
  re_solve_fp32_kernel<NL, QM, W><<<grid, W, smem, st>>>(
      g, c0, max_segs, ygg, bvec, sigma2, anchors, Y, x_hat, sinr, llr, flags, err);
  return cudaGetLastError();
}

// The solve kernel with CTA width w (128 or 64 REs per CTA).
template <int NL, int QM>
cudaError_t launch_solve(const Geo& g, int w, int c0, int nc, const float4* ygg, const cf* bvec,
                         const float* sigma2, const phy_c32* anchors, const phy_c32* Y,
                         phy_c32* x_hat, float* sinr, float* llr, uint8_t* flags,
                         const unsigned* err, cudaStream_t st) {
  if (w == 64)
    return launch_solve_w<NL, QM, 64>(g, c0, nc, ygg, bvec, sigma2, anchors, Y, x_hat, sinr, llr,
                                      flags, err, st);
  return launch_solve_w<NL, QM, 128>(g, c0, nc, ygg, bvec, sigma2, anchors, Y, x_hat, sinr, llr,
                                     flags, err, st);
}

template <int NL>
cudaError_t launch_direct(const Geo& g, const phy_c32* anchors, const phy_c32* Y,
                          const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                          uint8_t* flags, cudaStream_t st) {
  if (2 * g.L < NL) return cudaErrorInvalidValue;  // the anchor stage is sized for L >= NL / 2
  dim3 grid((g.n_sc + kDirectThreads - 1) / kDirectThreads, g.n_dsym, g.n_cells);
  switch (g.qm) {
    case 2: direct_fp32_kernel<NL, 2><<<grid, kDirectThreads, 0, st>>>(g, anchors, Y, sigma2, x_hat, sinr, llr, flags); break;
    case 4: direct_fp32_kernel<NL, 4><<<grid, kDirectThreads, 0, st>>>(g, anchors, Y, sigma2, x_hat, sinr, llr, flags); break;
    case 6: direct_fp32_kernel<NL, 6><<<grid, kDirectThreads, 0, st>>>(g, anchors, Y, sigma2, x_hat, sinr, llr, flags); break;
    default: direct_fp32_kernel<NL, 8><<<grid, kDirectThreads, 0, st>>>(g, anchors, Y, sigma2, x_hat, sinr, llr, flags); break;
  }
  return cudaGetLastError();
}

template <int NL>
cudaError_t run_chunks(const Geo& g, int wmax, const Sizes& s, const phy_c32* anchors,
                       const phy_c32* Y, const float* sigma2, phy_c32* x_hat, float* sinr,
                       float* llr, uint8_t* flags, void* scratch, int stages, cudaStream_t st) {
  const PrepLayout f = prep_layout(NL, g.n_dmrs, g.n_rx, wmax);
  const size_t smem = (size_t)f.total * sizeof(cf);
  static size_t configured_on[kMaxDevices] = {};
  size_t& configured = configured_on[current_device()];
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(seg_prep_fp32_kernel<NL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(seg_prep_fp32_kernel<NL>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  char* base = static_cast<char*>(scratch);
  unsigned* err = reinterpret_cast<unsigned*>(base);
  float4* ygg = reinterpret_cast<float4*>(base + 256);
  cf* bvec = reinterpret_cast<cf*>(base + 256 + align256(s.ygg_per_cell * s.chunk));
  for (int c0 = 0; c0 < g.n_cells; c0 += s.chunk) {
    const int nc = std::min(s.chunk, g.n_cells - c0);
    cudaError_t e = cudaSuccess;
    // the segment kernels' error word (bumped by a timed-out wait), read by the solve kernel
    if ((stages & kStageGramMf) &&
        (e = cudaMemsetAsync(err, 0, sizeof(unsigned), st)) != cudaSuccess)
      return e;
    if ((stages & kStageGramMf) && g.prec == PHY_PREC_FP32) {
      dim3 grid(g.n_seg, nc);
      seg_prep_fp32_kernel<NL><<<grid, kPrepThreads, smem, st>>>(g, wmax, c0, anchors, Y, ygg,
                                                                bvec);
    } else if (stages & kStageGramMf) {
      e = launch_seg_prep_tc(g, NL, c0, nc, anchors, Y, ygg, bvec, err, st);
      if (e != cudaSuccess) return e;
    }
    if (!(stages & kStageSolve)) continue;
    const int w = tuned_tile(g).solve_w == 64 ? 64 : kSolveThreads;
    switch (g.qm) {
      case 2: e = launch_solve<NL, 2>(g, w, c0, nc, ygg, bvec, sigma2, anchors, Y, x_hat, sinr,
                                      llr, flags, err, st); break;
      case 4: e = launch_solve<NL, 4>(g, w, c0, nc, ygg, bvec, sigma2, anchors, Y, x_hat, sinr,
                                      llr, flags, err, st); break;
      case 6: e = launch_solve<NL, 6>(g, w, c0, nc, ygg, bvec, sigma2, anchors, Y, x_hat, sinr,
                                      llr, flags, err, st); break;
      default: e = launch_solve<NL, 8>(g, w, c0, nc, ygg, bvec, sigma2, anchors, Y, x_hat, sinr,
                                       llr, flags, err, st); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace

int nl_class_of(int n_layers) { return nl_class(n_layers); }
int batch_direct_class(int nl_cls) { return nl_cls <= 4 ? 1 : 0; }

// ---------------------------------------------------------------- batched receiver, host side
int batch_wmax(const Geo& g) { return host_max_segment_width(g); }
int batch_max_segs(const Geo& g) { return max_segments_per_block(g); }
size_t batch_ygg_bytes(const Geo& g) { return sizes(g, 1).ygg_per_cell * g.n_cells; }
size_t batch_bvec_bytes(const Geo& g) { return sizes(g, 1).b_per_cell * g.n_cells; }

namespace {

// Shared memory and persistent grids of one layer class's batched kernels, bounded over every
// geometry the batched path accepts for that class (automatic cover length, 1..275 PRB, one or
// two DMRS symbols, up to 64 antennas), so that one captured launch serves any batch.
struct BatchClassLaunch {
  size_t smem_seg = 0, smem_solve = 0;
  int grid_seg = 0, grid_solve = 0, grid_direct = 0;
};

// Shared-memory bounds of one class (pure host arithmetic, no CUDA call).
template <int NL>
BatchClassLaunch batch_class_smem() {
  static const BatchClassLaunch b = [] {
    BatchClassLaunch r;
    const int L = NL <= 2 ? 1 : NL / 2;  // the automatic cover of the class's layer counts
    int wmax = 1, msegs = 1;
    for (int prb = 1; prb <= 275; ++prb) {
      Geo g{};
      g.n_sc = 12 * prb;
      g.n_comb = g.n_sc / 2;
      g.L = L;
      if (g.n_comb < L) continue;
      g.G = (g.n_comb + L - 1) / L;
      g.n_seg = g.G > 1 ? g.G - 1 : 1;
      wmax = std::max(wmax, host_max_segment_width(g));
      msegs = std::max(msegs, max_segments_per_block(g));
    }
    r.smem_seg = (size_t)prep_layout(NL, 2, kMaxRx, wmax).total * sizeof(cf);
    r.smem_solve = solve_smem_bytes(NL, 0, msegs);
    return r;
  }();
  return b;
}

// The bounds plus persistent grids filling every SM at the kernels' occupancy (per device).
template <int NL>
BatchClassLaunch batch_class_launch() {
  static BatchClassLaunch on[kMaxDevices];
  BatchClassLaunch& b = on[current_device()];
  if (b.grid_seg > 0) return b;
  b = batch_class_smem<NL>();
  const int sms = device_sm_count();
  int occ = 0;
  cudaFuncSetAttribute(seg_prep_batch_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)b.smem_seg);
  cudaFuncSetAttribute(re_solve_batch_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)b.smem_solve);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, seg_prep_batch_kernel<NL>, kPrepThreads,
                                                    b.smem_seg) != cudaSuccess || occ < 1)
    occ = 1;
  b.grid_seg = sms * occ;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, re_solve_batch_kernel<NL>,
                                                    kSolveThreads, b.smem_solve) != cudaSuccess ||
      occ < 1)
    occ = 1;
  b.grid_solve = sms * occ;
  if constexpr (NL <= 4) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, direct_batch_kernel<NL>,
                                                      kDirectThreads, 0) != cudaSuccess ||
        occ < 1)
      occ = 1;
    b.grid_direct = 2 * sms * occ;  // two waves: CTAs that finish early take the next ones
  }
  cudaGetLastError();
  return b;
}

// One layer class: the direct form (FP32, <= 4 layers), the FP32 segment kernel (>= 5
// layers), the tensor-core segment kernel (FP16 jobs), then the solve of every job that went
// through a segment kernel. Empty stages exit at once.
template <int NL>
cudaError_t launch_batch_nl(const BatchTable* t, cudaStream_t st) {
  const BatchClassLaunch b = batch_class_launch<NL>();
  if constexpr (NL <= 4) {
    direct_batch_kernel<NL><<<b.grid_direct, kDirectThreads, 0, st>>>(t);
  } else {
    seg_prep_batch_kernel<NL><<<b.grid_seg, kPrepThreads, b.smem_seg, st>>>(t);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_seg_prep_tc_batch(t, NL, st)) != cudaSuccess) return e;
  re_solve_batch_kernel<NL><<<b.grid_solve, kSolveThreads, b.smem_solve, st>>>(
      t, (int)b.smem_solve);
  return cudaGetLastError();
}

}  // namespace

bool batch_geometry_fits(const Geo& g) {
  const int NL = nl_class(g.n_layers);
  size_t seg = 0, solve = 0;
  BatchClassLaunch b;
  switch (NL) {
    case 2: b = batch_class_smem<2>(); break;
    case 4: b = batch_class_smem<4>(); break;
    case 8: b = batch_class_smem<8>(); break;
    default: b = batch_class_smem<16>(); break;
  }
  seg = b.smem_seg;
  solve = b.smem_solve;
  const PrepLayout f = prep_layout(NL, g.n_dmrs, g.n_rx, host_max_segment_width(g));
  return (size_t)f.total * sizeof(cf) <= seg &&
         solve_smem_bytes(NL, 0, max_segments_per_block(g)) <= solve;
}

bool batch_solve_fits(const Geo& g) {
  const int NL = nl_class(g.n_layers);
  BatchClassLaunch b;
  switch (NL) {
    case 2: b = batch_class_smem<2>(); break;
    case 4: b = batch_class_smem<4>(); break;
    case 8: b = batch_class_smem<8>(); break;
    default: b = batch_class_smem<16>(); break;
  }
  return solve_smem_bytes(NL, 0, max_segments_per_block(g)) <= b.smem_solve;
}

namespace {

// Side streams on which the batched receiver runs three of its four layer classes next to the
// fourth (per device, created on the first launch that is not being captured; a launch captured
// before that runs the classes one after another on the caller's stream).
struct BatchFork {
  cudaStream_t s[3] = {};
  cudaEvent_t fork = nullptr, join[3] = {};
  bool ok = false;
};
std::mutex g_fork_mu;  // one fork/join sequence at a time (the events are shared)

BatchFork& batch_fork(bool may_create) {
  static BatchFork on[kMaxDevices];
  BatchFork& f = on[current_device()];
  if (f.ok || !may_create) return f;
  bool ok = cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 3 && ok; ++i)
    ok = cudaStreamCreateWithFlags(&f.s[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&f.join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) cudaGetLastError();
  f.ok = ok;
  return f;
}

}  // namespace

// The layer classes are independent once the LS stage is done: each runs its chain (direct
// form, or segment kernels then solve) on its own stream, forked from and joined back into the
// caller's, so that a batch's critical path is its longest chain, not the sum of the four.
cudaError_t launch_batch_stages(const BatchTable* t, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_fork_mu);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;
  }
  BatchFork& f = batch_fork(cs == cudaStreamCaptureStatusNone);
  cudaError_t e;
  if (!f.ok) {
    if ((e = launch_batch_nl<2>(t, st)) != cudaSuccess) return e;
    if ((e = launch_batch_nl<4>(t, st)) != cudaSuccess) return e;
    if ((e = launch_batch_nl<8>(t, st)) != cudaSuccess) return e;
    return launch_batch_nl<16>(t, st);
  }
  if ((e = cudaEventRecord(f.fork, st)) != cudaSuccess) return e;
  for (int i = 0; i < 3; ++i)
    if ((e = cudaStreamWaitEvent(f.s[i], f.fork, 0)) != cudaSuccess) return e;
  if ((e = launch_batch_nl<2>(t, f.s[0])) != cudaSuccess) return e;
  if ((e = launch_batch_nl<4>(t, f.s[1])) != cudaSuccess) return e;
  if ((e = launch_batch_nl<8>(t, f.s[2])) != cudaSuccess) return e;
  if ((e = launch_batch_nl<16>(t, st)) != cudaSuccess) return e;
  for (int i = 0; i < 3; ++i) {
    if ((e = cudaEventRecord(f.join[i], f.s[i])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, f.join[i], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int host_max_segment_width(const Geo& g) {
  auto start = [&](int grp) { return std::min(g.L * grp, g.n_comb - g.L); };
  auto pos1 = [&](int grp) { return 2 * start(grp) + g.L; };
  if (g.G == 1) return g.n_sc;
  int w = 0;
  for (int j = 0; j < g.G - 1; ++j) {
    int lo = (j == 0) ? 0 : pos1(j);
    int hi = (j == g.G - 2) ? g.n_sc : pos1(j + 1);
    w = std::max(w, hi - lo);
  }
  return w;
}

size_t fused_fp32_smem_bytes(const Geo& g) {
  const PrepLayout f =
      prep_layout(nl_class(g.n_layers), g.n_dmrs, g.n_rx, host_max_segment_width(g));
  return (size_t)f.total * sizeof(cf);
}

size_t detect_scratch_bytes(const Geo& g, int chunk) {
  return scratch_bytes(sizes(g, chunk), std::min(std::max(chunk, 1), g.n_cells));
}

int detect_preferred_chunk(const Geo& g) {
  const Sizes s = sizes(g, 1);
  const size_t per = s.ygg_per_cell + s.b_per_cell;
  return (int)std::min<size_t>(std::max<size_t>(1, chunk_budget() / per), (size_t)g.n_cells);
}

cudaError_t launch_detect(const Geo& g, const phy_c32* anchors, const phy_c32* Y,
                          const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                          uint8_t* flags, void* scratch, size_t scratch_bytes_avail, int stages,
                          cudaStream_t st) {
  const int wmax = host_max_segment_width(g);
  // the largest chunk of cells (up to the tuned or preferred one) whose intermediates fit the
  // scratch; a single stage needs the whole batch in one chunk
  const int tuned = tuned_tile(g).chunk;
  int chunk = stages != (kStageGramMf | kStageSolve) ? g.n_cells
              : tuned > 0                            ? std::min(tuned, g.n_cells)
                                                     : detect_preferred_chunk(g);
  Sizes s = sizes(g, chunk);
  while (chunk > 1 && scratch_bytes(s, chunk) > scratch_bytes_avail) s = sizes(g, --chunk);
  if (scratch_bytes(s, chunk) > scratch_bytes_avail) return cudaErrorInvalidValue;
  // a single stage is only meaningful when the whole batch is one chunk
  if (stages != (kStageGramMf | kStageSolve) && chunk != g.n_cells) return cudaErrorInvalidValue;
  // FP32 products with up to four layers: the direct form does everything in the solve stage
  if (g.prec == PHY_PREC_FP32 && s.NL <= 4) {
    if (!(stages & kStageSolve)) return cudaSuccess;
    return s.NL == 2 ? launch_direct<2>(g, anchors, Y, sigma2, x_hat, sinr, llr, flags, st)
                     : launch_direct<4>(g, anchors, Y, sigma2, x_hat, sinr, llr, flags, st);
  }
  switch (s.NL) {
    case 2:
      return run_chunks<2>(g, wmax, s, anchors, Y, sigma2, x_hat, sinr, llr, flags, scratch,
                           stages, st);
    case 4:
      return run_chunks<4>(g, wmax, s, anchors, Y, sigma2, x_hat, sinr, llr, flags, scratch,
                           stages, st);
    case 8:
      return run_chunks<8>(g, wmax, s, anchors, Y, sigma2, x_hat, sinr, llr, flags, scratch,
                           stages, st);
    default:
      return run_chunks<16>(g, wmax, s, anchors, Y, sigma2, x_hat, sinr, llr, flags, scratch,
                            stages, st);
  }
}

}  // namespace phy
