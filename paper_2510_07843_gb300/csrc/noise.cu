// Noise-variance estimate from the DMRS anchor residuals. The paper takes the noise level as a
// known input of the LMMSE block (Sec. IV); this is the step in front of it.
//
// Residuals of the LS anchors H_d,l(g, r) (anchors[cell][d][g][l][r]):
//   frequency  e = H_d,l(g) - a_g H_d,l(g-1) - b_g H_d,l(g+1), interior g = 1 .. G-2, every d,
//              with a_g, b_g the weights of the linear interpolation between the neighbours'
//              anchor subcarriers evaluated at anchor g's;
//   time       e = H_0,l(g) - H_1,l(g), every g (two DMRS symbols).
// Each residual is a fixed linear function sum_k c_k Y(k) of DMRS REs; white noise of variance s2
// per RE leaves E|e|^2 = s2 gamma, gamma = sum_k |c_k|^2 with c_k = (1/L) conj(P(k)) times the
// signed weight of the group(s) holding k. s2_hat = sum |e|^2 / (n_rx sum gamma), per mode; the
// "min" mode keeps the smaller of the two (channel variation only ever adds to either).
//
// Two kernels. noise_partial_kernel: CTA per (1024 anchor entries of one cell); each thread
// takes four entries (coalesced over the antenna index) and both residual kinds, and the CTA
// also sums the gains of the (group, layer) pairs whose first antenna entry it owns, one work
// item per (pair, comb index of the pair's span) so that every thread shares that part; one
// float4 of partial sums per CTA. noise_final_kernel: CTA per cell, sums the partials in a fixed
// order (FP64) and divides (with alpha < 1 it blends the estimate into the cell's tracked value,
// alpha est + (1 - alpha) prior); it is launched as a programmatic dependent of the first (it
// starts while the first drains and waits on griddepcontrol before reading). No atomics: the
// result does not depend on scheduling.
#include <math.h>

#include "batch.cuh"
#include "launch.h"

namespace phy {

namespace {

constexpr int kNoiseThreads = 256;
constexpr int kNoiseItems = 4;  // anchor entries per thread
constexpr int kNoiseEntries = kNoiseThreads * kNoiseItems;

// Weights (a_g, b_g) of anchors g-1 and g+1 in the linear prediction of interior anchor g. The
// anchor subcarriers of the two combs differ by one, so the weights are the same on both.
__device__ __forceinline__ float2 neighbour_weights(const Geo& g, int grp) {
  const int p0 = anchor_pos(g, grp - 1, 0), p1 = anchor_pos(g, grp, 0);
  const int p2 = anchor_pos(g, grp + 1, 0);
  const float span = (float)(p2 - p0);
  return make_float2((float)(p2 - p1) / span, (float)(p1 - p0) / span);
}

__device__ __forceinline__ float pilot_pow(const phy_c32* p) { return cabs2(ld(p)); }

// a / b for 0 <= a < 2^24 and b >= 1 without an integer division: the float estimate is off by
// at most one, which the two corrections remove.
__device__ __forceinline__ int div_small(int a, int b, float inv_b) {
  int q = __float2int_rz((float)a * inv_b);
  if (q * b > a) --q;
  if ((q + 1) * b <= a) ++q;
  return q;
}

// Partial sums of block `blk` (of n_blk) of one cell's anchor entries; every thread of the CTA
// calls it. red: CTA scratch of kNoiseThreads / 32 float4.
__device__ __forceinline__ void noise_partial_body(const Geo& g, int cell, int blk, int n_blk,
                                                   const phy_c32* __restrict__ anchors,
                                                   const phy_c32* __restrict__ pilots,
                                                   float4* __restrict__ part,
                                                   float4* __restrict__ red) {
  const int nl = g.n_layers, nr = g.n_rx;
  const int per_grp = nl * nr;                  // entries between neighbouring groups
  const int per_d = g.G * per_grp;              // entries of one DMRS symbol
  const phy_c32* A0 = anchors + (size_t)cell * g.n_dmrs * per_d;
  const phy_c32* A1 = A0 + (g.n_dmrs == 2 ? per_d : 0);
  const int i0 = blk * kNoiseEntries;
  const int i1 = min(i0 + kNoiseEntries, per_d);
  const float inv_grp = 1.f / (float)per_grp;
  float ef = 0.f, et = 0.f, gf = 0.f, gt = 0.f;

  // ---- residual energies, entry i = (group * nl + layer) * nr + antenna
#pragma unroll
  for (int it = 0; it < kNoiseItems; ++it) {
    const int i = i0 + it * kNoiseThreads + threadIdx.x;
    if (i < i1) {
      const int grp = div_small(i, per_grp, inv_grp);
      const cf h0 = ld(A0 + i);
      if (g.n_dmrs == 2) et += cabs2(h0 - ld(A1 + i));
      if (grp >= 1 && grp <= g.G - 2) {
        const float2 w = neighbour_weights(g, grp);
        for (int d = 0; d < g.n_dmrs; ++d) {
          const phy_c32* A = d ? A1 : A0;
          const cf h = d ? ld(A1 + i) : h0;
          const cf lo = ld(A + i - per_grp), hi = ld(A + i + per_grp);
          cf e;
          e.x = h.x - fmaf(w.x, lo.x, w.y * hi.x);
          e.y = h.y - fmaf(w.x, lo.y, w.y * hi.y);
          ef += cabs2(e);
        }
      }
    }
  }

  // ---- gains of the (group, layer) pairs p whose antenna-0 entry p * nr lies in [i0, i1).
  // One work item per (pair, offset j < 3L): the comb index j into the pair's frequency span
  // [s_g-1, s_g+1 + L) (at most 3L indices) and, for j < L, into its own group for the time term.
  const float inv_l2 = 1.f / (float)(g.L * g.L);
  const int p_lo = (i0 + nr - 1) / nr, p_hi = (i1 + nr - 1) / nr;
  const int span = 3 * g.L;
  const float inv_span = 1.f / (float)span, inv_nl = 1.f / (float)nl;
  for (int q = threadIdx.x; q < (p_hi - p_lo) * span; q += kNoiseThreads) {
    const int pq = div_small(q, span, inv_span);
    const int p = p_lo + pq, j = q - pq * span;
    const int grp = div_small(p, nl, inv_nl), l = p - grp * nl, c = l & 1;
    const phy_c32* P0 = pilots + ((size_t)(cell * g.n_dmrs) * nl + l) * g.n_sc + c;
    const phy_c32* P1 = P0 + (g.n_dmrs == 2 ? (size_t)nl * g.n_sc : 0);
    const int s = group_start(g, grp);
    if (g.n_dmrs == 2 && j < g.L)
      gt += (pilot_pow(P0 + 2 * (s + j)) + pilot_pow(P1 + 2 * (s + j))) * inv_l2;
    if (grp >= 1 && grp <= g.G - 2) {
      const int sm = group_start(g, grp - 1), sp = group_start(g, grp + 1);
      const int m = sm + j;
      if (m < sp + g.L) {
        // signed weight of comb index m: its own group, minus the neighbours' shares
        const float2 w = neighbour_weights(g, grp);
        float wm = (m >= s && m < s + g.L) ? 1.f : 0.f;
        if (m < sm + g.L) wm -= w.x;
        if (m >= sp) wm -= w.y;
        float pw = pilot_pow(P0 + 2 * m);
        if (g.n_dmrs == 2) pw += pilot_pow(P1 + 2 * m);
        gf = fmaf(wm * wm * inv_l2, pw, gf);
      }
    }
  }

  // ---- CTA sums in a fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ef += __shfl_xor_sync(0xffffffffu, ef, o);
    gf += __shfl_xor_sync(0xffffffffu, gf, o);
    et += __shfl_xor_sync(0xffffffffu, et, o);
    gt += __shfl_xor_sync(0xffffffffu, gt, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float4(ef, gf, et, gt);
  __syncthreads();
  if (threadIdx.x == 0) {
    float4 s = red[0];
#pragma unroll
    for (int w = 1; w < kNoiseThreads / 32; ++w) {
      s.x += red[w].x;
      s.y += red[w].y;
      s.z += red[w].z;
      s.w += red[w].w;
    }
    part[(size_t)cell * n_blk + blk] = s;
  }
}

__global__ void __launch_bounds__(kNoiseThreads)
    noise_partial_kernel(Geo g, const phy_c32* __restrict__ anchors,
                         const phy_c32* __restrict__ pilots, float4* __restrict__ part) {
  __shared__ float4 red[kNoiseThreads / 32];
  // the final kernel may launch now and wait for this grid's completion (programmatic launch)
  asm volatile("griddepcontrol.launch_dependents;");
  noise_partial_body(g, blockIdx.y, blockIdx.x, gridDim.x, anchors, pilots, part, red);
}

// One cell's estimate from its n_part partial sums (and, with alpha < 1, its blend into the
// cell's state); every thread of the CTA calls it. red: CTA scratch of 4 x kNoiseThreads doubles.
__device__ __forceinline__ void noise_final_body(const Geo& g, int cell, int mode, float alpha,
                                                 int n_part, const float4* __restrict__ part,
                                                 float* __restrict__ sigma2_out,
                                                 double (*red)[kNoiseThreads]) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n_part; i += kNoiseThreads) {
    const float4 v = part[(size_t)cell * n_part + i];
    s[0] += v.x;
    s[1] += v.y;
    s[2] += v.z;
    s[3] += v.w;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int h = kNoiseThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nr = (double)g.n_rx;
    const double f = red[1][0] > 0.0 ? red[0][0] / (nr * red[1][0]) : (double)NAN;
    const double t = (g.n_dmrs == 2 && red[3][0] > 0.0) ? red[2][0] / (nr * red[3][0])
                                                         : (double)NAN;
    double r = f;
    if (mode == PHY_NOISE_TIME) r = t;
    if (mode == PHY_NOISE_MIN) r = fmin(f, t);  // NaN only if both are
    if (alpha < 1.f) {  // tracking: blend into the cell's state, which a bad value leaves alone
      const float prior = sigma2_out[cell];
      const bool have = isfinite(prior) && prior > 0.f;
      if (!isfinite(r)) r = have ? (double)prior : r;
      else if (have) r = (double)alpha * r + (1.0 - (double)alpha) * (double)prior;
    }
    sigma2_out[cell] = (float)r;
  }
}

__global__ void __launch_bounds__(kNoiseThreads)
    noise_final_kernel(Geo g, int mode, float alpha, int n_part, const float4* __restrict__ part,
                       float* __restrict__ sigma2_out) {
  __shared__ double red[4][kNoiseThreads];
  // launched programmatically behind the partial kernel: wait until its sums are complete
  asm volatile("griddepcontrol.wait;" ::: "memory");
  noise_final_body(g, blockIdx.x, mode, alpha, n_part, part, sigma2_out, red);
}

int n_parts(const Geo& g) {
  const int per_d = g.G * g.n_layers * g.n_rx;
  return (per_d + kNoiseEntries - 1) / kNoiseEntries;
}

// Batched forms: CTAs stride over the (block, cell) items, then the cells, of the jobs in the
// table that track their noise level; the job's sigma2 pointer is its state.
__global__ void __launch_bounds__(kNoiseThreads)
    noise_partial_batch_kernel(const BatchTable* __restrict__ t) {
  __shared__ Geo sg;
  __shared__ BatchIndex ix;
  __shared__ float4 red[kNoiseThreads / 32];
  const int n = t->n_items[kBatchNoisePart][0];
  if ((int)blockIdx.x >= n) return;
  batch_index_load(ix, t, kBatchNoisePart, 0);
  __syncthreads();
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    int local;
    const BatchJob& J = t->job[batch_find(ix, w, local)];
    batch_load_geo(sg, J.g);
    __syncthreads();
    noise_partial_body(sg, local / J.noise_blocks, local % J.noise_blocks, J.noise_blocks,
                       J.anchors, J.pilots, J.noise_part, red);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kNoiseThreads)
    noise_final_batch_kernel(const BatchTable* __restrict__ t) {
  __shared__ Geo sg;
  __shared__ BatchIndex ix;
  __shared__ double red[4][kNoiseThreads];
  const int n = t->n_items[kBatchNoiseFinal][0];
  if ((int)blockIdx.x >= n) return;
  batch_index_load(ix, t, kBatchNoiseFinal, 0);
  __syncthreads();
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    int local;
    const BatchJob& J = t->job[batch_find(ix, w, local)];
    batch_load_geo(sg, J.g);
    __syncthreads();
    noise_final_body(sg, local, J.noise_mode, J.noise_alpha, J.noise_blocks, J.noise_part,
                     const_cast<float*>(J.sigma2), red);
    __syncthreads();
  }
}

}  // namespace

int noise_blocks(const Geo& g) { return n_parts(g); }

cudaError_t launch_noise_batch(const BatchTable* t, cudaStream_t st) {
  const int grid = 2 * device_sm_count();
  noise_partial_batch_kernel<<<grid, kNoiseThreads, 0, st>>>(t);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  noise_final_batch_kernel<<<grid, kNoiseThreads, 0, st>>>(t);
  return cudaGetLastError();
}

size_t noise_scratch_bytes(const Geo& g) {
  return (size_t)g.n_cells * n_parts(g) * sizeof(float4);
}

cudaError_t launch_noise_est(const Geo& g, int mode, float alpha, const phy_c32* anchors,
                             const phy_c32* pilots, float* sigma2_out, void* scratch,
                             cudaStream_t st) {
  const int np = n_parts(g);
  float4* part = static_cast<float4*>(scratch);
  noise_partial_kernel<<<dim3(np, g.n_cells), kNoiseThreads, 0, st>>>(g, anchors, pilots, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // programmatic dependent launch: the final kernel's launch overlaps the partial kernel's tail
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(g.n_cells);
  lc.blockDim = dim3(kNoiseThreads);
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  const float4* cpart = part;
  return cudaLaunchKernelEx(&lc, noise_final_kernel, g, mode, alpha, np, cpart, sigma2_out);
}

}  // namespace phy
