// Pieces shared by the FP32 and tensor-core segment kernels: index helpers and the folding of
// the corner cross-Gram X into the per-symbol Gram blocks Y_gg'(t).
#pragma once

#include "common.cuh"

namespace phy {

// Row l and column m (l >= m) of packed lower-triangle index e.
__device__ __forceinline__ void tri_decode(int e, int& l, int& m) {
  int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  while (r * (r + 1) / 2 > e) --r;
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  l = r;
  m = e - r * (r + 1) / 2;
}

// Frequency segment holding subcarrier k (see segment_range).
__device__ __forceinline__ int seg_of(const Geo& g, int k) {
  if (g.G == 1) return 0;
  int j = (k - g.L) / (2 * g.L);
  if (k < g.L) j = 0;
  return j < g.n_seg - 1 ? j : g.n_seg - 1;
}

// Y_gg'(t)[l][m] = sum_{d,d'} tau_d(t) tau_d'(t) X[(d,g) l][(d',g') m] for every data symbol and
// every lower-triangle entry (l, m), written as 4-tuples (Y00, Y01, Y10, Y11) of complex values
// (two float4 per entry) to out[jj][e]. Xget(i, k) returns X at corner-layer indices
// i = (2 d + g) NL + l (corners ordered (d0,g0), (d0,g1), (d1,g0), (d1,g1)).
// With tau_0 = 1 - t, tau_1 = t the sum is (1-t)^2 X00 + (1-t) t (X01 + X10) + t^2 X11 (X_dd' the
// DMRS-pair blocks), so each work item (entry e, first corner g) reads X once and sweeps the
// symbols; consecutive threads write consecutive float4 (Y_g0, Y_g1).
template <int NL, int NT, class XGet>
__device__ __forceinline__ void form_gram_blocks(const Geo& g, XGet Xget, float4* out, int tid) {
  constexpr int NTRI = NL * (NL + 1) / 2;
  const int nds = g.n_dsym;
  for (int i = tid; i < 2 * NTRI; i += NT) {
    const int te = i >> 1, gg = i & 1;
    int l, m;
    tri_decode(te, l, m);
    cf x00[2], xs[2], x11[2];
#pragma unroll
    for (int gp = 0; gp < 2; ++gp) {
      x00[gp] = Xget(gg * NL + l, gp * NL + m);
      if (g.n_dmrs == 2) {
        xs[gp] = Xget(gg * NL + l, (2 + gp) * NL + m) + Xget((2 + gg) * NL + l, gp * NL + m);
        x11[gp] = Xget((2 + gg) * NL + l, (2 + gp) * NL + m);
      } else {
        xs[gp] = x11[gp] = mk(0.f, 0.f);
      }
    }
    float4* o = out + i;
#pragma unroll
    for (int jj = 0; jj < kMaxSym; ++jj) {
      if (jj < nds) {
        const float t1 = g.tw[jj], t0 = 1.f - t1;
        const float w00 = t0 * t0, w01 = t0 * t1, w11 = t1 * t1;
        cf y[2];
#pragma unroll
        for (int gp = 0; gp < 2; ++gp) {
          y[gp].x = fmaf(w00, x00[gp].x, fmaf(w01, xs[gp].x, w11 * x11[gp].x));
          y[gp].y = fmaf(w00, x00[gp].y, fmaf(w01, xs[gp].y, w11 * x11[gp].y));
        }
        o[(size_t)jj * NTRI * 2] = make_float4(y[0].x, y[0].y, y[1].x, y[1].y);
      }
    }
  }
}

}  // namespace phy
