// Device-side helpers shared by the receiver kernels: complex arithmetic, slot geometry,
// interpolation weights and the max-log Gray QAM demapper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/phy.h"

namespace phy {

constexpr int kMaxSym = 14;
constexpr int kMaxRx = 64;
constexpr int kMaxLayers = 16;

// Everything a kernel needs to know about the slot, resolved on the host from phy_slot_cfg.
struct Geo {
  int n_cells, n_sc, n_sym, n_rx, n_layers, qm;
  int n_dmrs, dmrs0, dmrs1;
  int L;        // Walsh cover length
  int G;        // LS groups per comb
  int n_comb;   // n_sc / 2
  int n_dsym;   // data symbols
  int n_seg;    // frequency segments (anchor pairs), max(G - 1, 1)
  float pivot_min;
  int dsym[kMaxSym];    // data symbol index j -> OFDM symbol t
  float tw[kMaxSym];    // weight of the second DMRS estimate at data symbol j
};

// ---------------------------------------------------------------- complex float
struct cf {
  float x, y;
};
__device__ __forceinline__ cf mk(float a, float b) { return cf{a, b}; }
__device__ __forceinline__ cf operator+(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cf operator-(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cf operator*(float s, cf a) { return cf{s * a.x, s * a.y}; }
// a * b
__device__ __forceinline__ cf cmul(cf a, cf b) {
  return cf{fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)};
}
// acc + conj(a) * b
__device__ __forceinline__ cf cfma_cj(cf a, cf b, cf acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
// acc + a * b
__device__ __forceinline__ cf cfma(cf a, cf b, cf acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
// acc - a * conj(b)
__device__ __forceinline__ cf cfms_cjb(cf a, cf b, cf acc) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
// acc - a * b
__device__ __forceinline__ cf cfms(cf a, cf b, cf acc) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(-a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float cabs2(cf a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ cf ld(const phy_c32* p) {
  float2 v = *reinterpret_cast<const float2*>(p);
  return cf{v.x, v.y};
}
__device__ __forceinline__ void st(phy_c32* p, cf v) {
  *reinterpret_cast<float2*>(p) = make_float2(v.x, v.y);
}
__device__ __forceinline__ bool finite_cf(cf a) { return isfinite(a.x) && isfinite(a.y); }

// ---------------------------------------------------------------- LS groups and anchors
// Start (comb index) of LS group g; the last group is pulled back to stay inside the comb.
__device__ __forceinline__ int group_start(const Geo& g, int grp) {
  int s = g.L * grp;
  int last = g.n_comb - g.L;
  return s < last ? s : last;
}
// Subcarrier of group grp's anchor on comb c.
__device__ __forceinline__ int anchor_pos(const Geo& g, int grp, int c) {
  return 2 * group_start(g, grp) + g.L - 1 + c;
}
// Subcarrier range [lo, hi) of frequency segment j: the subcarriers whose interpolation, on both
// combs, uses anchors j and j+1 (the first and last segments also take the hold regions).
__device__ __forceinline__ void segment_range(const Geo& g, int j, int& lo, int& hi) {
  if (g.G == 1) {
    lo = 0;
    hi = g.n_sc;
    return;
  }
  lo = (j == 0) ? 0 : anchor_pos(g, j, 1);
  hi = (j == g.G - 2) ? g.n_sc : anchor_pos(g, j + 1, 1);
}
// Weight of anchor j+1 (segment j) at subcarrier k for comb c, clamped to [0, 1].
__device__ __forceinline__ float seg_beta(const Geo& g, int j, int k, int c) {
  if (g.G == 1) return 0.f;
  int p0 = anchor_pos(g, j, c), p1 = anchor_pos(g, j + 1, c);
  float b = (float)(k - p0) / (float)(p1 - p0);
  return fminf(fmaxf(b, 0.f), 1.f);
}
// Second group of segment j's anchor pair (equal to the first when there is one group).
__device__ __forceinline__ int seg_g1(const Geo& g, int j) { return g.G == 1 ? 0 : j + 1; }

// ---------------------------------------------------------------- max-log demapper
// PAM level (in units of the unnormalised odd-integer grid) of the axis bits e_0..e_{H-1}, where
// e_0 = bits & (1 << (H-1)) ... following the NR nesting
// (1-2e0)(2^(H-1) - (1-2e1)(2^(H-2) - ... (2 - (1-2e_{H-1})))).
template <int H>
__device__ __forceinline__ float pam_level(int bits) {
  float inner = 1.f;
#pragma unroll
  for (int i = H - 1; i >= 1; --i) {
    int e = (bits >> (H - 1 - i)) & 1;
    inner = (float)(1 << (H - i)) - (1 - 2 * e) * inner;
  }
  int e0 = (bits >> (H - 1)) & 1;
  return (1 - 2 * e0) * inner;
}

// Max-log LLRs of the H axis bits for axis value v (already scaled to the odd-integer grid),
// out[i] = (min_{e_i=1} (v-s)^2 - min_{e_i=0} (v-s)^2) * scale.
template <int H>
__device__ __forceinline__ void pam_llr(float v, float scale, float* out) {
  float m0[H], m1[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    m0[i] = 3.0e38f;
    m1[i] = 3.0e38f;
  }
#pragma unroll
  for (int b = 0; b < (1 << H); ++b) {
    float d = v - pam_level<H>(b);
    d = d * d;
#pragma unroll
    for (int i = 0; i < H; ++i) {
      if ((b >> (H - 1 - i)) & 1)
        m1[i] = fminf(m1[i], d);
      else
        m0[i] = fminf(m0[i], d);
    }
  }
#pragma unroll
  for (int i = 0; i < H; ++i) out[i] = (m1[i] - m0[i]) * scale;
}

// LLRs of one layer's QM bits (b0, b1, ... interleaving I and Q) from the unbiased symbol x~ and
// effective noise s2eff. The axis grid is the NR normalisation sqrt(2 (4^H - 1) / 3).
template <int QM>
__device__ __forceinline__ void qam_llr(cf xt, float s2eff, float* llr) {
  constexpr int H = QM / 2;
  constexpr float nrm2 = 2.f * ((1 << (2 * H)) - 1) / 3.f;  // squared normalisation
  const float a = sqrtf(nrm2);
  // distances in grid units squared are nrm2 times the normalised ones
  const float scale = 1.f / (nrm2 * s2eff);
  float li[H], lq[H];
  pam_llr<H>(xt.x * a, scale, li);
  pam_llr<H>(xt.y * a, scale, lq);
#pragma unroll
  for (int i = 0; i < H; ++i) {
    llr[2 * i] = li[i];
    llr[2 * i + 1] = lq[i];
  }
}

// Per-layer SINR bookkeeping from d = (A^-1)_kk.
struct LayerOut {
  float sinr, mu, s2eff;
};
__device__ __forceinline__ LayerOut layer_stats(float sigma2, float dkk) {
  float e = sigma2 * dkk;
  e = fminf(fmaxf(e, 1e-30f), 1.f - 1e-7f);
  float mu = 1.f - e;
  LayerOut o;
  o.mu = mu;
  o.sinr = mu / e;
  o.s2eff = e / mu;
  return o;
}

}  // namespace phy
