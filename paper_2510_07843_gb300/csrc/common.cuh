// Device-side helpers shared by the receiver kernels: complex arithmetic, slot geometry,
// interpolation weights and the max-log Gray QAM demapper.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/phy.h"

namespace phy {

constexpr int kMaxSym = 14;
constexpr int kMaxRx = 64;
constexpr int kMaxLayers = 16;
// Default first-level wait limits (polls): the tensor-core kernel's polls sleep up to ~1 us each.
constexpr unsigned kWaitSegDefault = 1u << 20;
constexpr unsigned kWaitSolveDefault = 1u << 22;

// Everything a kernel needs to know about the slot, resolved on the host from phy_slot_cfg.
struct Geo {
  int n_cells, n_sc, n_sym, n_rx, n_layers, qm;
  int n_dmrs, dmrs0, dmrs1;
  int L;        // Walsh cover length
  int G;        // LS groups per comb
  int n_comb;   // n_sc / 2
  int n_dsym;   // data symbols
  int n_seg;    // frequency segments (anchor pairs), max(G - 1, 1)
  int prec;     // phy_precision of the Gram and matched-filter products
  int refactor; // 1: recompute flagged (ill-conditioned) REs in FP64
  int llr_f16;  // 1: LLR outputs as binary16
  float pivot_min;
  // Poll limits of the first-level device waits (a wait that runs out is a timeout): in the
  // tensor-core segment kernel and in the solve kernel. The waits that only let copies and
  // MMAs already in flight land before a CTA ends keep their own, longer limits.
  unsigned wait_seg, wait_solve;
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
// NR Gray QAM: bits b0, b2, ... (e_0, e_1, ... of the in-phase axis) and b1, b3, ... (the
// quadrature axis) each pick a PAM level (1-2e0)(2^(H-1) - (1-2e1)(2^(H-2) - ... (2 - (1-2e_{H-1}))))
// on the odd-integer grid, scaled by 1/sqrt(2 (4^H - 1) / 3).

// Nearest odd integer to x, clamped to the odd interval [a, b].
__device__ __forceinline__ float nearest_odd(float x, float a, float b) {
  return fminf(fmaxf(fmaf(2.f, floorf(0.5f * x), 1.f), a), b);
}

// Max-log LLRs of the H axis bits for axis value v (already scaled to the odd-integer grid),
// out[i] = (min_{e_i=1} (v-s)^2 - min_{e_i=0} (v-s)^2) * scale, without visiting every level.
// Bit e_0 is the sign: the nearest level of each set is a clamped nearest odd integer. For
// i >= 1 the nesting |s| = 2^(H-1) - s_1 (2^(H-2) - s_2 (...)) means the level set of e_i is
// symmetric under the reflections v -> |v| and u -> |u - 2^(H-j)| (j < i), so its distance to v
// equals the distance of the folded value u_i to {1, 3, ..., 2^(H-i) - 1} (e_i = 0) or to
// {2^(H-i) + 1, ..., 2^(H-i+1) - 1} (e_i = 1). Equal to the exhaustive search up to rounding.
template <int H>
__device__ __forceinline__ void pam_llr(float v, float scale, float* out) {
  constexpr float M = (float)((1 << H) - 1);
  {
    const float n0 = nearest_odd(v, 1.f, M), n1 = nearest_odd(v, -M, -1.f);
    const float d0 = v - n0, d1 = v - n1;
    out[0] = fmaf(d1, d1, -d0 * d0) * scale;
  }
  float u = fabsf(v);
#pragma unroll
  for (int i = 1; i < H; ++i) {
    const float half = (float)(1 << (H - i));
    const float n0 = nearest_odd(u, 1.f, half - 1.f);
    const float n1 = nearest_odd(u, half + 1.f, 2.f * half - 1.f);
    const float d0 = u - n0, d1 = u - n1;
    out[i] = fmaf(d1, d1, -d0 * d0) * scale;
    u = fabsf(u - half);
  }
}

// LLRs of one layer's QM bits (b0, b1, ... interleaving I and Q) from the unbiased symbol x~,
// given the scale 1 / (nrm2 s2eff) for effective noise s2eff, nrm2 = 2 (4^H - 1) / 3 the squared
// NR grid normalisation (distances in grid units squared are nrm2 times the normalised ones).
// With s2eff = e / mu and SINR = mu / e the scale is SINR / nrm2 (qam_inv_nrm2).
template <int QM>
__device__ __forceinline__ constexpr float qam_inv_nrm2() {
  return 3.f / (2.f * ((1 << QM) - 1));
}
template <int QM>
__device__ __forceinline__ void qam_llr_scaled(cf xt, float scale, float* llr) {
  constexpr int H = QM / 2;
  constexpr float nrm2 = 2.f * ((1 << (2 * H)) - 1) / 3.f;  // squared normalisation
  const float a = sqrtf(nrm2);
  float li[H], lq[H];
  pam_llr<H>(xt.x * a, scale, li);
  pam_llr<H>(xt.y * a, scale, lq);
#pragma unroll
  for (int i = 0; i < H; ++i) {
    llr[2 * i] = li[i];
    llr[2 * i + 1] = lq[i];
  }
}
// The same from the effective noise s2eff.
template <int QM>
__device__ __forceinline__ void qam_llr(cf xt, float s2eff, float* llr) {
  constexpr float nrm2 = 2.f * ((1 << QM) - 1) / 3.f;
  qam_llr_scaled<QM>(xt, 1.f / (nrm2 * s2eff), llr);
}

// An LLR pair to the output at element index idx (even): FP32, or binary16 rounded to nearest
// with saturation at +-65504 (the largest finite binary16) when f16.
__device__ __forceinline__ void store_llr_pair(float* base, size_t idx, float a, float b,
                                               bool f16) {
  if (f16) {
    const float m = 65504.f;
    *reinterpret_cast<__half2*>(reinterpret_cast<__half*>(base) + idx) =
        __floats2half2_rn(fminf(fmaxf(a, -m), m), fminf(fmaxf(b, -m), m));
  } else {
    *reinterpret_cast<float2*>(base + idx) = make_float2(a, b);
  }
}

// Per-layer SINR bookkeeping from d = (A^-1)_kk.
struct LayerOut {
  float sinr, inv_mu, s2eff;  // SINR, 1 / mu (unbiasing gain), effective noise e / mu
};
__device__ __forceinline__ LayerOut layer_stats(float sigma2, float dkk) {
  float e = sigma2 * dkk;
  e = fminf(fmaxf(e, 1e-30f), 1.f - 1e-7f);
  float mu = 1.f - e;
  LayerOut o;
  // correctly rounded reciprocals, then products (one rounding more than a division)
  o.inv_mu = __frcp_rn(mu);
  o.sinr = mu * __frcp_rn(e);
  o.s2eff = e * o.inv_mu;
  return o;
}

}  // namespace phy
