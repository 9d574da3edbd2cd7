// FP64 re-computation of one RE whose FP32 factorisation was flagged ill-conditioned.
//
// The FP32 path's Gram matrix already carries FP32 rounding, which an ill-conditioned matrix
// amplifies, so re-factoring it alone would not help: this routine redoes the RE from its inputs
// in double precision (interpolated channel from the LS anchors, A = H^H H + s2 I, b = H^H y,
// Cholesky, both solves and the inverse diagonal). It is written with rolled loops over thread-
// private arrays (local memory): only flagged REs run it, and its code stays small.
#pragma once

#include "common.cuh"

namespace phy {

struct cd {
  double x, y;
};

// Outputs of the FP64 recomputation, narrowed to the output precision by the caller.
struct Refactor64Out {
  bool ok;
  cf x[kMaxLayers];
  float d[kMaxLayers];
};

__device__ __noinline__ void refactor_fp64(const Geo& g, const phy_c32* __restrict__ anchors,
                                           const phy_c32* __restrict__ Y, int cell, int jj, int k,
                                           int j, float sigma2, Refactor64Out* out) {
  const int nr = g.n_rx, nl = g.n_layers;
  const int t = g.dsym[jj];
  // time weight of the second DMRS symbol and frequency weights of anchor j+1 per comb
  double a1 = 0.0;
  if (g.n_dmrs == 2) {
    a1 = (double)(t - g.dmrs0) / (double)(g.dmrs1 - g.dmrs0);
    a1 = a1 < 0.0 ? 0.0 : (a1 > 1.0 ? 1.0 : a1);
  }
  double be[2] = {0.0, 0.0};
  const int g1 = seg_g1(g, j);
  if (g.G > 1) {
    for (int c = 0; c < 2; ++c) {
      const int p0 = anchor_pos(g, j, c), p1 = anchor_pos(g, j + 1, c);
      double b = (double)(k - p0) / (double)(p1 - p0);
      be[c] = b < 0.0 ? 0.0 : (b > 1.0 ? 1.0 : b);
    }
  }
  cd A[kMaxLayers * (kMaxLayers + 1) / 2];
  cd bv[kMaxLayers];
  for (int e = 0; e < nl * (nl + 1) / 2; ++e) A[e] = cd{0.0, 0.0};
  for (int l = 0; l < nl; ++l) bv[l] = cd{0.0, 0.0};
  const phy_c32* yk = Y + ((size_t)cell * g.n_sym + t) * nr * g.n_sc + k;
  for (int r = 0; r < nr; ++r) {
    cd h[kMaxLayers];
    for (int l = 0; l < nl; ++l) {
      const double w1 = be[l & 1], w0 = 1.0 - w1;
      cd acc{0.0, 0.0};
      for (int d = 0; d < g.n_dmrs; ++d) {
        const double td = (g.n_dmrs == 2) ? (d ? a1 : 1.0 - a1) : 1.0;
        const phy_c32 c0 = anchors[((((size_t)cell * g.n_dmrs + d) * g.G + j) * nl + l) * nr + r];
        const phy_c32 c1 = anchors[((((size_t)cell * g.n_dmrs + d) * g.G + g1) * nl + l) * nr + r];
        acc.x += td * (w0 * c0.re + w1 * c1.re);
        acc.y += td * (w0 * c0.im + w1 * c1.im);
      }
      h[l] = acc;
    }
    const phy_c32 y = yk[(size_t)r * g.n_sc];
    for (int l = 0; l < nl; ++l) {
      bv[l].x += h[l].x * y.re + h[l].y * y.im;  // conj(h) y
      bv[l].y += h[l].x * y.im - h[l].y * y.re;
      for (int m = 0; m <= l; ++m) {
        cd& a = A[l * (l + 1) / 2 + m];  // conj(h_l) h_m
        a.x += h[l].x * h[m].x + h[l].y * h[m].y;
        a.y += h[l].x * h[m].y - h[l].y * h[m].x;
      }
    }
  }
  // Cholesky (left-looking), L stored over A; rinv = 1 / L_jj
  double rinv[kMaxLayers];
  bool ok = true;
  for (int c = 0; c < nl; ++c) {
    double dg = A[c * (c + 1) / 2 + c].x + (double)sigma2;
    for (int m = 0; m < c; ++m) {
      const cd v = A[c * (c + 1) / 2 + m];
      dg -= v.x * v.x + v.y * v.y;
    }
    ok = ok && dg > 0.0;
    const double r = dg > 0.0 ? 1.0 / sqrt(dg) : 0.0;
    rinv[c] = r;
    for (int i = c + 1; i < nl; ++i) {
      cd s = A[i * (i + 1) / 2 + c];
      for (int m = 0; m < c; ++m) {  // s -= L_im conj(L_cm)
        const cd p = A[i * (i + 1) / 2 + m], q = A[c * (c + 1) / 2 + m];
        s.x -= p.x * q.x + p.y * q.y;
        s.y -= p.y * q.x - p.x * q.y;
      }
      A[i * (i + 1) / 2 + c] = cd{s.x * r, s.y * r};
    }
  }
  out->ok = ok;
  if (!ok) return;
  // forward z = L^-1 b, backward x = L^-H z
  cd z[kMaxLayers];
  for (int i = 0; i < nl; ++i) {
    cd s = bv[i];
    for (int m = 0; m < i; ++m) {
      const cd p = A[i * (i + 1) / 2 + m];
      s.x -= p.x * z[m].x - p.y * z[m].y;
      s.y -= p.x * z[m].y + p.y * z[m].x;
    }
    z[i] = cd{s.x * rinv[i], s.y * rinv[i]};
  }
  cd x[kMaxLayers];
  for (int i = nl - 1; i >= 0; --i) {
    cd s = z[i];
    for (int m = i + 1; m < nl; ++m) {  // s -= conj(L_mi) x_m
      const cd p = A[m * (m + 1) / 2 + i];
      s.x -= p.x * x[m].x + p.y * x[m].y;
      s.y -= p.x * x[m].y - p.y * x[m].x;
    }
    x[i] = cd{s.x * rinv[i], s.y * rinv[i]};
  }
  // diag(A^-1): column norms of L^-1, one column at a time
  for (int c = 0; c < nl; ++c) {
    cd v[kMaxLayers];
    v[c] = cd{rinv[c], 0.0};
    double nrm = rinv[c] * rinv[c];
    for (int i = c + 1; i < nl; ++i) {
      cd s{0.0, 0.0};
      for (int m = c; m < i; ++m) {
        const cd p = A[i * (i + 1) / 2 + m];
        s.x += p.x * v[m].x - p.y * v[m].y;
        s.y += p.x * v[m].y + p.y * v[m].x;
      }
      v[i] = cd{-s.x * rinv[i], -s.y * rinv[i]};
      nrm += v[i].x * v[i].x + v[i].y * v[i].y;
    }
    out->d[c] = (float)nrm;
    out->x[c] = mk((float)x[c].x, (float)x[c].y);
  }
}

}  // namespace phy
