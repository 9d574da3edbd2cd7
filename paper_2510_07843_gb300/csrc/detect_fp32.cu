// Fused LMMSE detection on FP32 CUDA cores: interpolation, Gram, matched filter, Cholesky,
// solves, SINR and max-log LLRs for one frequency segment of one cell per CTA.
//
// With linear interpolation every RE's channel is a weighted sum of the four "corner" anchor
// matrices of its segment (anchors j and j+1 of both DMRS symbols): column l of H(k, t) is
//   sum_{d,g} tau_d(t) w_g(k, comb(l)) C_{d,g}[:, l].
// So the Gram matrix of every RE of the segment is a quadratic form in the same corner
// cross-Gram X = C^H C (C = [C_00 C_01 C_10 C_11], n_rx x 4 n_layers), computed once per CTA.
// That is the paper's covariance-by-FMA step (Fig. 2(b)) done once per segment instead of once
// per RE, exact up to rounding. Per data symbol the time weights fold X into three blocks
// Y_gg'(t) = H_g(t)^H H_g'(t); per RE A = sum_{g,g'} D_g Y_gg' D_g' + s2 I with diagonal D_g of
// the frequency weights. The matched filter uses the time-interpolated anchors H_g(t) directly:
// b = D_0 H_0(t)^H y + D_1 H_1(t)^H y.
//
// Phases (one CTA, all data symbols of the segment):
//   A0 corners -> smem (layout [r][corner*NL + l])        A1 X = C^H C (4x4 register tiles)
//   A2 Y_gg'(t) for every data symbol                     A3 per symbol: H_g(t), matched filter
//   B  one thread per RE: build A, solve (solver.cuh), SINR, unbias, LLR, store.
#include <algorithm>

#include "launch.h"
#include "solver.cuh"

namespace phy {

namespace {

template <int NL>
struct FusedTraits {
  static constexpr int NT = (NL == 16) ? 192 : 128;
};

struct FusedLayout {
  int NC, NX, xs, hs;
  int off_ygg, off_b, off_C, off_X, off_Hg, off_scr;  // in cf units
  int total;                                         // cf units
};

__host__ __device__ inline FusedLayout fused_layout(int NL, int NT, int n_dmrs, int n_rx,
                                                   int n_dsym, int wmax) {
  FusedLayout f;
  f.NC = 2 * n_dmrs;
  f.NX = f.NC * NL;
  f.xs = f.NX + 2;  // row stride keeps 16-byte alignment and spreads banks
  f.hs = 2 * NL + 2;
  f.off_ygg = 0;
  int ygg = n_dsym * 3 * NL * NL;
  f.off_b = f.off_ygg + ygg;
  int bv = wmax * n_dsym * NL;
  bv = (bv + 1) & ~1;
  int u0 = f.off_b + bv;
  f.off_C = u0;
  f.off_X = f.off_C + n_rx * f.xs;
  f.off_Hg = f.off_X + f.NX * f.xs;
  int endA = f.off_Hg + n_rx * f.hs;
  f.off_scr = u0;
  int endB = (NL == 16) ? u0 + 64 * NT : u0;
  f.total = endA > endB ? endA : endB;
  return f;
}

struct SmemScratch {
  cf* base;  // points at this thread's first element
  int stride;
  __device__ __forceinline__ void st(int i, int j, cf v) const { base[(i * 8 + j) * stride] = v; }
  __device__ __forceinline__ cf ld(int i, int j) const { return base[(i * 8 + j) * stride]; }
};

template <int QM>
__device__ __forceinline__ void store_llr(float* dst, cf xt, float s2eff) {
  float l[QM];
  qam_llr<QM>(xt, s2eff, l);
#pragma unroll
  for (int q = 0; q < QM; q += 2) *reinterpret_cast<float2*>(dst + q) = make_float2(l[q], l[q + 1]);
}

__device__ __forceinline__ void store_llr_rt(int qm, float* dst, cf xt, float s2eff) {
  switch (qm) {
    case 2: store_llr<2>(dst, xt, s2eff); break;
    case 4: store_llr<4>(dst, xt, s2eff); break;
    case 6: store_llr<6>(dst, xt, s2eff); break;
    default: store_llr<8>(dst, xt, s2eff); break;
  }
}

template <int NL>
__global__ void __launch_bounds__(FusedTraits<NL>::NT, 1)
    detect_fp32_kernel(Geo g, int wmax, const phy_c32* __restrict__ anchors,
                       const phy_c32* __restrict__ Y, const float* __restrict__ sigma2,
                       phy_c32* __restrict__ x_hat, float* __restrict__ sinr_out,
                       float* __restrict__ llr_out, uint8_t* __restrict__ flags_out) {
  constexpr int NT = FusedTraits<NL>::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  const int tid = threadIdx.x;
  const int j = blockIdx.x, cell = blockIdx.y;
  const int nr = g.n_rx, nl = g.n_layers, nds = g.n_dsym;
  const FusedLayout f = fused_layout(NL, NT, g.n_dmrs, nr, nds, wmax);
  cf* Ygg = sm + f.off_ygg;
  cf* bvec = sm + f.off_b;
  cf* Cs = sm + f.off_C;
  cf* Xs = sm + f.off_X;
  cf* Hg = sm + f.off_Hg;
  int lo, hi;
  segment_range(g, j, lo, hi);
  const int W = hi - lo;
  const int nre = W * nds;
  const float s2 = sigma2[cell];

  // ---- A0: corner anchors
  {
    const int total = f.NC * NL * nr;
    const int g1 = seg_g1(g, j);
    for (int idx = tid; idx < total; idx += NT) {
      const int r = idx % nr;
      const int rest = idx / nr;
      const int l = rest % NL;
      const int corner = rest / NL;
      const int d = corner >> 1, gr = corner & 1;
      const int grp = gr ? g1 : j;
      cf v = mk(0.f, 0.f);
      if (l < nl)
        v = ld(anchors + ((((size_t)cell * g.n_dmrs + d) * g.G + grp) * nl + l) * nr + r);
      Cs[r * f.xs + corner * NL + l] = v;
    }
  }
  __syncthreads();
  // ---- A1: X = C^H C, full NX x NX in 4x4 tiles
  {
    const int nt4 = f.NX / 4;
    for (int tile = tid; tile < nt4 * nt4; tile += NT) {
      const int ti = tile / nt4, tj = tile % nt4;
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
  // ---- A2: Y_gg'(t) = sum_{d,d'} tau_d tau_d' X[(d,g)][(d',g')] for (g,g') in 00, 10, 11
  {
    const int per = 3 * NL * NL;
    for (int e = tid; e < nds * per; e += NT) {
      const int m = e % NL;
      const int l = (e / NL) % NL;
      const int blk = (e / (NL * NL)) % 3;
      const int jj = e / per;
      const int gg = blk == 0 ? 0 : 1;
      const int gp = blk == 2 ? 1 : 0;
      cf v;
      if (g.n_dmrs == 2) {
        const float t1 = g.tw[jj], t0 = 1.f - t1;
        const cf x00 = Xs[(gg * NL + l) * f.xs + gp * NL + m];
        const cf x01 = Xs[(gg * NL + l) * f.xs + (2 + gp) * NL + m];
        const cf x10 = Xs[((2 + gg) * NL + l) * f.xs + gp * NL + m];
        const cf x11 = Xs[((2 + gg) * NL + l) * f.xs + (2 + gp) * NL + m];
        v = (t0 * t0) * x00 + (t0 * t1) * x01 + (t1 * t0) * x10 + (t1 * t1) * x11;
      } else {
        v = Xs[(gg * NL + l) * f.xs + gp * NL + m];
      }
      Ygg[e] = v;
    }
  }
  // ---- A3: per data symbol, time-interpolated anchors and the matched filter
  for (int jj = 0; jj < nds; ++jj) {
    const float t1 = g.tw[jj], t0 = 1.f - t1;
    __syncthreads();  // previous symbol's readers of Hg are done (and A2 done reading X)
    for (int e = tid; e < nr * 2 * NL; e += NT) {
      const int col = e % (2 * NL);
      const int r = e / (2 * NL);
      const int gg = col / NL, l = col % NL;
      cf v = Cs[r * f.xs + gg * NL + l];
      if (g.n_dmrs == 2) v = t0 * v + t1 * Cs[r * f.xs + (2 + gg) * NL + l];
      Hg[r * f.hs + col] = v;
    }
    __syncthreads();
    const int t = g.dsym[jj];
    const phy_c32* ysym = Y + ((size_t)cell * g.n_sym + t) * nr * g.n_sc;
    for (int e = tid; e < W * NL; e += NT) {
      const int l = e % NL, kk = e / NL;
      const int k = lo + kk;
      cf z0 = mk(0.f, 0.f), z1 = mk(0.f, 0.f);
      if (l < nl) {
        const phy_c32* yp = ysym + k;
#pragma unroll 8
        for (int r = 0; r < nr; ++r) {
          const cf y = ld(yp + (size_t)r * g.n_sc);
          z0 = cfma_cj(Hg[r * f.hs + l], y, z0);
          z1 = cfma_cj(Hg[r * f.hs + NL + l], y, z1);
        }
      }
      const float be = seg_beta(g, j, k, l & 1);
      bvec[(jj * W + kk) * NL + l] = (1.f - be) * z0 + be * z1;
    }
  }
  __syncthreads();
  // ---- B: one thread per RE
  for (int re = tid; re < nre; re += NT) {
    const int jj = re / W, kk = re % W;
    const int k = lo + kk;
    const float be0 = seg_beta(g, j, k, 0), be1 = seg_beta(g, j, k, 1);
    const cf* Yj = Ygg + jj * 3 * NL * NL;
    auto getA = [&](int l, int m) -> cf {
      if (l >= nl || m >= nl) return (l == m) ? mk(1.f, 0.f) : mk(0.f, 0.f);
      const float bl = (l & 1) ? be1 : be0, bm = (m & 1) ? be1 : be0;
      const float wl0 = 1.f - bl, wm0 = 1.f - bm;
      const cf y00 = Yj[l * NL + m];
      const cf y10 = Yj[NL * NL + l * NL + m];
      const cf y10t = Yj[NL * NL + m * NL + l];  // Y01[l][m] = conj(Y10[m][l])
      const cf y11 = Yj[2 * NL * NL + l * NL + m];
      cf a;
      a.x = wl0 * wm0 * y00.x + wl0 * bm * y10t.x + bl * wm0 * y10.x + bl * bm * y11.x;
      a.y = wl0 * wm0 * y00.y - wl0 * bm * y10t.y + bl * wm0 * y10.y + bl * bm * y11.y;
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
      b[l] = (l < nl) ? bvec[re * NL + l] : mk(0.f, 0.f);
      fin = fin && finite_cf(b[l]);
    }
    SolveInfo si;
    if constexpr (NL == 16) {
      SmemScratch scr{sm + f.off_scr + tid, NT};
      si = solve16(getA, scr, b, x, dd);
    } else {
      si = solve_small<NL>(getA, b, x, dd);
    }
    fin = fin && si.fin;
    uint8_t flag = 0;
    const bool ok = si.ok && fin;
    if (!fin) flag |= 4;
    if (!si.ok || si.pmin < g.pivot_min * si.pmax) flag |= 1;
    const size_t ridx = ((size_t)cell * nds + jj) * g.n_sc + k;
    flags_out[ridx] = flag;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      if (l < nl) {
        const LayerOut o = layer_stats(s2, dd[l]);
        const size_t li = ridx * nl + l;
        if (ok) {
          if (x_hat) st(x_hat + li, x[l]);
          if (sinr_out) sinr_out[li] = o.sinr;
          if (llr_out) {
            const float im = 1.f / o.mu;
            store_llr_rt(g.qm, llr_out + li * g.qm, im * x[l], o.s2eff);
          }
        } else {
          if (x_hat) st(x_hat + li, mk(0.f, 0.f));
          if (sinr_out) sinr_out[li] = 0.f;
          if (llr_out)
            for (int q = 0; q < g.qm; ++q) llr_out[li * g.qm + q] = 0.f;
        }
      }
    }
  }
}

template <int NL>
cudaError_t launch_fused(const Geo& g, int wmax, const phy_c32* anchors, const phy_c32* Y,
                         const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                         uint8_t* flags, cudaStream_t st) {
  constexpr int NT = FusedTraits<NL>::NT;
  const FusedLayout f = fused_layout(NL, NT, g.n_dmrs, g.n_rx, g.n_dsym, wmax);
  const size_t bytes = (size_t)f.total * sizeof(cf);
  static size_t configured = 0;  // largest dynamic smem opted into so far
  if (bytes > configured) {
    cudaError_t e = cudaFuncSetAttribute(detect_fp32_kernel<NL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = bytes;
  }
  dim3 grid(g.n_seg, g.n_cells);
  detect_fp32_kernel<NL><<<grid, NT, bytes, st>>>(g, wmax, anchors, Y, sigma2, x_hat, sinr, llr,
                                                   flags);
  return cudaGetLastError();
}

int nl_class(int nl) { return nl <= 2 ? 2 : nl <= 4 ? 4 : nl <= 8 ? 8 : 16; }

}  // namespace

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
  const int NL = nl_class(g.n_layers);
  const int NT = NL == 16 ? FusedTraits<16>::NT : FusedTraits<8>::NT;
  const FusedLayout f =
      fused_layout(NL, NT, g.n_dmrs, g.n_rx, g.n_dsym, host_max_segment_width(g));
  return (size_t)f.total * sizeof(cf);
}

cudaError_t launch_detect_fp32(const Geo& g, const phy_c32* anchors, const phy_c32* Y,
                               const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                               uint8_t* flags, cudaStream_t st) {
  const int wmax = host_max_segment_width(g);
  switch (nl_class(g.n_layers)) {
    case 2: return launch_fused<2>(g, wmax, anchors, Y, sigma2, x_hat, sinr, llr, flags, st);
    case 4: return launch_fused<4>(g, wmax, anchors, Y, sigma2, x_hat, sinr, llr, flags, st);
    case 8: return launch_fused<8>(g, wmax, anchors, Y, sigma2, x_hat, sinr, llr, flags, st);
    default: return launch_fused<16>(g, wmax, anchors, Y, sigma2, x_hat, sinr, llr, flags, st);
  }
}

}  // namespace phy
