// LMMSE detection on an explicitly given channel (genie or materialised H), one thread per RE.
// Builds A = H^H H + s2 I and b = H^H y directly (the covariance-by-FMA step of Fig. 2(b), once
// per RE) and hands them to the shared per-RE solver. This is the checking path behind
// phy_mmse_detect; the fused path never materialises H.
#include "launch.h"
#include "solver.cuh"

namespace phy {

namespace {

struct LocalScratch {
  cf* base;
  __device__ __forceinline__ void st(int e, cf v) const { base[e] = v; }
  __device__ __forceinline__ cf ld(int e) const { return base[e]; }
};

// The solver's 8x8 L21/T matrix in the same thread-local array, entry (i, j) at 8 i + j.
struct LocalRows {
  cf* base;
  __device__ __forceinline__ void st_row(int i, const cf (&r)[8]) const {
#pragma unroll
    for (int j = 0; j < 8; ++j) base[8 * i + j] = r[j];
  }
  __device__ __forceinline__ void ld_row(int i, cf (&r)[8]) const {
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = base[8 * i + j];
  }
  __device__ __forceinline__ void ld_col(int c, cf (&r)[8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = base[8 * i + c];
  }
  __device__ __forceinline__ void sync_st() const {}
};

template <int NL>
__global__ void __launch_bounds__(128) detect_h_kernel(Geo g, const phy_c32* __restrict__ H,
                                                       const phy_c32* __restrict__ Y,
                                                       const float* __restrict__ sigma2,
                                                       phy_c32* __restrict__ x_hat,
                                                       float* __restrict__ sinr_out,
                                                       uint8_t* __restrict__ flags_out) {
  const int nr = g.n_rx, nl = g.n_layers, nds = g.n_dsym;
  const size_t n_re = (size_t)g.n_cells * nds * g.n_sc;
  const size_t re = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (re >= n_re) return;
  const int k = (int)(re % g.n_sc);
  const int jj = (int)((re / g.n_sc) % nds);
  const int cell = (int)(re / ((size_t)g.n_sc * nds));
  const int t = g.dsym[jj];
  const float s2 = sigma2[cell];
  const phy_c32* h = H + re * nr * nl;  // [rx][layer]
  const phy_c32* y = Y + ((size_t)cell * g.n_sym + t) * nr * g.n_sc + k;

  cf a[NL * (NL + 1) / 2];
  cf b[NL];
#pragma unroll
  for (int i = 0; i < NL * (NL + 1) / 2; ++i) a[i] = mk(0.f, 0.f);
#pragma unroll
  for (int l = 0; l < NL; ++l) b[l] = mk(0.f, 0.f);
  bool fin = true;
  for (int r = 0; r < nr; ++r) {
    cf hr[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) hr[l] = (l < nl) ? ld(h + r * nl + l) : mk(0.f, 0.f);
    const cf yr = ld(y + (size_t)r * g.n_sc);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      b[l] = cfma_cj(hr[l], yr, b[l]);
#pragma unroll
      for (int m = 0; m <= l; ++m) a[tri(l, m)] = cfma_cj(hr[l], hr[m], a[tri(l, m)]);
    }
  }
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    fin = fin && finite_cf(b[l]);
    a[tri(l, l)].y = 0.f;
    a[tri(l, l)].x += (l < nl) ? s2 : 1.f;
  }
  auto getA = [&](int l, int m) -> cf { return a[tri(l, m)]; };
  cf x[NL];
  float dd[NL];
  SolveInfo si;
  if constexpr (NL == 16) {
    cf scratch[kScrSlots];
    // runtime row of the register-held matrix by predicated compile-time selects
    auto rowA = [&](int l, cf (&row)[8]) {
#pragma unroll
      for (int li = 8; li < 16; ++li)
        if (li == l)
#pragma unroll
          for (int k = 0; k < 8; ++k) row[k] = a[tri(li, k)];
    };
    si = solve16(getA, rowA, LocalScratch{scratch + kScrV}, LocalRows{scratch + kScrL21}, b, x, dd);
  } else {
    si = solve_small<NL>(getA, b, x, dd);
  }
  fin = fin && si.fin;
  const bool ok = si.ok && fin;
  uint8_t flag = 0;
  if (!fin) flag |= 4;
  if (!si.ok || si.pmin < g.pivot_min * si.pmax) flag |= 1;
  flags_out[re] = flag;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    if (l < nl) {
      const LayerOut o = layer_stats(s2, dd[l]);
      st(x_hat + re * nl + l, ok ? x[l] : mk(0.f, 0.f));
      sinr_out[re * nl + l] = ok ? o.sinr : 0.f;
    }
  }
}

template <int NL>
cudaError_t launch_h(const Geo& g, const phy_c32* H, const phy_c32* Y, const float* sigma2,
                     phy_c32* x_hat, float* sinr, uint8_t* flags, cudaStream_t st) {
  const size_t n_re = (size_t)g.n_cells * g.n_dsym * g.n_sc;
  const int threads = 128;
  const unsigned blocks = (unsigned)((n_re + threads - 1) / threads);
  detect_h_kernel<NL><<<blocks, threads, 0, st>>>(g, H, Y, sigma2, x_hat, sinr, flags);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_detect_h(const Geo& g, const phy_c32* H, const phy_c32* Y, const float* sigma2,
                            phy_c32* x_hat, float* sinr, uint8_t* flags, cudaStream_t st) {
  const int nl = g.n_layers;
  if (nl <= 2) return launch_h<2>(g, H, Y, sigma2, x_hat, sinr, flags, st);
  if (nl <= 4) return launch_h<4>(g, H, Y, sigma2, x_hat, sinr, flags, st);
  if (nl <= 8) return launch_h<8>(g, H, Y, sigma2, x_hat, sinr, flags, st);
  return launch_h<16>(g, H, Y, sigma2, x_hat, sinr, flags, st);
}

}  // namespace phy
