// DMRS least-squares channel estimation (the channel-estimation block named in Sec. III-B).
//
// One CTA per (LS group, DMRS symbol, cell); one thread per receive antenna. Each thread reads
// the 2L subcarriers of its group on its antenna row of Y (one contiguous 16L-byte run) and, for
// every layer, despreads the pilots of that layer's comb:
//   anchor[cell][d][g][l][r] = (1/L) sum_{i<L} Y[cell][t_d][r][k_i] conj(P[cell][d][l][k_i]),
//   k_i = 2 (s_g + i) + (l % 2).
// Writes are coalesced over r. The pilots of a group are shared by all antennas (L1 broadcast).
#include "launch.h"

namespace phy {

__global__ void __launch_bounds__(64) chest_ls_kernel(Geo g, const phy_c32* __restrict__ Y,
                                                      const phy_c32* __restrict__ P,
                                                      phy_c32* __restrict__ anchors) {
  const int grp = blockIdx.x, d = blockIdx.y, cell = blockIdx.z;
  const int r = threadIdx.x;
  if (r >= g.n_rx) return;
  const int t = (d == 0) ? g.dmrs0 : g.dmrs1;
  const int s = group_start(g, grp);
  const phy_c32* yrow = Y + ((size_t)(cell * g.n_sym + t) * g.n_rx + r) * g.n_sc;
  const phy_c32* prow = P + (size_t)(cell * g.n_dmrs + d) * g.n_layers * g.n_sc;
  phy_c32* out = anchors + (((size_t)(cell * g.n_dmrs + d) * g.G + grp) * g.n_layers) * g.n_rx;
  const float inv_l = 1.f / (float)g.L;
  for (int l = 0; l < g.n_layers; ++l) {
    const int c = l & 1;
    cf acc = mk(0.f, 0.f);
    for (int i = 0; i < g.L; ++i) {
      const int k = 2 * (s + i) + c;
      acc = cfma_cj(ld(prow + (size_t)l * g.n_sc + k), ld(yrow + k), acc);  // y conj(p)
    }
    st(out + (size_t)l * g.n_rx + r, inv_l * acc);
  }
}

cudaError_t launch_chest(const Geo& g, const phy_c32* Y, const phy_c32* pilots, phy_c32* anchors,
                         cudaStream_t st) {
  dim3 grid(g.G, g.n_dmrs, g.n_cells);
  int threads = g.n_rx <= 32 ? 32 : 64;
  chest_ls_kernel<<<grid, threads, 0, st>>>(g, Y, pilots, anchors);
  return cudaGetLastError();
}

}  // namespace phy
