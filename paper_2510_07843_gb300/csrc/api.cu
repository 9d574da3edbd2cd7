// C ABI of libphy.so: argument validation, slot geometry, workspace carving, stream enqueue.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/phy.h"
#include "launch.h"

using phy::Geo;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int auto_occ(int n_layers) {
  int half = (n_layers + 1) / 2, L = 1;
  while (L < half) L *= 2;
  return L;
}

// First-level device wait limits set by phy_debug_set_wait_polls (negative: the defaults).
std::atomic<long long> g_wait_polls[2] = {{-1}, {-1}};

unsigned wait_polls(int kernel, unsigned dflt) {
  const long long v = g_wait_polls[kernel].load(std::memory_order_relaxed);
  return v < 0 ? dflt : (unsigned)std::min<long long>(v, 0xFFFFFFFFll);
}

// Validates cfg and fills g. Returns PHY_OK, PHY_ERR_INVALID_ARG or PHY_ERR_UNSUPPORTED.
phy_status make_geo(const phy_slot_cfg* c, Geo* g) {
  if (!c) return PHY_ERR_INVALID_ARG;
  if (c->n_cells < 1 || c->n_cells > 65535) return PHY_ERR_INVALID_ARG;
  if (c->n_prb < 1 || c->n_prb > 275) return PHY_ERR_INVALID_ARG;
  if (c->n_sym < 1 || c->n_sym > phy::kMaxSym) return PHY_ERR_INVALID_ARG;
  if (c->n_rx < 1 || c->n_rx > phy::kMaxRx) return PHY_ERR_INVALID_ARG;
  if (c->n_layers < 1 || c->n_layers > phy::kMaxLayers || c->n_layers > c->n_rx)
    return PHY_ERR_INVALID_ARG;
  if (c->qm != 2 && c->qm != 4 && c->qm != 6 && c->qm != 8) return PHY_ERR_INVALID_ARG;
  if (c->n_dmrs != 1 && c->n_dmrs != 2) return PHY_ERR_INVALID_ARG;
  for (int d = 0; d < c->n_dmrs; ++d)
    if (c->dmrs_sym[d] < 0 || c->dmrs_sym[d] >= c->n_sym) return PHY_ERR_INVALID_ARG;
  if (c->n_dmrs == 2 && c->dmrs_sym[1] <= c->dmrs_sym[0]) return PHY_ERR_INVALID_ARG;
  if (c->precision < PHY_PREC_FP32 || c->precision > PHY_PREC_TC_FP16) return PHY_ERR_INVALID_ARG;
  if (!(c->pivot_ratio_min >= 0.f) || c->pivot_ratio_min > 1.f) return PHY_ERR_INVALID_ARG;
  const int need = auto_occ(c->n_layers);
  const int L = c->occ_len == 0 ? need : c->occ_len;
  if (!pow2(L) || L < need || L > 16) return PHY_ERR_INVALID_ARG;
  const int n_sc = 12 * c->n_prb;
  const int n_comb = n_sc / 2;
  if (n_comb < L) return PHY_ERR_INVALID_ARG;
  Geo t;
  std::memset(&t, 0, sizeof(t));
  t.n_cells = c->n_cells;
  t.n_sc = n_sc;
  t.n_sym = c->n_sym;
  t.n_rx = c->n_rx;
  t.n_layers = c->n_layers;
  t.qm = c->qm;
  t.n_dmrs = c->n_dmrs;
  t.dmrs0 = c->dmrs_sym[0];
  t.dmrs1 = c->n_dmrs == 2 ? c->dmrs_sym[1] : c->dmrs_sym[0];
  t.L = L;
  t.n_comb = n_comb;
  t.G = (n_comb + L - 1) / L;
  t.n_seg = t.G > 1 ? t.G - 1 : 1;
  t.pivot_min = c->pivot_ratio_min;
  t.prec = c->precision;
  t.refactor = c->fp64_refactor ? 1 : 0;
  if (c->llr_format != PHY_LLR_F32 && c->llr_format != PHY_LLR_F16) return PHY_ERR_INVALID_ARG;
  t.llr_f16 = c->llr_format == PHY_LLR_F16;
  t.wait_seg = wait_polls(PHY_WAIT_SEGMENT_KERNEL, phy::kWaitSegDefault);
  t.wait_solve = wait_polls(PHY_WAIT_SOLVE_KERNEL, phy::kWaitSolveDefault);
  int nd = 0;
  for (int s = 0; s < c->n_sym; ++s) {
    bool is_dmrs = false;
    for (int d = 0; d < c->n_dmrs; ++d) is_dmrs |= (c->dmrs_sym[d] == s);
    if (is_dmrs) continue;
    t.dsym[nd] = s;
    if (c->n_dmrs == 2) {
      double a = (double)(s - t.dmrs0) / (double)(t.dmrs1 - t.dmrs0);
      a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
      t.tw[nd] = (float)a;
    } else {
      t.tw[nd] = 0.f;
    }
    ++nd;
  }
  t.n_dsym = nd;
  if (nd < 1) return PHY_ERR_INVALID_ARG;
  *g = t;
  return PHY_OK;
}

size_t anchor_bytes(const Geo& g) {
  return (size_t)g.n_cells * g.n_dmrs * g.G * g.n_layers * g.n_rx * sizeof(phy_c32);
}

phy_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PHY_OK : PHY_ERR_CUDA; }

phy_status check_shape(const Geo& g) {
  if (phy::fused_fp32_smem_bytes(g) > 227 * 1024) return PHY_ERR_UNSUPPORTED;
  if (g.prec != PHY_PREC_FP32 && !phy::seg_prep_tc_supported(g)) return PHY_ERR_UNSUPPORTED;
  return PHY_OK;
}

// Workspace layout: anchors | noise-estimate partial sums | detection scratch (one chunk).
size_t head_bytes(const Geo& g) {
  return align_up(anchor_bytes(g)) + align_up(phy::noise_scratch_bytes(g));
}

size_t workspace_for_chunk(const Geo& g, int chunk) {
  return head_bytes(g) + align_up(phy::detect_scratch_bytes(g, chunk));
}

phy_status check_noise_mode(const Geo& g, int mode) {
  if (mode < PHY_NOISE_FREQ || mode > PHY_NOISE_MIN) return PHY_ERR_INVALID_ARG;
  if (mode == PHY_NOISE_TIME && g.n_dmrs != 2) return PHY_ERR_INVALID_ARG;
  return PHY_OK;
}

// ---------------------------------------------------------------- autotuner table
// Key: every Geo field that shapes the work (sizes, symbols, DMRS, cover, precision, refactor).
struct TuneKey {
  int v[12];
  bool operator<(const TuneKey& o) const {
    for (int i = 0; i < 12; ++i)
      if (v[i] != o.v[i]) return v[i] < o.v[i];
    return false;
  }
};
TuneKey tune_key(const Geo& g) {
  return TuneKey{{g.n_cells, g.n_sc, g.n_sym, g.n_rx, g.n_layers, g.qm, g.n_dmrs, g.dmrs0,
                  g.dmrs1, g.L, g.prec, g.refactor}};
}
std::mutex g_tune_mu;
std::map<TuneKey, phy::Tile> g_tuned;

}  // namespace

namespace phy {

Tile tuned_tile(const Geo& g) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(tune_key(g));
  return it == g_tuned.end() ? Tile{0, 0, 0} : it->second;
}

size_t min_workspace_bytes(const phy_slot_cfg* cfg) {
  Geo g;
  if (make_geo(cfg, &g) != PHY_OK) return 0;
  return workspace_for_chunk(g, 1);
}

phy_status slot_run_fit(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                        const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                        uint8_t* flags, void* workspace, size_t workspace_bytes,
                        cudaStream_t st) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!Y || !pilots || !sigma2 || !flags || !workspace || ((uintptr_t)Y % 16))
    return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < workspace_for_chunk(g, 1)) return PHY_ERR_NO_MEMORY;
  s = check_shape(g);
  if (s != PHY_OK) return s;
  phy_c32* anchors = (phy_c32*)workspace;
  const size_t a = head_bytes(g);
  cudaError_t e = launch_chest(g, Y, pilots, anchors, st);
  if (e != cudaSuccess) return PHY_ERR_CUDA;
  e = launch_detect(g, anchors, Y, sigma2, x_hat, sinr, llr, flags,
                    static_cast<char*>(workspace) + a, workspace_bytes - a,
                    kStageGramMf | kStageSolve, st);
  return cuda_status(e);
}

}  // namespace phy

namespace phy {
phy_status make_geo_checked(const phy_slot_cfg* cfg, Geo* g) {
  const phy_status s = make_geo(cfg, g);
  return s != PHY_OK ? s : check_shape(*g);
}
}  // namespace phy

extern "C" {

phy_status phy_debug_set_wait_polls(int32_t kernel, int64_t polls) {
  if (kernel != PHY_WAIT_SEGMENT_KERNEL && kernel != PHY_WAIT_SOLVE_KERNEL)
    return PHY_ERR_INVALID_ARG;
  g_wait_polls[kernel].store(polls < 0 ? -1 : (long long)polls, std::memory_order_relaxed);
  return PHY_OK;
}

const char* phy_status_str(phy_status s) {
  switch (s) {
    case PHY_OK: return "ok";
    case PHY_ERR_INVALID_ARG: return "invalid argument";
    case PHY_ERR_UNSUPPORTED: return "unsupported configuration";
    case PHY_ERR_NO_MEMORY: return "workspace too small";
    case PHY_ERR_CUDA: return "CUDA error";
    case PHY_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

int32_t phy_n_groups(const phy_slot_cfg* cfg) {
  Geo g;
  return make_geo(cfg, &g) == PHY_OK ? g.G : -1;
}

int32_t phy_n_data_symbols(const phy_slot_cfg* cfg) {
  Geo g;
  return make_geo(cfg, &g) == PHY_OK ? g.n_dsym : -1;
}

size_t phy_workspace_size(const phy_slot_cfg* cfg) {
  Geo g;
  if (make_geo(cfg, &g) != PHY_OK) return 0;
  return workspace_for_chunk(g, phy::detect_preferred_chunk(g));
}

phy_status phy_chest(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                     phy_c32* anchors, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!Y || !pilots || !anchors || ((uintptr_t)Y % 16)) return PHY_ERR_INVALID_ARG;
  return cuda_status(phy::launch_chest(g, Y, pilots, anchors, (cudaStream_t)stream));
}

phy_status phy_mmse_detect(const phy_slot_cfg* cfg, const phy_c32* H, const phy_c32* Y,
                           const float* sigma2, phy_c32* x_hat, float* sinr, uint8_t* flags,
                           void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!H || !Y || !sigma2 || !x_hat || !sinr || !flags) return PHY_ERR_INVALID_ARG;
  return cuda_status(
      phy::launch_detect_h(g, H, Y, sigma2, x_hat, sinr, flags, (cudaStream_t)stream));
}

phy_status phy_llr_demap(const phy_slot_cfg* cfg, const phy_c32* x_hat, const float* sinr,
                         float* llr, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!x_hat || !sinr || !llr) return PHY_ERR_INVALID_ARG;
  return cuda_status(phy::launch_llr(g, x_hat, sinr, llr, (cudaStream_t)stream));
}

phy_status phy_detect_anchors(const phy_slot_cfg* cfg, const phy_c32* anchors, const phy_c32* Y,
                              const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                              uint8_t* flags, void* workspace, size_t workspace_bytes,
                              void* stream) {
  return phy_detect_stage(cfg, -1, anchors, Y, sigma2, x_hat, sinr, llr, flags, workspace,
                          workspace_bytes, stream);
}

int32_t phy_stage_supported(const phy_slot_cfg* cfg) {
  Geo g;
  if (make_geo(cfg, &g) != PHY_OK) return 0;
  return phy::detect_preferred_chunk(g) == g.n_cells ? 1 : 0;
}

phy_status phy_detect_stage(const phy_slot_cfg* cfg, int32_t stage, const phy_c32* anchors,
                            const phy_c32* Y, const float* sigma2, phy_c32* x_hat, float* sinr,
                            float* llr, uint8_t* flags, void* workspace, size_t workspace_bytes,
                            void* stream) {
  // stage -1 (internal): both stages, chunked as the workspace allows
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (stage < -1 || stage > PHY_STAGE_SOLVE) return PHY_ERR_INVALID_ARG;
  if (!anchors || !Y || !sigma2 || !flags || !workspace) return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign || ((uintptr_t)Y % 16) || ((uintptr_t)anchors % 16))
    return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  if (stage >= 0 && !phy_stage_supported(cfg)) return PHY_ERR_UNSUPPORTED;
  s = check_shape(g);
  if (s != PHY_OK) return s;
  const int stages = stage < 0 ? (phy::kStageGramMf | phy::kStageSolve)
                               : (stage == PHY_STAGE_GRAM_MF ? phy::kStageGramMf
                                                             : phy::kStageSolve);
  const size_t a = head_bytes(g);
  return cuda_status(phy::launch_detect(g, anchors, Y, sigma2, x_hat, sinr, llr, flags,
                                        static_cast<char*>(workspace) + a, workspace_bytes - a,
                                        stages, (cudaStream_t)stream));
}

phy_status phy_slot_run(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                        const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                        uint8_t* flags, void* workspace, size_t workspace_bytes, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!Y || !pilots || !sigma2 || !flags || !workspace || ((uintptr_t)Y % 16))
    return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  return phy::slot_run_fit(cfg, Y, pilots, sigma2, x_hat, sinr, llr, flags, workspace,
                           workspace_bytes, (cudaStream_t)stream);
}

phy_status phy_noise_est(const phy_slot_cfg* cfg, int32_t mode, const phy_c32* anchors,
                         const phy_c32* pilots, float* sigma2_out, void* workspace,
                         size_t workspace_bytes, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  s = check_noise_mode(g, mode);
  if (s != PHY_OK) return s;
  if (!anchors || !pilots || !sigma2_out || !workspace) return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  return cuda_status(phy::launch_noise_est(g, mode, 1.f, anchors, pilots, sigma2_out,
                                           static_cast<char*>(workspace) +
                                               align_up(anchor_bytes(g)),
                                           (cudaStream_t)stream));
}

phy_status phy_noise_track(const phy_slot_cfg* cfg, int32_t mode, float alpha,
                           const phy_c32* anchors, const phy_c32* pilots, float* sigma2_state,
                           void* workspace, size_t workspace_bytes, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  s = check_noise_mode(g, mode);
  if (s != PHY_OK) return s;
  if (!(alpha > 0.f && alpha <= 1.f)) return PHY_ERR_INVALID_ARG;
  if (!anchors || !pilots || !sigma2_state || !workspace) return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  return cuda_status(phy::launch_noise_est(g, mode, alpha, anchors, pilots, sigma2_state,
                                           static_cast<char*>(workspace) +
                                               align_up(anchor_bytes(g)),
                                           (cudaStream_t)stream));
}

phy_status phy_slot_run_track(const phy_slot_cfg* cfg, int32_t mode, float alpha,
                              const phy_c32* Y, const phy_c32* pilots, float* sigma2_state,
                              phy_c32* x_hat, float* sinr, float* llr, uint8_t* flags,
                              void* workspace, size_t workspace_bytes, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  s = check_noise_mode(g, mode);
  if (s != PHY_OK) return s;
  if (!(alpha > 0.f && alpha <= 1.f)) return PHY_ERR_INVALID_ARG;
  if (!Y || !pilots || !sigma2_state || !flags || !workspace || ((uintptr_t)Y % 16))
    return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  s = check_shape(g);
  if (s != PHY_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  phy_c32* anchors = (phy_c32*)workspace;
  char* ws = static_cast<char*>(workspace);
  cudaError_t e = phy::launch_chest(g, Y, pilots, anchors, st);
  if (e == cudaSuccess)
    e = phy::launch_noise_est(g, mode, alpha, anchors, pilots, sigma2_state,
                              ws + align_up(anchor_bytes(g)), st);
  if (e == cudaSuccess)
    e = phy::launch_detect(g, anchors, Y, sigma2_state, x_hat, sinr, llr, flags,
                           ws + head_bytes(g), workspace_bytes - head_bytes(g),
                           phy::kStageGramMf | phy::kStageSolve, st);
  return cuda_status(e);
}

phy_status phy_slot_run_est(const phy_slot_cfg* cfg, int32_t mode, const phy_c32* Y,
                            const phy_c32* pilots, float* sigma2_out, phy_c32* x_hat,
                            float* sinr, float* llr, uint8_t* flags, void* workspace,
                            size_t workspace_bytes, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  s = check_noise_mode(g, mode);
  if (s != PHY_OK) return s;
  if (!Y || !pilots || !sigma2_out || !flags || !workspace || ((uintptr_t)Y % 16))
    return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  s = check_shape(g);
  if (s != PHY_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  phy_c32* anchors = (phy_c32*)workspace;
  char* ws = static_cast<char*>(workspace);
  cudaError_t e = phy::launch_chest(g, Y, pilots, anchors, st);
  if (e == cudaSuccess)
    e = phy::launch_noise_est(g, mode, 1.f, anchors, pilots, sigma2_out,
                              ws + align_up(anchor_bytes(g)), st);
  if (e == cudaSuccess)
    e = phy::launch_detect(g, anchors, Y, sigma2_out, x_hat, sinr, llr, flags,
                           ws + head_bytes(g), workspace_bytes - head_bytes(g),
                           phy::kStageGramMf | phy::kStageSolve, st);
  return cuda_status(e);
}

size_t phy_bfp_bytes(const phy_slot_cfg* cfg, int32_t iq_width) {
  Geo g;
  if (make_geo(cfg, &g) != PHY_OK || iq_width < 1 || iq_width > 16) return 0;
  return (size_t)g.n_cells * g.n_sym * g.n_rx * (g.n_sc / 12) * (size_t)(1 + 3 * iq_width);
}

namespace {
phy_status check_bfp(int32_t iq_width, float scale, const uint8_t* Yc) {
  if (iq_width < 1 || iq_width > 16) return PHY_ERR_INVALID_ARG;
  if (!(scale > 0.f) || !(scale < 3.0e38f)) return PHY_ERR_INVALID_ARG;
  if (!Yc || ((uintptr_t)Yc % 4)) return PHY_ERR_INVALID_ARG;
  return PHY_OK;
}
}  // namespace

phy_status phy_bfp_decompress(const phy_slot_cfg* cfg, const uint8_t* Yc, int32_t iq_width,
                              float scale, int32_t data_only, phy_c32* Y, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  s = check_bfp(iq_width, scale, Yc);
  if (s != PHY_OK) return s;
  if (!Y || ((uintptr_t)Y % 16)) return PHY_ERR_INVALID_ARG;
  return cuda_status(phy::launch_bfp_decompress(g, Yc, iq_width, scale, data_only ? 1 : 0, Y,
                                                (cudaStream_t)stream));
}

phy_status phy_chest_bfp(const phy_slot_cfg* cfg, const uint8_t* Yc, int32_t iq_width,
                         float scale, const phy_c32* pilots, phy_c32* anchors, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  s = check_bfp(iq_width, scale, Yc);
  if (s != PHY_OK) return s;
  if (!pilots || !anchors) return PHY_ERR_INVALID_ARG;
  return cuda_status(phy::launch_chest_bfp(g, Yc, iq_width, scale, pilots, anchors,
                                           (cudaStream_t)stream));
}

phy_status phy_slot_run_bfp(const phy_slot_cfg* cfg, const uint8_t* Yc, int32_t iq_width,
                            float scale, phy_c32* Y, const phy_c32* pilots, const float* sigma2,
                            phy_c32* x_hat, float* sinr, float* llr, uint8_t* flags,
                            void* workspace, size_t workspace_bytes, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  s = check_bfp(iq_width, scale, Yc);
  if (s != PHY_OK) return s;
  if (!Y || !pilots || !sigma2 || !flags || !workspace || ((uintptr_t)Y % 16))
    return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  s = check_shape(g);
  if (s != PHY_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  phy_c32* anchors = (phy_c32*)workspace;
  // Decoding the whole grid and estimating from it beats decoding the data symbols and
  // estimating from the stream: the DMRS rows cost the decoder a few microseconds, while the LS
  // kernel's per-antenna runs cut across the compressed blocks.
  cudaError_t e = phy::launch_bfp_decompress(g, Yc, iq_width, scale, 0, Y, st);
  if (e == cudaSuccess) e = phy::launch_chest(g, Y, pilots, anchors, st);
  if (e == cudaSuccess)
    e = phy::launch_detect(g, anchors, Y, sigma2, x_hat, sinr, llr, flags,
                           static_cast<char*>(workspace) + head_bytes(g),
                           workspace_bytes - head_bytes(g), phy::kStageGramMf | phy::kStageSolve,
                           st);
  return cuda_status(e);
}

phy_status phy_slot_run_bfp_host(const phy_slot_cfg* cfg, const uint8_t* Yc_host,
                                 int32_t iq_width, float scale, const phy_c32* pilots_host,
                                 const float* sigma2_host, float* llr_host, uint8_t* flags_host,
                                 uint8_t* Yc, phy_c32* Y, phy_c32* pilots, float* sigma2,
                                 phy_c32* x_hat, float* sinr, float* llr, uint8_t* flags,
                                 void* workspace, size_t workspace_bytes, void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!Yc_host || !pilots_host || !sigma2_host || !llr_host || !flags_host || !pilots ||
      !sigma2 || !llr || !flags)
    return PHY_ERR_INVALID_ARG;
  s = check_bfp(iq_width, scale, Yc);
  if (s != PHY_OK) return s;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  s = check_shape(g);
  if (s != PHY_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t c_bytes = phy_bfp_bytes(cfg, iq_width);
  const size_t p_bytes = (size_t)g.n_cells * g.n_dmrs * g.n_layers * g.n_sc * sizeof(phy_c32);
  const size_t n_re = (size_t)g.n_cells * g.n_dsym * g.n_sc;
  const size_t l_bytes = n_re * g.n_layers * g.qm * (g.llr_f16 ? 2 : sizeof(float));
  if (cudaMemcpyAsync(Yc, Yc_host, c_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(pilots, pilots_host, p_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(sigma2, sigma2_host, g.n_cells * sizeof(float), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return PHY_ERR_CUDA;
  s = phy_slot_run_bfp(cfg, Yc, iq_width, scale, Y, pilots, sigma2, x_hat, sinr, llr, flags,
                       workspace, workspace_bytes, stream);
  if (s != PHY_OK) return s;
  if (cudaMemcpyAsync(llr_host, llr, l_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(flags_host, flags, n_re, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PHY_ERR_CUDA;
  return PHY_OK;
}

// ---------------------------------------------------------------- learned channel denoiser
int32_t phy_cnn_param_count(void) { return phy::cnn_param_count(); }

size_t phy_cnn_workspace_size(int32_t n_tiles) {
  if (n_tiles < 1) return 0;
  return phy::cnn_scratch_floats(n_tiles) * sizeof(float);
}

phy_status phy_cnn_forward(int32_t n_tiles, const float* params, const float* tiles_in,
                           float* tiles_out, void* workspace, size_t workspace_bytes,
                           void* stream) {
  if (n_tiles < 1 || !params || !tiles_in || !tiles_out || !workspace) return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_cnn_workspace_size(n_tiles)) return PHY_ERR_NO_MEMORY;
  return cuda_status(phy::cnn_forward(n_tiles, params, tiles_in, tiles_out, (float*)workspace,
                                      (cudaStream_t)stream));
}

phy_status phy_cnn_train_step(int32_t n_tiles, float* params, float* adam_m, float* adam_v,
                              int32_t step, float lr, const float* tiles_in,
                              const float* tiles_label, float* grad, float* grad_in,
                              float* loss, void* workspace, size_t workspace_bytes,
                              void* stream) {
  if (n_tiles < 1 || !params || !tiles_in || !tiles_label || !grad || !workspace)
    return PHY_ERR_INVALID_ARG;
  if (step > 0 && (!adam_m || !adam_v || !(lr >= 0.f))) return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_cnn_workspace_size(n_tiles)) return PHY_ERR_NO_MEMORY;
  return cuda_status(phy::cnn_train_step(n_tiles, params, adam_m, adam_v, step, lr, tiles_in,
                                         tiles_label, grad, grad_in, loss, (float*)workspace,
                                         (cudaStream_t)stream));
}

phy_status phy_cnn_train_step_bf16(int32_t n_tiles, float* params, float* adam_m, float* adam_v,
                                   int32_t step, float lr, const float* tiles_in,
                                   const float* tiles_label, float* grad, float* grad_in,
                                   float* loss, void* workspace, size_t workspace_bytes,
                                   void* stream) {
  if (n_tiles < 1 || !params || !tiles_in || !tiles_label || !grad || !workspace)
    return PHY_ERR_INVALID_ARG;
  if (step > 0 && (!adam_m || !adam_v || !(lr >= 0.f))) return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_cnn_workspace_size(n_tiles)) return PHY_ERR_NO_MEMORY;
  return cuda_status(phy::cnn_train_step(n_tiles, params, adam_m, adam_v, step, lr, tiles_in,
                                         tiles_label, grad, grad_in, loss, (float*)workspace,
                                         (cudaStream_t)stream, true));
}

size_t phy_cnn_train_error_offset(int32_t n_tiles) {
  return n_tiles < 1 ? 0 : phy::cnn_train_error_float(n_tiles) * sizeof(float);
}

namespace {
phy_status check_tiles(const phy_slot_cfg* cfg, Geo* g) {
  phy_status s = make_geo(cfg, g);
  if (s != PHY_OK) return s;
  if (g->n_sym != 14) return PHY_ERR_UNSUPPORTED;  // tiles span the 14 symbols of a slot
  return PHY_OK;
}
}  // namespace

int32_t phy_cnn_n_tiles(const phy_slot_cfg* cfg) {
  Geo g;
  if (check_tiles(cfg, &g) != PHY_OK) return -1;
  return g.n_cells * (g.n_sc / 12) * g.n_rx * g.n_layers;
}

phy_status phy_interp_channel(const phy_slot_cfg* cfg, const phy_c32* anchors, phy_c32* H,
                              void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!anchors || !H) return PHY_ERR_INVALID_ARG;
  return cuda_status(phy::launch_interp_all(g, anchors, H, (cudaStream_t)stream));
}

phy_status phy_cnn_tiles(const phy_slot_cfg* cfg, const phy_c32* H, float* tiles, void* stream) {
  Geo g;
  phy_status s = check_tiles(cfg, &g);
  if (s != PHY_OK) return s;
  if (!H || !tiles) return PHY_ERR_INVALID_ARG;
  return cuda_status(phy::launch_tiles_from_h(g, H, tiles, (cudaStream_t)stream));
}

phy_status phy_cnn_untile(const phy_slot_cfg* cfg, const float* tiles, phy_c32* H_data,
                          void* stream) {
  Geo g;
  phy_status s = check_tiles(cfg, &g);
  if (s != PHY_OK) return s;
  if (!tiles || !H_data) return PHY_ERR_INVALID_ARG;
  return cuda_status(phy::launch_tiles_to_h(g, tiles, H_data, (cudaStream_t)stream));
}

size_t phy_cnn_denoise_workspace_size(const phy_slot_cfg* cfg) {
  Geo g;
  if (check_tiles(cfg, &g) != PHY_OK) return 0;
  const size_t n = (size_t)g.n_cells * (g.n_sc / 12) * g.n_rx * g.n_layers;
  const size_t h = (size_t)g.n_cells * g.n_sym * g.n_sc * g.n_rx * g.n_layers * sizeof(phy_c32);
  return align_up(h) + 2 * align_up(n * 2 * 168 * sizeof(float)) +
         phy::cnn_scratch_floats((int)n) * sizeof(float);
}

phy_status phy_cnn_denoise(const phy_slot_cfg* cfg, const float* params, const phy_c32* anchors,
                           phy_c32* H_data, void* workspace, size_t workspace_bytes,
                           void* stream) {
  Geo g;
  phy_status s = check_tiles(cfg, &g);
  if (s != PHY_OK) return s;
  if (!params || !anchors || !H_data || !workspace) return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_cnn_denoise_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  const int n = g.n_cells * (g.n_sc / 12) * g.n_rx * g.n_layers;
  const size_t h = (size_t)g.n_cells * g.n_sym * g.n_sc * g.n_rx * g.n_layers * sizeof(phy_c32);
  char* ws = static_cast<char*>(workspace);
  phy_c32* H = (phy_c32*)ws;
  float* t_in = (float*)(ws + align_up(h));
  float* t_out = (float*)(ws + align_up(h) + align_up((size_t)n * 2 * 168 * sizeof(float)));
  float* scratch = (float*)(ws + align_up(h) + 2 * align_up((size_t)n * 2 * 168 * sizeof(float)));
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = phy::launch_interp_all(g, anchors, H, st);
  if (e == cudaSuccess) e = phy::launch_tiles_from_h(g, H, t_in, st);
  if (e == cudaSuccess) e = phy::cnn_forward(n, params, t_in, t_out, scratch, st);
  if (e == cudaSuccess) e = phy::launch_tiles_to_h(g, t_out, H_data, st);
  return cuda_status(e);
}

phy_status phy_cnn_forward_bf16(int32_t n_tiles, const float* params, const float* tiles_in,
                                float* tiles_out, void* workspace, size_t workspace_bytes,
                                void* stream) {
  if (n_tiles < 0 || !params || (n_tiles > 0 && (!tiles_in || !tiles_out)) || !workspace)
    return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % 4) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < sizeof(unsigned)) return PHY_ERR_NO_MEMORY;
  return cuda_status(phy::cnn_forward_tc(n_tiles, params, tiles_in, tiles_out,
                                         (unsigned*)workspace, (cudaStream_t)stream));
}

phy_status phy_cnn_denoise_bf16(const phy_slot_cfg* cfg, const float* params,
                                const phy_c32* anchors, phy_c32* H_data, void* workspace,
                                size_t workspace_bytes, void* stream) {
  Geo g;
  phy_status s = check_tiles(cfg, &g);
  if (s != PHY_OK) return s;
  if (!params || !anchors || !H_data || !workspace) return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_cnn_denoise_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  const int n = g.n_cells * (g.n_sc / 12) * g.n_rx * g.n_layers;
  const size_t h = (size_t)g.n_cells * g.n_sym * g.n_sc * g.n_rx * g.n_layers * sizeof(phy_c32);
  char* ws = static_cast<char*>(workspace);
  phy_c32* H = (phy_c32*)ws;
  float* t_in = (float*)(ws + align_up(h));
  float* t_out = (float*)(ws + align_up(h) + align_up((size_t)n * 2 * 168 * sizeof(float)));
  // the error word sits where the FP32 pass keeps its scratch
  unsigned* err =
      (unsigned*)(ws + align_up(h) + 2 * align_up((size_t)n * 2 * 168 * sizeof(float)));
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = phy::launch_interp_all(g, anchors, H, st);
  if (e == cudaSuccess) e = phy::launch_tiles_from_h(g, H, t_in, st);
  if (e == cudaSuccess) e = phy::cnn_forward_tc(n, params, t_in, t_out, err, st);
  if (e == cudaSuccess) e = phy::launch_tiles_to_h(g, t_out, H_data, st);
  return cuda_status(e);
}

size_t phy_cnn_denoise_error_offset(const phy_slot_cfg* cfg) {
  Geo g;
  if (check_tiles(cfg, &g) != PHY_OK) return 0;
  const int n = g.n_cells * (g.n_sc / 12) * g.n_rx * g.n_layers;
  const size_t h = (size_t)g.n_cells * g.n_sym * g.n_sc * g.n_rx * g.n_layers * sizeof(phy_c32);
  return align_up(h) + 2 * align_up((size_t)n * 2 * 168 * sizeof(float));
}

phy_status phy_slot_run_host(const phy_slot_cfg* cfg, const phy_c32* Y_host,
                             const phy_c32* pilots_host, const float* sigma2_host,
                             float* llr_host, uint8_t* flags_host, phy_c32* Y, phy_c32* pilots,
                             float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                             uint8_t* flags, void* workspace, size_t workspace_bytes,
                             void* stream) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!Y_host || !pilots_host || !sigma2_host || !llr_host || !flags_host || !Y || !pilots ||
      !sigma2 || !llr || !flags)
    return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  s = check_shape(g);
  if (s != PHY_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t y_bytes = (size_t)g.n_cells * g.n_sym * g.n_rx * g.n_sc * sizeof(phy_c32);
  const size_t p_bytes = (size_t)g.n_cells * g.n_dmrs * g.n_layers * g.n_sc * sizeof(phy_c32);
  const size_t n_re = (size_t)g.n_cells * g.n_dsym * g.n_sc;
  const size_t l_bytes = n_re * g.n_layers * g.qm * (g.llr_f16 ? 2 : sizeof(float));
  if (cudaMemcpyAsync(Y, Y_host, y_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(pilots, pilots_host, p_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(sigma2, sigma2_host, g.n_cells * sizeof(float), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return PHY_ERR_CUDA;
  s = phy_slot_run(cfg, Y, pilots, sigma2, x_hat, sinr, llr, flags, workspace, workspace_bytes,
                   stream);
  if (s != PHY_OK) return s;
  if (cudaMemcpyAsync(llr_host, llr, l_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(flags_host, flags, n_re, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PHY_ERR_CUDA;
  return PHY_OK;
}

phy_status phy_autotune(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                        const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                        uint8_t* flags, void* workspace, size_t workspace_bytes, void* stream,
                        int32_t* chunk_out) {
  Geo g;
  phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (!Y || !pilots || !sigma2 || !flags || !workspace || ((uintptr_t)Y % 16))
    return PHY_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % kAlign) return PHY_ERR_INVALID_ARG;
  if (workspace_bytes < phy_workspace_size(cfg)) return PHY_ERR_NO_MEMORY;
  s = check_shape(g);
  if (s != PHY_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PHY_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PHY_ERR_CUDA;
  }
  const TuneKey key = tune_key(g);
  phy_status rs = PHY_OK;
  // median of three timed runs (after one warm-up) with tile t in force; < 0 on an error
  auto trial = [&](const phy::Tile& t) -> float {
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[key] = t;
    }
    float ms[3];
    for (int rep = -1; rep < 3 && rs == PHY_OK; ++rep) {
      if (rep >= 0 && cudaEventRecord(e0, st) != cudaSuccess) rs = PHY_ERR_CUDA;
      if (rs == PHY_OK)
        rs = phy::slot_run_fit(cfg, Y, pilots, sigma2, x_hat, sinr, llr, flags, workspace,
                               workspace_bytes, st);
      if (rep >= 0 && rs == PHY_OK) {
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms[rep], e0, e1) != cudaSuccess)
          rs = PHY_ERR_CUDA;
      }
    }
    if (rs != PHY_OK) return -1.f;
    std::sort(ms, ms + 3);
    return ms[1];
  };
  // coordinate search: cells per chunk with the default tiles, then the solve CTA width, then
  // (tensor-core products) the ring depth, each keeping the best so far
  phy::Tile best{0, 128, 0};
  float best_ms = -1.f;
  auto consider = [&](const phy::Tile& t) {
    const float ms = trial(t);
    if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
      best = t;
      best_ms = ms;
    }
  };
  std::vector<int> cand;
  for (int c = 1; c < g.n_cells; c *= 2) cand.push_back(c);
  cand.push_back(g.n_cells);
  for (int c : cand)
    if (rs == PHY_OK && workspace_for_chunk(g, c) <= workspace_bytes) consider({c, 128, 0});
  if (rs == PHY_OK && best.chunk > 0) consider({best.chunk, 64, 0});
  if (rs == PHY_OK && best.chunk > 0 && phy::tc_deep_ring_fits(g))
    consider({best.chunk, best.solve_w, 12});
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (rs == PHY_OK && best.chunk > 0)
      g_tuned[key] = best;
    else
      g_tuned.erase(key);
  }
  if (rs != PHY_OK) return rs;
  // leave the outputs as a plain call with the chosen tiles produces them
  rs = phy::slot_run_fit(cfg, Y, pilots, sigma2, x_hat, sinr, llr, flags, workspace,
                         workspace_bytes, st);
  if (rs != PHY_OK) return rs;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PHY_ERR_CUDA;
  if (chunk_out) *chunk_out = best.chunk;
  return PHY_OK;
}

phy_status phy_autotune_set_tiles(const phy_slot_cfg* cfg, int32_t chunk, int32_t solve_width,
                                  int32_t ring_stages) {
  Geo g;
  const phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  if (chunk < 0 || chunk > g.n_cells || (solve_width != 0 && solve_width != 64 &&
                                         solve_width != 128) ||
      (ring_stages != 0 && ring_stages != 12))
    return PHY_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[tune_key(g)] = phy::Tile{chunk, solve_width, ring_stages};
  return PHY_OK;
}

phy_status phy_autotune_tiles(const phy_slot_cfg* cfg, int32_t* chunk, int32_t* solve_width,
                              int32_t* ring_stages) {
  Geo g;
  const phy_status s = make_geo(cfg, &g);
  if (s != PHY_OK) return s;
  const phy::Tile t = phy::tuned_tile(g);
  if (chunk) *chunk = t.chunk;
  if (solve_width) *solve_width = t.solve_w;
  // the ring the kernel runs with: a pinned deeper ring that does not fit reads back as 0
  if (ring_stages) *ring_stages = t.ring == 12 && !phy::tc_deep_ring_fits(g) ? 0 : t.ring;
  return PHY_OK;
}

void phy_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.clear();
}

}  // extern "C"
