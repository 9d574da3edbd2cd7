// Host-side launchers of the receiver kernels (internal to libphy.so).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace phy {

// Kernel attributes (cudaFuncSetAttribute) and SM counts belong to a device: host-side caches of
// them are kept per device, indexed by the current device (ids below kMaxDevices).
constexpr int kMaxDevices = 64;
inline int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) d = 0;
  return d;
}
inline int device_sm_count() {
  static int sms[kMaxDevices] = {};
  const int d = current_device();
  if (sms[d] <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0)
      v = 1;
    sms[d] = v;
  }
  return sms[d];
}

// Widest frequency segment (subcarriers) for g, computed on the host.
int host_max_segment_width(const Geo& g);
// Dynamic shared memory of the FP32 segment kernel for g (bytes).
size_t fused_fp32_smem_bytes(const Geo& g);
// Detection runs in chunks of cells; its scratch holds one chunk's intermediates.
// Scratch bytes for chunks of `chunk` cells, and the chunk size the library prefers.
size_t detect_scratch_bytes(const Geo& g, int chunk);
int detect_preferred_chunk(const Geo& g);
// Tile shapes phy_autotune() chooses per geometry (each 0 where it was never tuned: the library
// default): cells per detection chunk, the solve kernel's CTA width (64 or 128 REs) and the
// tensor-core segment kernel's ring depth (stages of one 16-subcarrier box).
struct Tile {
  int chunk, solve_w, ring;
};
Tile tuned_tile(const Geo& g);

cudaError_t launch_chest(const Geo& g, const phy_c32* Y, const phy_c32* pilots, phy_c32* anchors,
                         cudaStream_t st);

// Interpolation + detection + SINR + LLRs from anchors, in the largest chunks of cells whose
// intermediates fit `scratch_bytes` (cudaErrorInvalidValue if not even one cell fits). `stages`
// selects the Gram/matched-filter kernel, the solve kernel or both; a single stage needs the
// whole batch in one chunk.
constexpr int kStageGramMf = 1, kStageSolve = 2;
cudaError_t launch_detect(const Geo& g, const phy_c32* anchors, const phy_c32* Y,
                          const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                          uint8_t* flags, void* scratch, size_t scratch_bytes, int stages,
                          cudaStream_t st);

// phy_slot_run with any workspace that holds the anchors and one cell's intermediates
// (chunks sized to fit); for callers inside the library.
phy_status slot_run_fit(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                        const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                        uint8_t* flags, void* workspace, size_t workspace_bytes,
                        cudaStream_t st);
// Smallest workspace slot_run_fit accepts for cfg (0 if cfg is invalid).
size_t min_workspace_bytes(const phy_slot_cfg* cfg);

// 3-D FP32 tensor map (dims and box innermost first, strides of dims 1 and 2 in bytes), no
// swizzle, zero fill outside the tensor; false if the driver refuses it.
bool make_map(CUtensorMap* m, const void* base, const cuuint64_t (&dim)[3],
              const cuuint64_t (&stride)[2], const cuuint32_t (&box)[3]);

// Tensor-core segment kernel (same outputs as the FP32 one) for g.prec != PHY_PREC_FP32.
// Needs an even antenna count and 16-byte aligned anchors and grid (TMA tensor maps).
bool seg_prep_tc_supported(const Geo& g);
// Whether the tensor-core segment kernel's deeper ring (12 stages) fits shared memory for g.
bool tc_deep_ring_fits(const Geo& g);
cudaError_t launch_seg_prep_tc(const Geo& g, int NL, int c0, int nc, const phy_c32* anchors,
                               const phy_c32* Y, float4* ygg, cf* bvec, unsigned* err,
                               cudaStream_t st);

// Noise-variance estimate per cell from the LS anchors and pilots (mode: phy_noise_mode) into
// sigma2_out (alpha = 1), or blended into it as a tracked state (alpha < 1); scratch holds
// noise_scratch_bytes(g) of partial sums.
size_t noise_scratch_bytes(const Geo& g);
cudaError_t launch_noise_est(const Geo& g, int mode, float alpha, const phy_c32* anchors,
                             const phy_c32* pilots, float* sigma2_out, void* scratch,
                             cudaStream_t st);

// Block-floating-point fronthaul stream (format in bfp.cuh): decompression into the grid Y
// (data_only: the DMRS symbols' rows are left untouched), and LS estimation read straight from
// the stream (anchors bitwise equal to launch_chest on the decompressed grid).
cudaError_t launch_bfp_decompress(const Geo& g, const uint8_t* yc, int w, float scale,
                                  int data_only, phy_c32* Y, cudaStream_t st);
cudaError_t launch_chest_bfp(const Geo& g, const uint8_t* yc, int w, float scale,
                             const phy_c32* pilots, phy_c32* anchors, cudaStream_t st);

// Learned channel denoiser (cnn.cu): flat FP32 parameters, tiles [n][C][14][12].
int cnn_param_count();
size_t cnn_scratch_floats(int n_tiles);
cudaError_t cnn_forward(int n, const float* params, const float* x, float* out, float* ws,
                        cudaStream_t st);
// With tc_forward the forward pass runs on the tensor cores (cnn_forward_tc, keeping its BF16
// activations for the FP32 backward pass) and its error word is the workspace's float at
// cnn_train_error_float(n).
cudaError_t cnn_train_step(int n, float* params, float* m, float* v, int step, float lr,
                           const float* x, const float* label, float* grad_out, float* dx_out,
                           float* loss_out, float* ws, cudaStream_t st, bool tc_forward = false);
size_t cnn_train_error_float(int n_tiles);
// The same forward pass on the tensor cores with BF16 operands (cnn_tc.cu); err (device word)
// is cleared first and counts CTAs whose bounded MMA wait ran out. With acts set, the outputs
// of the first three layers (as the next layer reads them, rounded to BF16) are also written in
// FP32 to acts[layer][tile][channel][position].
cudaError_t cnn_forward_tc(int n, const float* params, const float* x, float* out, unsigned* err,
                           cudaStream_t st, float* acts = nullptr);
// Interpolated channel at every symbol H[cell][t][k][r][l]; tiles per (cell, PRB, Rx, layer)
// from such an H, and the data symbols of tiles back into Hd[cell][dsym][k][r][l].
cudaError_t launch_interp_all(const Geo& g, const phy_c32* anchors, phy_c32* H, cudaStream_t st);
cudaError_t launch_tiles_from_h(const Geo& g, const phy_c32* H, float* tiles, cudaStream_t st);
cudaError_t launch_tiles_to_h(const Geo& g, const float* tiles, phy_c32* Hd, cudaStream_t st);

cudaError_t launch_detect_h(const Geo& g, const phy_c32* H, const phy_c32* Y, const float* sigma2,
                            phy_c32* x_hat, float* sinr, uint8_t* flags, cudaStream_t st);

cudaError_t launch_llr(const Geo& g, const phy_c32* x_hat, const float* sinr, float* llr,
                       cudaStream_t st);

// Validated geometry of a configuration (make_geo plus the shape checks of the single-job path).
phy_status make_geo_checked(const phy_slot_cfg* cfg, Geo* g);
// Kernel layer class (2, 4, 8 or 16) of a layer count.
int nl_class_of(int n_layers);
// 1 if that class runs the direct per-subcarrier form with FP32 products (no segment stage).
int batch_direct_class(int nl_cls);

// Batched receiver (batch.cuh holds the table). Per-job intermediate sizes and launch bounds,
// the batched LS kernel, and the per-class segment and solve kernels.
struct BatchTable;
size_t batch_anchor_bytes(const Geo& g);
size_t batch_ygg_bytes(const Geo& g);
size_t batch_bvec_bytes(const Geo& g);
int batch_wmax(const Geo& g);
int batch_max_segs(const Geo& g);
bool batch_geometry_fits(const Geo& g);
cudaError_t launch_chest_batch(const BatchTable* t, cudaStream_t st);
// The noise estimate of the jobs that track their noise level (partial sums, then per cell).
cudaError_t launch_noise_batch(const BatchTable* t, cudaStream_t st);
int noise_blocks(const Geo& g);  // partial-sum blocks per cell
cudaError_t launch_batch_stages(const BatchTable* t, cudaStream_t st);
// TMA tensor maps of the tensor-core segment kernel for a geometry's grid and anchors.
bool encode_tc_maps(const Geo& g, const phy_c32* anchors, const phy_c32* Y, CUtensorMap* tmY,
                    CUtensorMap* tmA);
// Whether the batched solve (after either segment kernel) and, for FP32 products, the batched
// FP32 segment kernel fit the captured launches' shared memory for g.
bool batch_solve_fits(const Geo& g);
// The batched tensor-core segment kernel (FP16 products, two DMRS symbols) of one layer class.
cudaError_t launch_seg_prep_tc_batch(const BatchTable* t, int nl_cls, cudaStream_t st);

}  // namespace phy
