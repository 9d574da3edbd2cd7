/*
 * phy.h - C ABI of the GB300 uplink receiver library (libphy.so).
 *
 * The library runs the uplink PUSCH receiver inner loop that the paper accelerates with CPU SIMD:
 * DMRS least-squares channel estimation with linear frequency/time interpolation, per-resource-
 * element (RE) LMMSE MIMO detection (Gram matrix H^H H + s2 I, Cholesky, triangular solves,
 * equalisation W y, per-layer post-equalisation SINR), and max-log QAM LLR demapping over the NR
 * Gray constellations. The paper's LMMSE block is Sec. IV and Fig. 3 (covariance inversion by
 * LU with forward/backward substitution); its covariance-by-FMA step is Fig. 2(b); it names
 * channel estimation as a SIMD target in Sec. III-B. The estimation, interpolation and demapping
 * rules below are this library's readings where the paper gives no method.
 *
 * Conventions for every entry point:
 *  - All array arguments are DEVICE pointers owned by the caller, except where a name ends in
 *    _host. The library never allocates device memory; scratch space is a caller-provided
 *    workspace of phy_workspace_size() bytes (256-byte aligned). Y and caller-supplied anchors
 *    must be 16-byte aligned.
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL = legacy default stream)
 *    and the call returns without synchronising. Results are valid once the stream reaches
 *    the point after the call.
 *  - Arguments are validated on the host before anything is enqueued. A failed validation
 *    returns PHY_ERR_INVALID_ARG (bad sizes or pointers) or PHY_ERR_UNSUPPORTED (a valid but
 *    unimplemented shape) and enqueues nothing. A CUDA launch error returns PHY_ERR_CUDA.
 *  - Some kernels use the SM's tensor memory (TMEM): the tensor-core segment kernels and the
 *    denoiser's tensor-core forward pass for their accumulators, and the 9..16-layer solve of
 *    phy_slot_run / phy_detect_stage (128-subcarrier CTAs) for per-RE scratch, each CTA
 *    allocating at start and releasing before it ends. Another kernel that allocates tensor
 *    memory and runs at the same time on another stream (the caller's, or this library's on
 *    another stream) may wait for those columns. No kernel of this library waits for another
 *    kernel while it holds tensor memory, so this can delay work but not deadlock it.
 *  - Numerical trouble is data, not an error: it is reported per RE in `flags`
 *    (bit 0: ill-conditioned Gram matrix, Cholesky pivot ratio below cfg.pivot_ratio_min or a
 *    non-positive pivot; bit 1: RE re-computed in FP64; bit 2: non-finite input). An RE whose
 *    factorisation fails in FP32 and is not re-computed gets zero x_hat, SINR and LLRs.
 *    Bit 3 (alone) marks an RE whose results were never written because a bounded device wait
 *    in the detection kernels timed out (a stalled copy or tensor-core operation); its x_hat,
 *    SINR and LLRs hold whatever the buffers held before.
 *
 * Layouts (complex values are interleaved float pairs, phy_c32):
 *  Y        [cell][sym][rx][sc]                     received grid, all n_sym symbols
 *  pilots   [cell][dmrs][layer][sc]                 DMRS values; 0 off the layer's comb
 *  anchors  [cell][dmrs][group][layer][rx]          LS channel estimates
 *  H        [cell][dsym][sc][rx][layer]             full channel (phy_mmse_detect only)
 *  x_hat    [cell][dsym][sc][layer]                 biased LMMSE output W y
 *  sinr     [cell][dsym][sc][layer]      float      post-equalisation SINR
 *  llr      [cell][dsym][sc][layer][qm]  float      max-log LLRs, positive = bit 0 (IEEE
 *                                                   binary16 with cfg.llr_format = PHY_LLR_F16)
 *  flags    [cell][dsym][sc]             uint8      see above
 *  sigma2   [cell]                       float      noise variance per Rx per RE (given, or
 *                                                   estimated by phy_noise_est)
 * `dsym` counts data symbols only: the symbols 0..n_sym-1 that are not DMRS symbols, in order.
 *
 * DMRS and estimation rules: layer l uses comb c = l % 2 (subcarriers k = 2m + c) and Walsh row
 * o = l / 2 of length L = occ_len (0 selects the smallest power of two >= ceil(n_layers/2)).
 * LS group g covers comb indices m = s_g .. s_g + L - 1, s_g = min(L g, n_sc/2 - L) (the last
 * group overlaps its neighbour), with the estimate (1/L) sum Y conj(pilot) placed at subcarrier
 * 2 s_g + L - 1 + c. Frequency interpolation is linear between a layer's neighbouring anchors and
 * holds the end values; time interpolation with two DMRS symbols d0 < d1 is linear with weight
 * clamp((t - d0)/(d1 - d0), 0, 1) on d1, and holds with one DMRS symbol.
 *
 * Per-layer outputs: with e_k = s2 (A^-1)_kk clamped to [1e-30, 1 - 1e-7], mu_k = 1 - e_k,
 * SINR_k = mu_k / e_k; the LLRs use x~_k = x_hat_k / mu_k and noise e_k / mu_k.
 */
#ifndef PHY_H
#define PHY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  float re;
  float im;
} phy_c32;

typedef enum {
  PHY_OK = 0,
  PHY_ERR_INVALID_ARG = 1,
  PHY_ERR_UNSUPPORTED = 2,
  PHY_ERR_NO_MEMORY = 3, /* workspace smaller than phy_workspace_size() */
  PHY_ERR_CUDA = 4,
  PHY_ERR_TIMEOUT = 5
} phy_status;

typedef enum {
  PHY_PREC_FP32 = 0,    /* every product on FP32 CUDA cores */
  /* Gram and H^H y products on tcgen05 tensor cores, TF32 in, FP32 accumulation. The operands
     are streamed by TMA tensor copies, which need an even n_rx (PHY_ERR_UNSUPPORTED otherwise). */
  PHY_PREC_TC_TF32 = 1,
  PHY_PREC_TC_BF16 = 2, /* same with BF16 operands */
  PHY_PREC_TC_FP16 = 3  /* same with FP16 operands */
} phy_precision;

/* Element type of the llr outputs. PHY_LLR_F16 halves the largest output: each LLR is the FP32
   value rounded to nearest IEEE binary16, values beyond its range saturating to +-65504. The
   buffer is passed through the same float* parameters (cast); it holds 2-byte elements. */
typedef enum { PHY_LLR_F32 = 0, PHY_LLR_F16 = 1 } phy_llr_format;

typedef struct {
  int32_t n_cells;        /* independent cells (slots) in one call, >= 1 */
  int32_t n_prb;          /* physical resource blocks; n_sc = 12 n_prb, 1..275 */
  int32_t n_sym;          /* OFDM symbols in the slot, 1..14 */
  int32_t n_rx;           /* receive antennas, 1..64 */
  int32_t n_layers;       /* spatial layers, 1..16, <= n_rx */
  int32_t qm;             /* bits per QAM symbol: 2, 4, 6 or 8 */
  int32_t n_dmrs;         /* DMRS symbols, 1 or 2 */
  int32_t dmrs_sym[2];    /* their indices, increasing */
  int32_t occ_len;        /* Walsh cover length L (power of two, <= 16) or 0 for automatic */
  int32_t precision;      /* phy_precision */
  float pivot_ratio_min;  /* flag bit 0 threshold on min L_kk^2 / max L_kk^2, e.g. 1e-6 */
  int32_t fp64_refactor;  /* 1: re-compute flagged REs in FP64 (sets flag bit 1) */
  int32_t llr_format;     /* phy_llr_format of the llr outputs */
} phy_slot_cfg;

/* Human-readable name of a status code (static string). */
const char* phy_status_str(phy_status s);

/*
 * Failure-detection test hook (no counterpart in the paper). Every device wait in the detection
 * kernels polls a bounded number of times; a wait that runs out voids the CTA's work: the
 * tensor-core segment kernel bumps an error word that the solve kernel reads, and the solve
 * marks each affected RE with flag bit 3 alone. phy_debug_set_wait_polls() sets the poll limit
 * of the first-level waits of one kernel (PHY_WAIT_SEGMENT_KERNEL: the TMA ring, anchor, MMA
 * and drain hand-overs of the tensor-core segment kernel; PHY_WAIT_SOLVE_KERNEL: the solve
 * kernel's Gram-block copies) for every call made afterwards in this process; polls < 0
 * restores the default (about a second). With polls = 0 those waits give up at once, so a test
 * can make them run out without any fault: the waits that let copies and MMAs already in flight
 * land before a CTA ends keep their default limits. Returns PHY_ERR_INVALID_ARG for an unknown
 * kernel. Thread-safe; not for production use.
 */
typedef enum { PHY_WAIT_SEGMENT_KERNEL = 0, PHY_WAIT_SOLVE_KERNEL = 1 } phy_wait_kernel;

phy_status phy_debug_set_wait_polls(int32_t kernel, int64_t polls);

/*
 * FMA-throughput probe (measurement support, no counterpart in the paper): the measured peak
 * that the FP32 CUDA-core kernels' roofline fractions are reported against. Enqueues one kernel
 * of `blocks` CTAs x 256 threads on `stream`; every thread runs `iters` x 256 multiply-adds in
 * eight independent chains: FP32 (PHY_PROBE_FP32, one fma.rn.f32 each), FP32 pairs
 * (PHY_PROBE_FP32X2, one fma.rn.f32x2 per two) or FP64 (PHY_PROBE_FP64). CTA 0 writes its 256
 * thread sums to `sink` (device, 256 floats, or 256 doubles for FP64) so that no work is dead.
 * *flops_out (host, may be NULL) receives the flops the launch performs (2 per multiply-add);
 * divide by the launch's CUDA-event time. PHY_ERR_INVALID_ARG for an unknown kind, blocks < 1,
 * iters < 1 or a NULL sink. Size `blocks` as 8 per SM to fill every SM.
 */
typedef enum { PHY_PROBE_FP32 = 0, PHY_PROBE_FP32X2 = 1, PHY_PROBE_FP64 = 2 } phy_probe_kind;

phy_status phy_fma_probe(int32_t kind, int32_t blocks, int32_t iters, void* sink,
                         double* flops_out, void* stream);

/* Number of LS groups (anchors per DMRS symbol, layer and Rx) for cfg, or -1 if cfg is invalid. */
int32_t phy_n_groups(const phy_slot_cfg* cfg);

/* Number of data symbols for cfg (n_sym minus DMRS symbols), or -1 if cfg is invalid. */
int32_t phy_n_data_symbols(const phy_slot_cfg* cfg);

/* Workspace bytes phy_slot_run() needs for cfg; 0 if cfg is invalid. */
size_t phy_workspace_size(const phy_slot_cfg* cfg);

/*
 * DMRS least-squares estimation (the channel-estimation block of Sec. III-B): writes
 * anchors[cell][dmrs][group][layer][rx] from the DMRS symbols of Y and the pilots.
 */
phy_status phy_chest(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                     phy_c32* anchors, void* stream);

/*
 * LMMSE detection on a given full channel H[cell][dsym][sc][rx][layer] (Sec. IV): per data RE
 * x_hat = (H^H H + s2 I)^-1 H^H y, SINR and flags. sigma2 may be 0 (zero forcing); the SINR is
 * then clamped large. Used for genie-channel checks; the fused path is phy_slot_run().
 */
phy_status phy_mmse_detect(const phy_slot_cfg* cfg, const phy_c32* H, const phy_c32* Y,
                           const float* sigma2, phy_c32* x_hat, float* sinr, uint8_t* flags,
                           void* stream);

/*
 * Interpolation, LMMSE detection, SINR and LLRs from given LS anchors (as written by phy_chest,
 * or any estimate in that layout): the second half of phy_slot_run, with the same outputs,
 * rules and workspace (its first bytes, where phy_slot_run keeps the anchors, are unused).
 */
phy_status phy_detect_anchors(const phy_slot_cfg* cfg, const phy_c32* anchors, const phy_c32* Y,
                              const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                              uint8_t* flags, void* workspace, size_t workspace_bytes,
                              void* stream);

/*
 * The two stages of phy_detect_anchors, for callers that schedule or time them separately.
 * PHY_STAGE_GRAM_MF (the covariance products of Fig. 2(b)): per frequency segment the
 * time-folded Gram blocks of the interpolated channel and, per RE, the matched filter H^H y,
 * written into the workspace. PHY_STAGE_SOLVE (the LMMSE block of Sec. IV): per RE the Gram
 * matrix, Cholesky, solves, SINR and LLRs from those intermediates. The stages must run in that
 * order on the same workspace with no other call in between; both need the whole batch to fit
 * one chunk of the workspace (true when workspace_bytes >= phy_workspace_size(cfg) and
 * phy_stage_supported(cfg) is 1).
 */
typedef enum { PHY_STAGE_GRAM_MF = 0, PHY_STAGE_SOLVE = 1 } phy_stage;

/* 1 if phy_detect_stage() can run cfg's batch as one chunk with a phy_workspace_size()
   workspace. */
int32_t phy_stage_supported(const phy_slot_cfg* cfg);

phy_status phy_detect_stage(const phy_slot_cfg* cfg, int32_t stage, const phy_c32* anchors,
                            const phy_c32* Y, const float* sigma2, phy_c32* x_hat, float* sinr,
                            float* llr, uint8_t* flags, void* workspace, size_t workspace_bytes,
                            void* stream);

/*
 * Max-log LLR demapping of equalised symbols: from x_hat and SINR (as written by
 * phy_slot_run or phy_mmse_detect) computes llr[cell][dsym][sc][layer][qm].
 * REs whose SINR is not positive get zero LLRs.
 */
phy_status phy_llr_demap(const phy_slot_cfg* cfg, const phy_c32* x_hat, const float* sinr,
                         float* llr, void* stream);

/*
 * The whole receiver for one slot per cell: LS estimation, interpolation, LMMSE detection,
 * SINR and LLRs. Requires sigma2 > 0 for every cell. Any of x_hat, sinr, llr may be NULL to
 * skip writing that output; flags may not be NULL.
 */
phy_status phy_slot_run(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                        const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                        uint8_t* flags, void* workspace, size_t workspace_bytes, void* stream);

/*
 * phy_slot_run() with HOST inputs and outputs: copies Y_host, pilots_host and sigma2_host into
 * the caller's device staging buffers (Y, pilots, sigma2, same layouts), runs the receiver into
 * the device outputs, and copies llr and flags back into llr_host and flags_host, all on
 * `stream`. Host buffers should be page-locked for the copies to be asynchronous. x_hat and
 * sinr stay on the device (may be NULL).
 */
phy_status phy_slot_run_host(const phy_slot_cfg* cfg, const phy_c32* Y_host,
                             const phy_c32* pilots_host, const float* sigma2_host,
                             float* llr_host, uint8_t* flags_host, phy_c32* Y, phy_c32* pilots,
                             float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                             uint8_t* flags, void* workspace, size_t workspace_bytes,
                             void* stream);

/*
 * phy_slot_run() for callers that cannot allocate device memory. It has no counterpart in the
 * paper; it exists for hosts of this library that are not allowed to call cudaMalloc, for
 * example a real-time slot loop where an allocation could stall past the slot deadline (it may
 * synchronise the device), or a plugin whose host framework owns all device memory and hands
 * out only input and output buffers.
 *
 * The caller passes inputs and outputs only (same layouts and rules as phy_slot_run()). The
 * scratch space lives in one fixed array of PHY_NOALLOC_SCRATCH_BYTES in the library's device
 * memory: every GPU that loads libphy.so holds that array until the process exits, and the
 * call itself allocates nothing (no cudaMalloc, no cudaFree, no allocating library routine).
 *  - Limit: the array holds the LS anchors and noise-estimate partial sums of every cell plus
 *    the detection intermediates of at least one cell; the work then runs in chunks of as many
 *    cells as fit. A configuration for which even that minimum exceeds
 *    PHY_NOALLOC_SCRATCH_BYTES is rejected with PHY_ERR_NO_MEMORY before anything is enqueued.
 *    64 MiB takes 8 cells of 273 PRB with 64 Rx, 16 layers and two DMRS symbols (26.9 MB of
 *    anchors plus 16 MB per cell of intermediates, in chunks); 32 such cells (107 MB of
 *    anchors alone) are rejected.
 *  - The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 *    with that device current and caches it for the life of the process; make that first call
 *    before any stream capture. The cache does not survive cudaDeviceReset(): do not call this
 *    entry point after resetting a device it has already run on.
 *  - All calls on a device share the one array and it keeps the previous call's contents (every
 *    value a call reads is written earlier in the same call, so nothing needs clearing). Calls
 *    whose work overlaps on the GPU (different streams, or different host threads) race on it:
 *    serialise them, e.g. on one stream.
 */
#define PHY_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

phy_status phy_slot_run_noalloc(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                                const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                                uint8_t* flags, void* stream);

/*
 * Batched receiver for serving (no counterpart in the paper, which runs one cell per call): the
 * whole receiver of phy_slot_run() for up to 64 jobs of different shapes (PRB, antenna, layer,
 * modulation and DMRS counts, LLR format, FP64 re-computation) in one launch per stage and
 * layer class, so that a server can batch whatever jobs have arrived. A job is one
 * phy_slot_run() call's configuration and buffers (device pointers, same layouts and rules;
 * x_hat, sinr and llr may be NULL). On this path the Gram and matched-filter products run in
 * FP32 (cfg.precision PHY_PREC_FP32) or on the tensor cores with FP16 operands
 * (PHY_PREC_TC_FP16, two DMRS symbols, even n_rx); the cover length is the automatic one
 * (cfg.occ_len 0 or equal to it); other jobs get PHY_ERR_UNSUPPORTED. Each job's outputs are
 * bitwise those of phy_slot_run() on that job alone.
 *  - The job table lives in caller-owned, page-locked, device-mapped host memory of
 *    phy_batch_table_bytes() bytes (e.g. cudaHostAlloc), zeroed before first use, 128-byte
 *    aligned (the TMA tensor maps it holds need that); the device keeps a copy in a
 *    caller-owned device buffer of the same size, zeroed before first use, 128-byte aligned.
 *    One table pair per batch in flight.
 *  - phy_batch_workspace_size(): intermediates of a batch (the sum over its jobs); 0 if a job's
 *    cfg is invalid or n_jobs is outside 1..64.
 *  - phy_batch_post() (host only; for tensor-core jobs it encodes their TMA tensor maps, a
 *    driver call that touches no device): validates the jobs, lays out their intermediates in
 *    `workspace` (device, 256-byte aligned), writes the table into table_host and rings its
 *    doorbell last. Do not post into a table whose previous batch has not
 *    finished on the device. PHY_ERR_NO_MEMORY if the workspace is too small.
 *  - phy_batch_launch(): enqueues on `stream` a gate kernel that polls table_host's doorbell at
 *    most poll_limit times, about 1 us apart (poll_limit < 0: a million, about a second), copies
 *    a newly posted table into table_dev and then the stage kernels (LS estimation; the noise
 *    estimate of the jobs that track it; per layer class, on forked streams joined back into
 *    `stream`, the Gram/matched-filter and solve kernels, persistent over the table's items). Its
 *    arguments do not change between batches, so it may be captured once in a CUDA graph and
 *    replayed per batch; a launch may also be enqueued before the batch is posted (the gate
 *    waits for it). If no new table arrives within the limit, the stages run on an empty table
 *    and the gate records a timeout. PHY_ERR_INVALID_ARG if table_host is not mapped.
 *  - phy_batch_status(): after the launch has completed on the device, PHY_OK if it ran the last
 *    posted table, PHY_ERR_TIMEOUT if its gate timed out, PHY_ERR_INVALID_ARG if neither (not
 *    finished, or nothing launched since the post).
 */
typedef struct {
  phy_slot_cfg cfg;
  const phy_c32* Y;
  const phy_c32* pilots;
  const float* sigma2;
  phy_c32* x_hat;
  float* sinr;
  float* llr;
  uint8_t* flags;
  /* Noise level tracked on the device across slots (optional): with noise_state non-NULL the
   * job ignores sigma2 and runs as phy_slot_run_track() with (noise_mode, noise_alpha) on that
   * state (n_cells floats, device, kept by the caller between slots): the batch estimates each
   * cell's noise variance from this slot's DMRS, blends it into the state and detects with the
   * updated state. Tracking jobs of one batch must not share state (PHY_ERR_INVALID_ARG). */
  float* noise_state;
  float noise_alpha;   /* 0 < alpha <= 1 when noise_state is set */
  int32_t noise_mode;  /* phy_noise_mode */
} phy_job;

size_t phy_batch_table_bytes(void);
size_t phy_batch_workspace_size(const phy_job* jobs, int32_t n_jobs);
phy_status phy_batch_post(const phy_job* jobs, int32_t n_jobs, void* table_host, void* workspace,
                          size_t workspace_bytes);
phy_status phy_batch_launch(void* table_host, void* table_dev, int64_t poll_limit, void* stream);
phy_status phy_batch_status(const void* table_host);

/*
 * Tile autotuner (no counterpart in the paper). Detection runs in chunks
 * of cells: the Gram/matched-filter kernel writes one chunk's intermediates (about 16 MB per
 * 273-PRB cell at 64x16) and the solve kernel reads them back, so the chunk size trades L2
 * residency of those intermediates against launch count and tail effects. phy_autotune() runs
 * phy_slot_run() on the caller's buffers for every chunk size that fits `workspace_bytes`
 * (1, 2, 4, ... cells and the whole batch): one warm-up and three timed runs each (CUDA events
 * on `stream`), and keeps the fastest in a process-wide table keyed by every field of cfg that
 * shapes the work. Later phy_slot_run(), phy_detect_anchors() and phy_slot_run_host() calls
 * with an equal cfg use that chunk (still shrunk to fit their workspace); phy_detect_stage()
 * always runs the whole batch as one chunk.
 *  - Synchronises `stream` (a tuning call, not for the hot path); same arguments and rules as
 *    phy_slot_run(); afterwards the outputs hold a normal phy_slot_run() result.
 *  - *chunk_out (may be NULL) receives the chosen cells per chunk.
 * phy_autotune_clear() forgets every tuned configuration. Both are thread-safe.
 */
phy_status phy_autotune(const phy_slot_cfg* cfg, const phy_c32* Y, const phy_c32* pilots,
                        const float* sigma2, phy_c32* x_hat, float* sinr, float* llr,
                        uint8_t* flags, void* workspace, size_t workspace_bytes, void* stream,
                        int32_t* chunk_out);
void phy_autotune_clear(void);

/*
 * The tile shapes behind a configuration's calls, as phy_autotune() chose them or as set here;
 * 0 means the library default (and chunk 0: the preferred chunk for the workspace).
 *  - chunk: cells per detection chunk (1..n_cells);
 *  - solve_width: REs (threads) per CTA of the solve kernel, 128 (default) or 64;
 *  - ring_stages: depth of the tensor-core segment kernel's ring of 16-subcarrier boxes, the
 *    format's default (8 stages for FP16/BF16, 6 for TF32) or 12 where its shared-memory map
 *    still fits (otherwise the default is used, and phy_autotune_tiles() reads back 0).
 * phy_autotune() searches them in that order (chunk sizes, then the other solve width, then the
 * deeper ring for FP16/BF16 products where it fits), keeping each change only if it is faster. Tiles never
 * change the arithmetic: every choice gives bitwise the same outputs.
 * phy_autotune_set_tiles() pins them for cfg's key (PHY_ERR_INVALID_ARG for a value outside the
 * lists); phy_autotune_tiles() reads them back. Both are thread-safe and host-only.
 */
phy_status phy_autotune_set_tiles(const phy_slot_cfg* cfg, int32_t chunk, int32_t solve_width,
                                  int32_t ring_stages);
phy_status phy_autotune_tiles(const phy_slot_cfg* cfg, int32_t* chunk, int32_t* solve_width,
                              int32_t* ring_stages);

/*
 * Noise-variance estimate from the DMRS (the paper treats the noise level as a known input of the
 * LMMSE block, Sec. IV; no method is given, so the rule below is this library's). A noise sample
 * is the residual of an LS anchor against its prediction from other anchors of the same layer:
 *  - PHY_NOISE_FREQ: every interior anchor (groups 1 .. G-2) against the linear interpolation of
 *    its two neighbours at its own subcarrier, e = H(g) - a H(g-1) - b H(g+1), on each DMRS symbol;
 *  - PHY_NOISE_TIME: every anchor against the same anchor of the other DMRS symbol (needs two);
 *  - PHY_NOISE_MIN: both, keeping the smaller estimate (channel variation across the groups, or
 *    between the DMRS symbols, can only raise either one).
 * Each residual is a fixed linear combination of DMRS REs whose noise gain gamma (the squared norm
 * of its coefficients, from the pilots) is known, so
 *   sigma2_out[cell] = sum |e|^2 / (n_rx sum gamma)
 * is unbiased when the channel is constant over the three groups (frequency) or between the two
 * DMRS symbols (time), and too large otherwise. NaN where the mode has no residual (fewer than
 * three groups for the frequency rule and, with PHY_NOISE_MIN, no second DMRS symbol either).
 *  - anchors: as written by phy_chest (or any estimate in that layout); pilots as for phy_chest.
 *  - sigma2_out: n_cells floats (device). The sums run in a fixed order (deterministic).
 *  - workspace: at least phy_workspace_size(cfg) bytes; the call uses the bytes after the first
 *    n_cells n_dmrs G n_layers n_rx phy_c32 (where phy_slot_run keeps the anchors), rounded up to
 *    256, so anchors stored at the start of the same workspace stay intact.
 *  - PHY_ERR_INVALID_ARG for an unknown mode or PHY_NOISE_TIME with one DMRS symbol.
 */
typedef enum { PHY_NOISE_FREQ = 0, PHY_NOISE_TIME = 1, PHY_NOISE_MIN = 2 } phy_noise_mode;

phy_status phy_noise_est(const phy_slot_cfg* cfg, int32_t mode, const phy_c32* anchors,
                         const phy_c32* pilots, float* sigma2_out, void* workspace,
                         size_t workspace_bytes, void* stream);

/*
 * Noise-variance state kept on the device across slots: phy_noise_track() estimates as
 * phy_noise_est() and blends the estimate into sigma2_state[cell] (device, n_cells floats, kept
 * by the caller from slot to slot): state = alpha estimate + (1 - alpha) state, 0 < alpha <= 1.
 * A state that is not a positive finite number (e.g. zeroed before the first slot) takes the
 * estimate as it is; an estimate that is not finite leaves a valid state unchanged.
 * phy_slot_run_track() runs LS estimation, phy_noise_track() and detection with the updated state,
 * all on `stream`, like phy_slot_run_est() with a smoothed noise level.
 */
phy_status phy_noise_track(const phy_slot_cfg* cfg, int32_t mode, float alpha,
                           const phy_c32* anchors, const phy_c32* pilots, float* sigma2_state,
                           void* workspace, size_t workspace_bytes, void* stream);
phy_status phy_slot_run_track(const phy_slot_cfg* cfg, int32_t mode, float alpha,
                              const phy_c32* Y, const phy_c32* pilots, float* sigma2_state,
                              phy_c32* x_hat, float* sinr, float* llr, uint8_t* flags,
                              void* workspace, size_t workspace_bytes, void* stream);

/*
 * phy_slot_run() with the noise variance estimated on the way: LS estimation, phy_noise_est()
 * with `mode` into sigma2_out (n_cells floats, device), then interpolation, detection, SINR and
 * LLRs with that estimate, all on `stream`. Same outputs, rules and workspace as phy_slot_run();
 * the result equals phy_slot_run() called with sigma2 = the estimate.
 */
phy_status phy_slot_run_est(const phy_slot_cfg* cfg, int32_t mode, const phy_c32* Y,
                            const phy_c32* pilots, float* sigma2_out, phy_c32* x_hat,
                            float* sinr, float* llr, uint8_t* flags, void* workspace,
                            size_t workspace_bytes, void* stream);

/*
 * Block-floating-point (BFP) fronthaul input: the received grid as a split-7 fronthaul delivers it
 * to a software DU (the setting of the paper, which prints no format; this is the library's
 * reading of the usual shared-exponent block format). The stream Yc holds one block per (cell,
 * symbol, antenna, PRB), in that order, of 1 + 3 iq_width bytes:
 *  - a parameter byte whose low four bits are the exponent e (the high four bits are ignored);
 *  - the PRB's 24 values I0 Q0 I1 Q1 ... I11 Q11, each an iq_width-bit two's-complement
 *    mantissa m (1 <= iq_width <= 16), packed most significant bit first across the bytes.
 * The decoded value is m 2^e scale, rounded once to FP32 (m 2^e is exact). Yc must be 4-byte
 * aligned; scale finite and positive.
 *
 * phy_bfp_bytes: the stream's size in bytes for cfg (0 for an invalid cfg or width).
 * phy_bfp_decompress: decodes the stream into the grid Y [cell][sym][rx][sc] (16-byte aligned).
 *   With data_only != 0 the DMRS symbols' rows of Y are not written (phy_chest_bfp reads them
 *   from the stream itself).
 * phy_chest_bfp: phy_chest() reading the DMRS symbols straight from the stream; its anchors are
 *   bitwise those of phy_chest() on the decoded grid.
 * phy_slot_run_bfp: phy_slot_run() from the stream: decodes it into the caller's grid buffer Y
 *   (device, n_cells n_sym n_rx n_sc phy_c32) and runs the receiver on it; outputs bitwise those
 *   of phy_slot_run() on the decoded grid. Same workspace and rules as phy_slot_run().
 */
size_t phy_bfp_bytes(const phy_slot_cfg* cfg, int32_t iq_width);

phy_status phy_bfp_decompress(const phy_slot_cfg* cfg, const uint8_t* Yc, int32_t iq_width,
                              float scale, int32_t data_only, phy_c32* Y, void* stream);

phy_status phy_chest_bfp(const phy_slot_cfg* cfg, const uint8_t* Yc, int32_t iq_width,
                         float scale, const phy_c32* pilots, phy_c32* anchors, void* stream);

phy_status phy_slot_run_bfp(const phy_slot_cfg* cfg, const uint8_t* Yc, int32_t iq_width,
                            float scale, phy_c32* Y, const phy_c32* pilots, const float* sigma2,
                            phy_c32* x_hat, float* sinr, float* llr, uint8_t* flags,
                            void* workspace, size_t workspace_bytes, void* stream);

/*
 * phy_slot_run_bfp() with HOST inputs and outputs, as phy_slot_run_host() is to phy_slot_run():
 * copies the stream Yc_host (phy_bfp_bytes() bytes), pilots_host and sigma2_host into the device
 * buffers Yc (4-byte aligned), pilots and sigma2, runs phy_slot_run_bfp() (decoding into the
 * device grid buffer Y), and copies llr and flags back into llr_host and flags_host, all on
 * `stream`. Host buffers should be page-locked for the copies to be asynchronous.
 */
phy_status phy_slot_run_bfp_host(const phy_slot_cfg* cfg, const uint8_t* Yc_host,
                                 int32_t iq_width, float scale, const phy_c32* pilots_host,
                                 const float* sigma2_host, float* llr_host, uint8_t* flags_host,
                                 uint8_t* Yc, phy_c32* Y, phy_c32* pilots, float* sigma2,
                                 phy_c32* x_hat, float* sinr, float* llr, uint8_t* flags,
                                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * Learned channel denoiser (the paper has no learned part; this is a refinement between channel
 * estimation and detection). A residual CNN maps a 12-subcarrier x 14-symbol tile of the
 * interpolated LS estimate of one (PRB, Rx antenna, layer) channel entry to a refined tile:
 * 3x3 cross-correlations with zero padding, channels 2 -> 32 -> 32 -> 32 -> 2 (real, imaginary),
 * ReLU after the first three, the input added to the output. Everything runs in FP32.
 *  - Parameters: one flat float vector of phy_cnn_param_count() = 19682 values, in the order
 *    W1 [32][2][3][3], b1 [32], W2 [32][32][3][3], b2 [32], W3 [32][32][3][3], b3 [32],
 *    W4 [2][32][3][3], b4 [2].
 *  - Tiles: float [n][2][14][12] (channel, symbol, subcarrier within the PRB).
 *  - phy_cnn_forward: out = network(in) for n tiles; workspace of phy_cnn_workspace_size(n).
 *  - phy_cnn_train_step: forward pass, loss = mean over tiles and positions of |out - label|^2
 *    (written to *loss, device, if loss is not NULL), its gradient w.r.t. the parameters into
 *    grad (phy_cnn_param_count() floats) and, if grad_in is not NULL, w.r.t. the input tiles;
 *    then, if step >= 1, one Adam update of params (beta1 0.9, beta2 0.999, eps 1e-8, bias
 *    correction for update number `step`) with moments adam_m, adam_v (zero before the first).
 *    Gradients are summed in a fixed order: repeated calls give identical results.
 *  - phy_cnn_n_tiles: tiles of a slot batch (n_cells n_prb n_rx n_layers; -1 unless n_sym == 14).
 *  - phy_interp_channel: the interpolated LS channel at every symbol (DMRS symbols included),
 *    H [cell][sym][sc][rx][layer], from anchors as written by phy_chest.
 *  - phy_cnn_tiles: such an H (estimated or true) cut into tiles, tile index
 *    ((cell n_prb + prb) n_rx + rx) n_layers + layer. phy_cnn_untile: the data symbols of tiles
 *    back into H_data [cell][dsym][sc][rx][layer], the layout phy_mmse_detect() takes.
 *  - phy_cnn_denoise: phy_interp_channel, phy_cnn_tiles, phy_cnn_forward and phy_cnn_untile in
 *    one call, with a workspace of phy_cnn_denoise_workspace_size(cfg).
 */
int32_t phy_cnn_param_count(void);
size_t phy_cnn_workspace_size(int32_t n_tiles);
phy_status phy_cnn_forward(int32_t n_tiles, const float* params, const float* tiles_in,
                           float* tiles_out, void* workspace, size_t workspace_bytes,
                           void* stream);
phy_status phy_cnn_train_step(int32_t n_tiles, float* params, float* adam_m, float* adam_v,
                              int32_t step, float lr, const float* tiles_in,
                              const float* tiles_label, float* grad, float* grad_in,
                              float* loss, void* workspace, size_t workspace_bytes,
                              void* stream);
int32_t phy_cnn_n_tiles(const phy_slot_cfg* cfg);
phy_status phy_interp_channel(const phy_slot_cfg* cfg, const phy_c32* anchors, phy_c32* H,
                              void* stream);
phy_status phy_cnn_tiles(const phy_slot_cfg* cfg, const phy_c32* H, float* tiles, void* stream);
phy_status phy_cnn_untile(const phy_slot_cfg* cfg, const float* tiles, phy_c32* H_data,
                          void* stream);
size_t phy_cnn_denoise_workspace_size(const phy_slot_cfg* cfg);
/*
 * The same network on the tcgen05 tensor cores with BF16 operands and FP32 accumulation: the
 * weights and every layer's input rounded to nearest BF16, biases, sums and the residual in FP32
 * (the bfloat16 form of the network). phy_cnn_forward_bf16 takes a workspace of at least 4 bytes
 * (4-byte aligned) whose first word it clears and then counts CTAs whose bounded wait for the
 * tensor core ran out (nonzero: the outputs are not valid). phy_cnn_denoise_bf16 is
 * phy_cnn_denoise with this forward pass (same workspace); its error word sits at byte
 * phy_cnn_denoise_error_offset(cfg) of the workspace.
 */
phy_status phy_cnn_forward_bf16(int32_t n_tiles, const float* params, const float* tiles_in,
                                float* tiles_out, void* workspace, size_t workspace_bytes,
                                void* stream);
phy_status phy_cnn_denoise_bf16(const phy_slot_cfg* cfg, const float* params,
                                const phy_c32* anchors, phy_c32* H_data, void* workspace,
                                size_t workspace_bytes, void* stream);
size_t phy_cnn_denoise_error_offset(const phy_slot_cfg* cfg);
/*
 * Mixed-precision training step: phy_cnn_train_step with its forward pass on the tensor cores
 * (the BF16 form above), which also keeps the activations the next layers read (BF16 values) for
 * the backward pass; the loss, the gradients and the Adam update of the FP32 master parameters
 * stay FP32 on the CUDA cores. The gradients are those of the BF16 network (weights and layer
 * inputs rounded in the forward pass, the backward pass through them in FP32). Same arguments
 * and workspace as phy_cnn_train_step; the forward pass's error word (nonzero: a bounded wait
 * for the tensor core ran out and the step's results are not valid) sits at byte
 * phy_cnn_train_error_offset(n_tiles) of the workspace.
 */
phy_status phy_cnn_train_step_bf16(int32_t n_tiles, float* params, float* adam_m, float* adam_v,
                                   int32_t step, float lr, const float* tiles_in,
                                   const float* tiles_label, float* grad, float* grad_in,
                                   float* loss, void* workspace, size_t workspace_bytes,
                                   void* stream);
size_t phy_cnn_train_error_offset(int32_t n_tiles);
phy_status phy_cnn_denoise(const phy_slot_cfg* cfg, const float* params, const phy_c32* anchors,
                           phy_c32* H_data, void* workspace, size_t workspace_bytes,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PHY_H */
