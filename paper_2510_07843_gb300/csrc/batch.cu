// Batched receiver for serving: every job of a batch (any mix of PRB, antenna, layer and
// modulation counts) in one launch per stage and layer class, behind a host doorbell.
//
// phy_batch_post() lays out each job's intermediates in the caller's workspace, writes the job
// table into caller-owned pinned host memory and rings the doorbell (bumps the table's seq).
// phy_batch_launch() enqueues the gate kernel and the persistent stage kernels; its arguments
// never change between batches, so a CUDA graph captured on it serves every batch. The gate
// polls the doorbell a bounded number of times: a posted table is copied into device memory for
// the stage kernels; a doorbell that never rings leaves the stages an empty table and reports a
// timeout in the host copy, which phy_batch_status() returns as PHY_ERR_TIMEOUT.
#include <algorithm>
#include <cstring>

#include "../../include/phy.h"
#include "batch.cuh"
#include "launch.h"

namespace phy {

size_t batch_anchor_bytes(const Geo& g) {
  return (size_t)g.n_cells * g.n_dmrs * g.G * g.n_layers * g.n_rx * sizeof(phy_c32);
}

namespace {

constexpr size_t kAlign = 256;
size_t up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

size_t job_workspace(const Geo& g) {
  return up(batch_anchor_bytes(g)) + up(batch_ygg_bytes(g)) + up(batch_bvec_bytes(g)) +
         up((size_t)g.n_cells * noise_blocks(g) * sizeof(float4)) + kAlign;
}

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr int kGateThreads = 1024;

// One CTA: waits for the doorbell (at most poll_limit polls of ~1 us), then copies the table.
__global__ void __launch_bounds__(kGateThreads)
    batch_gate_kernel(BatchTable* host_t, BatchTable* dev_t, unsigned poll_limit) {
  __shared__ uint32_t s_seq;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const uint32_t last = dev_t->done_seq;
    uint32_t seq = last;
    int ok = 0;
    for (unsigned i = 0;; ++i) {
      seq = ld_acquire_sys(&host_t->seq);
      if (seq != last) {
        ok = 1;
        break;
      }
      if (i >= poll_limit) break;
      __nanosleep(1000);
    }
    s_seq = seq;
    s_ok = ok;
  }
  __syncthreads();
  if (s_ok) {
    static_assert(sizeof(BatchTable) % 8 == 0, "the table is copied in 8-byte words");
    const volatile unsigned long long* src =
        reinterpret_cast<const volatile unsigned long long*>(host_t);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(dev_t);
    for (int i = threadIdx.x; i < (int)(sizeof(BatchTable) / 8); i += blockDim.x) dst[i] = src[i];
  } else {
    int* n = &dev_t->n_items[0][0];  // nothing for the stage kernels to do
    for (int i = threadIdx.x; i < kBatchStages * kBatchClasses; i += blockDim.x) n[i] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_ok) dev_t->done_seq = s_seq;
    volatile BatchTable* h = host_t;
    h->done_seq = s_ok ? s_seq : dev_t->done_seq;
    h->status = s_ok ? kBatchOk : kBatchTimedOut;
  }
}

}  // namespace
}  // namespace phy

using phy::BatchJob;
using phy::BatchTable;

extern "C" size_t phy_batch_table_bytes(void) { return sizeof(BatchTable); }

extern "C" size_t phy_batch_workspace_size(const phy_job* jobs, int32_t n_jobs) {
  if (!jobs || n_jobs < 1 || n_jobs > phy::kBatchMaxJobs) return 0;
  size_t total = 0;
  for (int i = 0; i < n_jobs; ++i) {
    phy::Geo g;
    if (phy::make_geo_checked(&jobs[i].cfg, &g) != PHY_OK) return 0;
    total += phy::job_workspace(g);
  }
  return total;
}

extern "C" phy_status phy_batch_post(const phy_job* jobs, int32_t n_jobs, void* table_host,
                                     void* workspace, size_t workspace_bytes) {
  if (!jobs || !table_host || n_jobs < 1 || n_jobs > phy::kBatchMaxJobs)
    return PHY_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(table_host) % alignof(BatchTable) ||
      reinterpret_cast<uintptr_t>(workspace) % 256)
    return PHY_ERR_INVALID_ARG;
  BatchTable* t = static_cast<BatchTable*>(table_host);
  // everything but the doorbell words is rebuilt
  const uint32_t seq = t->seq;
  std::memset(reinterpret_cast<char*>(t) + offsetof(BatchTable, n_jobs), 0,
              sizeof(BatchTable) - offsetof(BatchTable, n_jobs));
  char* ws = static_cast<char*>(workspace);
  size_t used = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const phy_job& jb = jobs[i];
    phy::Geo g;
    const phy_status s = phy::make_geo_checked(&jb.cfg, &g);
    if (s != PHY_OK) return s;
    // the batched path: FP32 or FP16 tensor-core products, automatic cover length, shapes
    // within the captured launches' shared memory; tensor-core jobs need two DMRS symbols and
    // the tensor-core kernel's shape rules
    int auto_l = 1;
    while (auto_l < (g.n_layers + 1) / 2) auto_l *= 2;
    const int nlc = phy::nl_class_of(g.n_layers), cls = phy::batch_class(nlc);
    const bool tc = g.prec == PHY_PREC_TC_FP16;
    const bool direct = !tc && phy::batch_direct_class(nlc) != 0;
    if ((g.prec != PHY_PREC_FP32 && !tc) || g.L != auto_l) return PHY_ERR_UNSUPPORTED;
    if (tc && (g.n_dmrs != 2 || !phy::seg_prep_tc_supported(g) || !phy::batch_solve_fits(g)))
      return PHY_ERR_UNSUPPORTED;
    if (!tc && !direct && !phy::batch_geometry_fits(g)) return PHY_ERR_UNSUPPORTED;
    const bool track = jb.noise_state != nullptr;
    if (!jb.Y || !jb.pilots || (!jb.sigma2 && !track) || !jb.flags) return PHY_ERR_INVALID_ARG;
    if (track) {
      if (!(jb.noise_alpha > 0.f && jb.noise_alpha <= 1.f) || jb.noise_mode < PHY_NOISE_FREQ ||
          jb.noise_mode > PHY_NOISE_MIN || (jb.noise_mode == PHY_NOISE_TIME && g.n_dmrs != 2))
        return PHY_ERR_INVALID_ARG;
      // tracking jobs of one batch update their states concurrently: no shared cells
      const uintptr_t a0 = reinterpret_cast<uintptr_t>(jb.noise_state);
      const uintptr_t a1 = a0 + (uintptr_t)g.n_cells * sizeof(float);
      for (int k = 0; k < i; ++k) {
        if (!jobs[k].noise_state) continue;
        const uintptr_t b0 = reinterpret_cast<uintptr_t>(jobs[k].noise_state);
        const uintptr_t b1 = b0 + (uintptr_t)t->job[k].g.n_cells * sizeof(float);
        if (a0 < b1 && b0 < a1) return PHY_ERR_INVALID_ARG;
      }
    }
    if (reinterpret_cast<uintptr_t>(jb.Y) % 16) return PHY_ERR_INVALID_ARG;
    const size_t need = phy::job_workspace(g);
    if (!workspace || used + need > workspace_bytes) return PHY_ERR_NO_MEMORY;
    BatchJob& J = t->job[i];
    J.g = g;
    J.Y = jb.Y;
    J.pilots = jb.pilots;
    J.sigma2 = track ? jb.noise_state : jb.sigma2;  // detection reads the updated state
    J.noise_alpha = track ? jb.noise_alpha : 0.f;
    J.noise_mode = jb.noise_mode;
    J.noise_blocks = phy::noise_blocks(g);
    J.x_hat = jb.x_hat;
    J.sinr = jb.sinr;
    J.llr = jb.llr;
    J.flags = jb.flags;
    char* p = ws + used;
    J.anchors = reinterpret_cast<phy_c32*>(p);
    p += phy::up(phy::batch_anchor_bytes(g));
    J.ygg = reinterpret_cast<float4*>(p);
    p += phy::up(phy::batch_ygg_bytes(g));
    J.bvec = reinterpret_cast<phy::cf*>(p);
    p += phy::up(phy::batch_bvec_bytes(g));
    J.noise_part = reinterpret_cast<float4*>(p);
    p += phy::up((size_t)g.n_cells * J.noise_blocks * sizeof(float4));
    J.err = reinterpret_cast<unsigned*>(p);
    used += need;
    J.wmax = phy::batch_wmax(g);
    J.max_segs = phy::batch_max_segs(g);
    if (tc && !phy::encode_tc_maps(g, J.anchors, jb.Y, &J.tmY, &J.tmA))
      return PHY_ERR_INVALID_ARG;
    // items per stage: LS (chunk of groups, DMRS symbol, cell) over all jobs; per layer class the segment
    // stage (FP32 or tensor-core: segment, cell) and the solve or, for the direct form, that
    // form (128 subcarriers, data symbol, cell)
    const int res = ((g.n_sc + 127) / 128) * g.n_dsym * g.n_cells;
    const int seg_items = g.n_seg * g.n_cells;
    const int gp = phy::chest_batch_groups(g.n_rx);
    if (gp * g.n_layers * 2 * g.L > phy::kChestBatchPilots) return PHY_ERR_UNSUPPORTED;
    const int items[phy::kBatchStages] = {(g.G + gp - 1) / gp * g.n_dmrs * g.n_cells,
                                          !tc && !direct ? seg_items : 0, tc ? seg_items : 0,
                                          direct ? 0 : res, direct ? res : 0,
                                          track ? J.noise_blocks * g.n_cells : 0,
                                          track ? g.n_cells : 0};
    for (int stg = 0; stg < phy::kBatchStages; ++stg) {
      if (stg != phy::kBatchChest && items[stg] == 0) continue;
      const bool per_job = stg == phy::kBatchChest || stg == phy::kBatchNoisePart ||
                           stg == phy::kBatchNoiseFinal;  // one class for every job
      const int c = per_job ? 0 : cls;
      int& nj = t->n_class_jobs[stg][c];
      t->job_of[stg][c][nj] = (unsigned char)i;
      t->start[stg][c][nj] = t->n_items[stg][c];
      t->n_items[stg][c] += items[stg];
      ++nj;
      t->start[stg][c][nj] = t->n_items[stg][c];
    }
  }
  t->n_jobs = (uint32_t)n_jobs;
  t->status = phy::kBatchPending;
  // the doorbell last: the gate reads the rest only after it sees the new seq
  __atomic_store_n(&t->seq, seq + 1, __ATOMIC_RELEASE);
  return PHY_OK;
}

extern "C" phy_status phy_batch_launch(void* table_host, void* table_dev, int64_t poll_limit,
                                       void* stream) {
  if (!table_host || !table_dev || reinterpret_cast<uintptr_t>(table_dev) % alignof(BatchTable) ||
      reinterpret_cast<uintptr_t>(table_host) % alignof(BatchTable))
    return PHY_ERR_INVALID_ARG;
  void* mapped = nullptr;
  if (cudaHostGetDevicePointer(&mapped, table_host, 0) != cudaSuccess || !mapped) {
    cudaGetLastError();  // not page-locked and mapped: not an error of later calls
    return PHY_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned limit =
      poll_limit < 0 ? 1000000u : (unsigned)std::min<int64_t>(poll_limit, 0x7FFFFFFF);
  phy::batch_gate_kernel<<<1, phy::kGateThreads, 0, st>>>(static_cast<BatchTable*>(mapped),
                                                          static_cast<BatchTable*>(table_dev),
                                                          limit);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return PHY_ERR_CUDA;
  const BatchTable* t = static_cast<const BatchTable*>(table_dev);
  if ((e = phy::launch_chest_batch(t, st)) != cudaSuccess ||
      (e = phy::launch_noise_batch(t, st)) != cudaSuccess)
    return PHY_ERR_CUDA;
  if ((e = phy::launch_batch_stages(t, st)) != cudaSuccess) return PHY_ERR_CUDA;
  return PHY_OK;
}

extern "C" phy_status phy_batch_status(const void* table_host) {
  if (!table_host) return PHY_ERR_INVALID_ARG;
  const volatile BatchTable* t = static_cast<const volatile BatchTable*>(table_host);
  if (t->status == phy::kBatchTimedOut) return PHY_ERR_TIMEOUT;
  if (t->status == phy::kBatchOk && t->done_seq == t->seq) return PHY_OK;
  return PHY_ERR_INVALID_ARG;
}
