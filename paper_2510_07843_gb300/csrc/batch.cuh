// Job table of the batched receiver (internal to libphy.so): one launch per stage and layer class
// serves every job of a batch, whatever its PRB, antenna, layer and modulation counts.
//
// The host writes the table into caller-owned pinned memory that the device can read, then
// publishes it by bumping `seq` (the doorbell). A one-CTA gate kernel waits for that bump (a
// bounded poll), copies the table into device memory and the stage kernels read the copy. Each
// stage kernel is persistent: its CTAs stride over the stage's work items of one layer class,
// find the item's job by its prefix offset, and run the same per-item body as the single-job
// kernels, on that job's geometry and buffers.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace phy {

constexpr int kBatchMaxJobs = 64;
constexpr int kBatchClasses = 4;  // layer classes 2, 4, 8, 16 (the kernels' NL)
// Stages: LS estimation (every job, class 0), FP32 segment kernel, tensor-core segment kernel
// (FP16 products), per-RE solve (after either segment kernel), direct form (FP32, <= 4 layers),
// and for jobs that track their noise level on the device the estimate's partial sums and its
// per-cell reduction into the state (class 0, between LS estimation and detection).
enum BatchStage : int {
  kBatchChest = 0,
  kBatchSeg = 1,
  kBatchSegTc = 2,
  kBatchSolve = 3,
  kBatchDirect = 4,
  kBatchNoisePart = 5,
  kBatchNoiseFinal = 6,
  kBatchStages = 7
};

__host__ __device__ constexpr int batch_class(int nl_class) {
  return nl_class <= 2 ? 0 : nl_class <= 4 ? 1 : nl_class <= 8 ? 2 : 3;
}

// LS items of the batched path: a CTA of kChestBatchThreads threads takes chest_batch_groups
// consecutive anchor groups of one (DMRS symbol, cell), one thread per (group, antenna) with the
// antennas padded to a power of two, so that jobs with few antennas still fill the CTA.
constexpr int kChestBatchThreads = 128;
constexpr int kChestBatchPilots = 2048;  // staged pilots: groups x layers x 2L (bounded below)
__host__ __device__ constexpr int chest_batch_groups(int n_rx) {
  return n_rx <= 1 ? 128 : n_rx <= 2 ? 64 : n_rx <= 4 ? 32 : n_rx <= 8 ? 16 : n_rx <= 16 ? 8
       : n_rx <= 32 ? 4 : 2;
}

struct BatchJob {
  // tensor maps of the job's grid and anchors (jobs with tensor-core products; encoded by the
  // host into the table, read by TMA from the device copy)
  CUtensorMap tmY, tmA;
  Geo g;
  const phy_c32* Y;
  const phy_c32* pilots;
  const float* sigma2;
  phy_c32* x_hat;
  float* sinr;
  float* llr;
  uint8_t* flags;
  phy_c32* anchors;   // intermediates in the batch workspace
  float4* ygg;
  cf* bvec;
  unsigned* err;
  float4* noise_part;  // the noise estimate's partial sums (jobs that track their noise level)
  float noise_alpha;   // > 0: sigma2 is the job's per-cell state, updated before detection
  int noise_mode, noise_blocks;
  int wmax, max_segs;
};

// Status words the gate writes back into the host copy.
enum : uint32_t { kBatchPending = 0, kBatchOk = 1, kBatchTimedOut = 2 };

struct BatchTable {
  // doorbell and results (host copy: written by the host, then by the gate)
  uint32_t seq;          // bumped by the host once the rest of the table is written
  uint32_t done_seq;     // the seq the gate last consumed
  uint32_t status;       // kBatch* for done_seq
  uint32_t n_jobs;
  // items per stage and class (the chest stage uses class 0 for every job), and per class the
  // jobs in order with the prefix offset of their items
  int n_items[kBatchStages][kBatchClasses];
  int n_class_jobs[kBatchStages][kBatchClasses];
  int start[kBatchStages][kBatchClasses][kBatchMaxJobs + 1];
  unsigned char job_of[kBatchStages][kBatchClasses][kBatchMaxJobs];
  BatchJob job[kBatchMaxJobs];
};

// Finds the job of item w among the class's jobs; returns the job index and w's offset in it.
__device__ __forceinline__ int batch_find(const BatchTable* __restrict__ t, int stage, int cls,
                                          int w, int& local) {
  const int* st = t->start[stage][cls];
  int lo = 0, hi = t->n_class_jobs[stage][cls] - 1;
  while (lo < hi) {  // last i with st[i] <= w
    const int mid = (lo + hi + 1) >> 1;
    if (st[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  local = w - st[lo];
  return t->job_of[stage][cls][lo];
}

// A CTA's shared-memory copy of one (stage, class) prefix table, so that finding an item's job
// is a search in shared memory instead of a chain of dependent global loads per item.
struct BatchIndex {
  int n;                           // jobs of the class
  int start[kBatchMaxJobs + 1];    // prefix offsets of their items
  unsigned char job[kBatchMaxJobs];
};

// Every thread of the block calls it; a barrier must follow before the copy is read.
__device__ __forceinline__ void batch_index_load(BatchIndex& s, const BatchTable* __restrict__ t,
                                                 int stage, int cls) {
  const int n = t->n_class_jobs[stage][cls];
  if (threadIdx.x == 0) s.n = n;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) s.start[i] = t->start[stage][cls][i];
  for (int i = threadIdx.x; i < n; i += blockDim.x) s.job[i] = t->job_of[stage][cls][i];
}

__device__ __forceinline__ int batch_find(const BatchIndex& s, int w, int& local) {
  int lo = 0, hi = s.n - 1;
  while (lo < hi) {  // last i with start[i] <= w
    const int mid = (lo + hi + 1) >> 1;
    if (s.start[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  local = w - s.start[lo];
  return s.job[lo];
}

// Cooperative copy of a job's geometry into shared memory (every thread of the block calls it;
// a barrier must follow before the copy is read).
__device__ __forceinline__ void batch_load_geo(Geo& dst, const Geo& src) {
  static_assert(sizeof(Geo) % 4 == 0, "Geo is copied as words");
  const int* s = reinterpret_cast<const int*>(&src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Geo) / 4); i += blockDim.x) d[i] = s[i];
}

}  // namespace phy
