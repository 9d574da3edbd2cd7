// Segment kernel on the tcgen05 tensor cores: the corner cross-Gram X = C^H C and the matched
// filter V = C^H y of every RE of a frequency segment, as real GEMMs with FP32 accumulation in
// tensor memory (the paper's covariance-by-FMA step of Fig. 2(b), on the dense unit).
//
// Complex products are embedded in real ones. With the corner-layer columns of C as rows of
// CC = [C ; iC] (row c: (Re C_rc, Im C_rc) interleaved over r; row NXP + c: (-Im, Re)), and y
// likewise interleaved over r:
//   (CC CC_C^T)[c][m]      = Re X[c][m],   (CC CC_C^T)[NXP + c][m] = Im X[c][m]    (M=128, N=NXP)
//   (Yt CC^T)[re][c]       = Re V[c][re],  (Yt CC^T)[re][NXP + c]  = Im V[c][re]   (M=128, N=2NXP)
// with K = 2 x 64 receive antennas (zero-padded). Operands are rounded to TF32, FP16 or BF16
// (round to nearest) when staged; everything after the products stays FP32. The epilogue folds X
// into the per-symbol Gram blocks (as the FP32 kernel does) and V into the matched filter
// b = sum over corners of the interpolation weights times V, per RE, straight from TMEM.
//
// One persistent CTA per SM, warp-specialised:
//  - a producer warp streams the received grid through a ring of shared-memory stages with TMA
//    tensor copies (one box = 16 subcarriers x all antennas of one data symbol) and the anchors
//    of the next segment's corners, running ahead of the consumers by up to the ring's depth;
//  - eight converter warps turn anchors into the CC operand and boxes into the RE-tile operand
//    (conversion to the MMA type and K-major core-matrix order);
//  - one warp issues the MMAs as operands become ready, so that conversion never waits on MMA
//    issue;
//  - four drain warps fold X into the Gram blocks and the accumulators into the matched filter.
// RE tiles are whole data symbols of the segment (floor(128 / W) of them), double-buffered in
// shared and tensor memory, so that converting one tile overlaps the MMA of the previous one
// and the drain of the one before. The groups hand over through mbarriers.
// Every wait is bounded: on a timeout a group agrees (barrier with OR-reduction), bumps an
// error counter and leaves; outstanding copies and MMAs are waited for before the CTA ends.
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "batch.cuh"
#include "launch.h"
#include "segment.cuh"
#include "tc.cuh"

namespace phy {

namespace {

constexpr int kConvWarps = 8;   // converters: anchors -> CC, boxes -> RE tiles, MMA issue
constexpr int kDrainWarps = 4;  // drain: X -> Gram blocks, accumulators -> matched filter
constexpr int kConv = 32 * kConvWarps;
constexpr int kMmaWarp = kConvWarps + kDrainWarps;  // issues every MMA of the CTA
constexpr int kProducerWarp = kMmaWarp + 1;
constexpr int kTcThreads = 32 * (kProducerWarp + 1);
constexpr int kRows = 128;                 // UMMA M and rows of every operand tile
constexpr int kK = 128;                    // K elements per operand row: (re, im) x 64 antennas
constexpr int kBoxSc = 16;                 // subcarriers per received-grid box
constexpr uint32_t kStageBytes = kBoxSc * 8 * 64;  // one box with 64 antennas
constexpr int kBoxItems = 16 * (kBoxSc / 2);       // converter work items per box
constexpr int kBoxWarps = kBoxItems / 32;          // converter warps per box
constexpr uint32_t kRingBytes = 64 * 1024;         // ring of boxes (FP16/BF16 tiles)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColX = 0, kColMf = 128;  // MF accumulator b at kColMf + 128 b
constexpr uint32_t kWaitIters = kWaitSegDefault;  // drains of work in flight (polls of ~1 us)

template <uint32_t FMT>
struct Layout {
  static constexpr int kEs = tc::Elem<FMT>::kBytes;
  static constexpr int kTileBytes = kRows * kK * kEs;
  // no-swizzle K-major core matrices (8 rows x 16 bytes), K-chunk major
  static constexpr uint32_t kLbo = (kRows / 8) * 128;  // next 16-byte K chunk
  static constexpr uint32_t kSbo = 128;                // next 8-row group
  static constexpr int kKSteps = kK * kEs / 32;        // one MMA per 32 bytes of K
  __device__ static uint32_t off(int row, int kel) {
    const int bk = kel * kEs;
    return ((bk >> 4) * (kRows / 8) + (row >> 3)) * 128 + (row & 7) * 16 + (bk & 15);
  }
  // RE-tile operand buffers and ring stages: TF32 tiles are twice as large, so that variant
  // keeps one tile buffer and a shallower ring to stay inside 227 KB.
  static constexpr int kYBufs = FMT == tc::kFmtTF32 ? 1 : 2;
  static constexpr int kStages = (FMT == tc::kFmtTF32 ? 48 * 1024 : kRingBytes) / kStageBytes;
};

constexpr int nxp_of(int nx) { return nx <= 16 ? 16 : (nx + 15) / 16 * 16; }
constexpr size_t up128(size_t v) { return (v + 127) & ~(size_t)127; }

// Shared-memory map: CC tile | RE tiles | X (FP32) | anchor corners | ring of RS stages |
// barriers.
template <int NL, int NC, uint32_t FMT, int RS>
struct Smem {
  using Lay = Layout<FMT>;
  static constexpr int NXP = nxp_of(NC * NL);
  static constexpr size_t kCc = 0;
  static constexpr size_t kYop = kCc + Lay::kTileBytes;
  static constexpr size_t kXs = kYop + (size_t)Lay::kYBufs * Lay::kTileBytes;
  static constexpr size_t kAnch = kXs + up128((size_t)NXP * (NXP + 1) / 2 * 8);  // X, lower
  static constexpr size_t kCorner = up128((size_t)NL * 64 * 8);  // one corner's [l][r] block
  static constexpr size_t kRing = kAnch + NC * kCorner;
  static constexpr size_t kBars = kRing + (size_t)RS * kStageBytes;
  // full[S], empty[S], anchors full / empty, X done / drained, MF done[2] / drained[2],
  // CC converted, RE tile converted[2]
  static constexpr int kNumBars = 2 * RS + 11;
  static constexpr size_t kMisc = kBars + 8 * kNumBars;  // TMEM address, consumed counts
  static constexpr size_t kTotal = kMisc + 16;
};

template <uint32_t FMT>
__device__ __forceinline__ void store_pair(unsigned char* p, float a, float b) {
  if constexpr (FMT == tc::kFmtTF32)
    *reinterpret_cast<uint2*>(p) = tc::Elem<FMT>::pack(a, b);
  else
    *reinterpret_cast<uint32_t*>(p) = tc::Elem<FMT>::pack(a, b);
}

// Four consecutive antennas (8 K elements) of one operand row: one 16-byte chunk in FP16/BF16,
// two in TF32.
template <uint32_t FMT>
__device__ __forceinline__ void store_quad(unsigned char* tile, int row, int q, const cf (&v)[4]) {
  using Lay = Layout<FMT>;
  if constexpr (FMT == tc::kFmtTF32) {
    const uint2 a = tc::Elem<FMT>::pack(v[0].x, v[0].y), b = tc::Elem<FMT>::pack(v[1].x, v[1].y);
    const uint2 c = tc::Elem<FMT>::pack(v[2].x, v[2].y), d = tc::Elem<FMT>::pack(v[3].x, v[3].y);
    *reinterpret_cast<uint4*>(tile + Lay::off(row, 8 * q)) = make_uint4(a.x, a.y, b.x, b.y);
    *reinterpret_cast<uint4*>(tile + Lay::off(row, 8 * q + 4)) = make_uint4(c.x, c.y, d.x, d.y);
  } else {
    *reinterpret_cast<uint4*>(tile + Lay::off(row, 8 * q)) =
        make_uint4(tc::Elem<FMT>::pack(v[0].x, v[0].y), tc::Elem<FMT>::pack(v[1].x, v[1].y),
                   tc::Elem<FMT>::pack(v[2].x, v[2].y), tc::Elem<FMT>::pack(v[3].x, v[3].y));
  }
}

// Issues one K-loop of MMAs (A and B tiles in the same layout) and commits to the barrier.
template <uint32_t FMT>
__device__ __forceinline__ void gemm_issue(uint32_t tmem, const unsigned char* a,
                                           const unsigned char* b, uint32_t idesc,
                                           uint64_t* bar) {
  using Lay = Layout<FMT>;
  // descriptors built once; each K step is a fixed byte offset from them
  const uint64_t da = tc::smem_desc(tc::smem_u32(a), Lay::kLbo, Lay::kSbo);
  const uint64_t db = tc::smem_desc(tc::smem_u32(b), Lay::kLbo, Lay::kSbo);
#pragma unroll
  for (int s = 0; s < Lay::kKSteps; ++s) {
    const uint32_t step = (uint32_t)s * 2u * Lay::kLbo;
    tc::mma<FMT>(tmem, tc::desc_advance(da, step), tc::desc_advance(db, step), idesc,
                 s > 0 ? 1u : 0u);
  }
  tc::mma_commit(bar);
}

// One (segment, cell) work item and its RE tiles: whole data symbols of the segment. Boxes
// start at the even subcarrier lo2 <= lo (TMA needs 16-byte aligned inner coordinates).
struct Item {
  int j, lc, cell, lo, lo2, W, spt, ntile, nb;  // nb: boxes per symbol
};
__device__ __forceinline__ Item item_of(const Geo& g, int w, int cell0) {
  Item it;
  it.j = w % g.n_seg;
  it.lc = w / g.n_seg;
  it.cell = cell0 + it.lc;
  int hi;
  segment_range(g, it.j, it.lo, hi);
  it.W = hi - it.lo;  // <= 64 (host-checked), so spt >= 2
  it.spt = kRows / it.W;
  it.ntile = (g.n_dsym + it.spt - 1) / it.spt;
  it.lo2 = it.lo & ~1;
  it.nb = (hi - it.lo2 + kBoxSc - 1) / kBoxSc;
  return it;
}
__device__ __forceinline__ int tile_syms(const Geo& g, const Item& it, int t) {
  return min(it.spt, g.n_dsym - t * it.spt);
}

// Where a work item's job lives: its geometry, tensor maps, outputs and error word, and the
// item's index within the job.
struct TcView {
  const Geo* g;
  const CUtensorMap* tmY;
  const CUtensorMap* tmA;
  float4* ygg;
  cf* bvec;
  unsigned* err;
  int w, cell0;
};
// One job: (segment, cell) items of the chunk starting at cell0; maps are kernel parameters.
struct TcSingle {
  static constexpr bool kBatched = false;
  const Geo* g;
  const CUtensorMap* tmY;
  const CUtensorMap* tmA;
  float4* ygg;
  cf* bvec;
  unsigned* err;
  int cell0, nc;
  __device__ int n_work() const { return g->n_seg * nc; }
  __device__ TcView at(int w) const { return TcView{g, tmY, tmA, ygg, bvec, err, w, cell0}; }
};
// The batched receiver's tensor-core jobs of one layer class; maps are in the device table.
struct TcBatch {
  static constexpr bool kBatched = true;
  const BatchTable* t;
  int cls;
  __device__ int n_work() const { return t->n_items[kBatchSegTc][cls]; }
  __device__ TcView at(int w) const {
    int local;
    const BatchJob& J = t->job[batch_find(t, kBatchSegTc, cls, w, local)];
    return TcView{&J.g, &J.tmY, &J.tmA, J.ygg, J.bvec, J.err, local, 0};
  }
};

// The kernel body over the work items of a source (TcSingle or TcBatch).
template <int NL, int NC, uint32_t FMT, int RS, class Src>
__device__ __forceinline__ void seg_prep_tc_body(const Src& src) {
  using Lay = Layout<FMT>;
  using Sm = Smem<NL, NC, FMT, RS>;
  constexpr int S = RS;
  constexpr int NX = NC * NL;
  constexpr int NXP = Sm::NXP;
  constexpr int NTRI = NL * (NL + 1) / 2;
  static_assert(2 * NXP <= kRows, "corner-layer count too large for one tile");
  static_assert(Sm::kTotal <= 227 * 1024, "shared memory map too large");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* cc = smem + Sm::kCc;
  cf* Xs = reinterpret_cast<cf*>(smem + Sm::kXs);
  unsigned char* anch = smem + Sm::kAnch;
  unsigned char* ring = smem + Sm::kRing;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Sm::kBars);
  uint64_t* empty = full + S;
  uint64_t* a_full = empty + S;
  uint64_t* a_empty = a_full + 1;
  uint64_t* x_bar = a_full + 2;
  uint64_t* x_free = a_full + 3;
  uint64_t* mf_bar = a_full + 4;     // [2]
  uint64_t* tmem_free = a_full + 6;  // [2]
  uint64_t* cc_ready = a_full + 8;
  uint64_t* tile_ready = a_full + 9;  // [2]
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + Sm::kMisc);  // TMEM address

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_work = src.n_work();

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(full + s, 1);
      tc::mbar_init(empty + s, kBoxWarps);  // arrivals: the converter warps of a box
    }
    tc::mbar_init(a_full, 1);
    tc::mbar_init(a_empty, kConvWarps);
    tc::mbar_init(x_bar, 1);
    tc::mbar_init(x_free, 4);  // arrivals: the four drain warps
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(mf_bar + b, 1);
      tc::mbar_init(tmem_free + b, 4);
      tc::mbar_init(tile_ready + b, kConvWarps);  // arrivals: the converter warps
    }
    tc::mbar_init(cc_ready, kConvWarps);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(misc, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = misc[0];

  if (warp == kProducerWarp) {
    // ------------------------------------------------------------ producer
    uint32_t nbox = 0, nitem = 0;  // boxes and anchor sets issued
    if (lane == 0) {
      bool ok = true;
      for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x) {
        const TcView v = src.at(w);
        const Geo& g = *v.g;
        const Item it = item_of(g, v.w, v.cell0);
        const int nds = g.n_dsym;
        const uint32_t y_box_bytes = (uint32_t)g.n_rx * kBoxSc * 8;
        const uint32_t a_box_bytes = (uint32_t)g.n_layers * g.n_rx * 8;
        if constexpr (Src::kBatched) {  // maps written through the generic proxy (the table copy)
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(v.tmY)
                       : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(v.tmA)
                       : "memory");
        }
        if (nitem > 0) ok = tc::mbar_wait_sleep(a_empty, (nitem - 1) & 1, g.wait_seg);
        if (!ok) break;
        tc::mbar_arrive_expect_tx(a_full, NC * a_box_bytes);
        const int g1 = seg_g1(g, it.j);
        for (int corner = 0; corner < NC; ++corner) {
          const int d = corner >> 1, grp = (corner & 1) ? g1 : it.j;
          tc::tma_load_3d(anch + corner * Sm::kCorner, v.tmA, 0, 0,
                          (it.cell * g.n_dmrs + d) * g.G + grp, a_full);
        }
        ++nitem;
        for (int jj = 0; jj < nds && ok; ++jj) {
          const int z = it.cell * g.n_sym + g.dsym[jj];
          for (int b = 0; b < it.nb; ++b) {
            const uint32_t s = nbox % S;
            if (nbox >= (uint32_t)S) ok = tc::mbar_wait_sleep(empty + s, ((nbox / S) - 1) & 1, g.wait_seg);
            if (!ok) break;
            tc::mbar_arrive_expect_tx(full + s, y_box_bytes);
            tc::tma_load_3d(ring + s * kStageBytes, v.tmY, 2 * (it.lo2 + kBoxSc * b), 0, z,
                            full + s);
            ++nbox;
          }
        }
      }
    }
    __syncwarp();
    __syncthreads();
    if (lane == 0) {
      // Copies the workers did not wait for (only after a timeout) must land before the CTA
      // ends. A stage's copies complete in order, so waiting for its latest one is enough.
      for (uint32_t s = 0; s < (uint32_t)S && s < nbox; ++s) {
        const uint32_t last = s + ((nbox - 1 - s) / S) * S;
        tc::mbar_wait_sleep(full + s, (last / S) & 1, kWaitIters);
      }
      if (nitem > 0) tc::mbar_wait_sleep(a_full, (nitem - 1) & 1, kWaitIters);
    }
    return;
  }

  // -------------------------------------------------------------- workers
  // Each group agrees on timeouts at its own named barrier (1: converters, 2: drain).
  const int quarter = warp & 3, gtid = warp < kConvWarps ? tid : tid - kConv;
  const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
  bool fail = false;  // this thread saw a timeout
  bool stop = false;  // a thread of its group did (agreed at a group barrier)

  if (warp < kConvWarps) {
    uint32_t nbox = 0, nitem = 0, ntile = 0;  // boxes, anchor sets and RE tiles consumed
    unsigned* err = nullptr;                   // the current item's error word
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
      const TcView v = src.at(w);
      const Geo& g = *v.g;
      const Item it = item_of(g, v.w, v.cell0);
      const int nr = g.n_rx, nl = g.n_layers;
      err = v.err;
      // every MMA of the previous item read CC; its last commit covers them all
      if (ntile > 0) fail |= !tc::mbar_wait_sleep(mf_bar + ((ntile - 1) & 1), ((ntile - 1) >> 1) & 1,
                                            g.wait_seg);
      fail |= !tc::mbar_wait_sleep(a_full, nitem & 1, g.wait_seg);
      ++nitem;
      // ---- CC = [C ; iC] from the anchors of the segment's corners, four antennas per item.
      // A warp takes 8 rows x 4 antenna quads: its 16-byte stores fill whole 128-byte core
      // matrix rows (no bank conflicts), its anchor loads spread over the banks.
#pragma unroll 2
      for (int e = gtid; e < NXP * 16; e += kConv) {
        const int rq = (e >> 3) & 15, c = ((e >> 7) << 3) | (e & 7);
        const int corner = c / NL, l = c % NL;
        cf v[4];
        const float2* src =
            reinterpret_cast<const float2*>(anch + corner * Sm::kCorner) + l * nr + 4 * rq;
        if (c < NX && l < nl && 4 * rq + 3 < nr) {
          const float4 a = reinterpret_cast<const float4*>(src)[0];
          const float4 b = reinterpret_cast<const float4*>(src)[1];
          v[0] = mk(a.x, a.y);
          v[1] = mk(a.z, a.w);
          v[2] = mk(b.x, b.y);
          v[3] = mk(b.z, b.w);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            v[u] = mk(0.f, 0.f);
            if (c < NX && l < nl && 4 * rq + u < nr) v[u] = mk(src[u].x, src[u].y);
          }
        }
        cf iv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) iv[u] = mk(-v[u].y, v[u].x);
        store_quad<FMT>(cc, c, rq, v);
        store_quad<FMT>(cc, NXP + c, rq, iv);
      }
      tc::fence_proxy_async();  // the generic stores before the MMAs' async-proxy reads
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(a_empty);
        tc::mbar_arrive(cc_ready);
      }
      stop = tc::bar_or<1, kConv>(fail);
      if (stop) break;
      for (int t = 0; t < it.ntile; ++t, ++ntile) {
        const uint32_t buf = ntile & 1;
        unsigned char* yop =
            smem + Sm::kYop + (size_t)(Lay::kYBufs == 2 ? buf : 0) * Lay::kTileBytes;
        // the tile buffer is free once the MMA that last read it (kYBufs tiles back) is done
        constexpr uint32_t back = Lay::kYBufs;
        if (ntile >= back)
          fail |= !tc::mbar_wait_sleep(mf_bar + ((ntile - back) & 1), ((ntile - back) >> 1) & 1,
                                 g.wait_seg);
        // ---- boxes of tile t -> RE-tile operand: kSlots boxes per round, each thread two
        // subcarriers x four antennas of a box (four 16-byte loads, two chunk stores)
        const int nbx = tile_syms(g, it, t) * it.nb;
        const int slot = gtid / kBoxItems, item = gtid % kBoxItems;
        const int qa = item / (kBoxSc / 2), pr = item % (kBoxSc / 2);  // antenna quad, pair
        int js = slot / it.nb, bb = slot % it.nb;  // (symbol, box) of box index slot
        // Box bx goes to slot bx % kSlots. A stage's consecutive boxes are kStages apart, so
        // with kStages a multiple of kSlots one slot consumes a stage's boxes in order and never
        // polls a stage for its next phase while the previous one is still pending (parity
        // waits cannot tell those two apart).
        constexpr int kSlots = kConv / kBoxItems;
        static_assert(S % kSlots == 0, "ring depth must be a multiple of the box slots");
        for (int bx = slot; bx < nbx; bx += kSlots) {
          const uint32_t n = nbox + bx, s = n % S;
          fail |= !tc::mbar_wait_sleep(full + s, (n / S) & 1, g.wait_seg);
          const float4* raw = reinterpret_cast<const float4*>(ring + s * kStageBytes);
          cf v0[4], v1[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = 4 * qa + u;
            const float4 f = r < nr ? raw[r * (kBoxSc / 2) + pr] : make_float4(0.f, 0.f, 0.f, 0.f);
            v0[u] = mk(f.x, f.y);
            v1[u] = mk(f.z, f.w);
          }
          const int kk = bb * kBoxSc + 2 * pr + it.lo2 - it.lo;
          if (kk >= 0 && kk < it.W) store_quad<FMT>(yop, js * it.W + kk, qa, v0);
          if (kk + 1 >= 0 && kk + 1 < it.W) store_quad<FMT>(yop, js * it.W + kk + 1, qa, v1);
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(empty + s);
          bb += kSlots;
          while (bb >= it.nb) {
            bb -= it.nb;
            ++js;
          }
        }
        nbox += nbx;
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(tile_ready + buf);
        stop = tc::bar_or<1, kConv>(fail);
        if (stop) break;
      }
      if (stop) break;
    }
    if (gtid == 0 && stop && err) atomicAdd(err, 1u);
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    // X = C^H C once CC is converted and the drain has read the previous X; V = C^H y per RE
    // tile once the tile is converted and the drain has emptied the accumulator buffer.
    uint32_t nitem = 0, ntile = 0, x_count = 0, mf_count[2] = {0, 0};
    unsigned* err = nullptr;
    if (lane == 0) {
      for (int w = blockIdx.x; w < n_work && !fail; w += gridDim.x) {
        const TcView v = src.at(w);
        const Geo& g = *v.g;
        const Item it = item_of(g, v.w, v.cell0);
        err = v.err;
        fail |= !tc::mbar_wait_sleep(cc_ready, nitem & 1, g.wait_seg);
        if (nitem > 0) fail |= !tc::mbar_wait_sleep(x_free, (nitem - 1) & 1, g.wait_seg);
        ++nitem;
        if (fail) break;
        tc::fence_after_sync();
        gemm_issue<FMT>(tmem + kColX, cc, cc, tc::instr_desc(FMT, kRows, NXP), x_bar);
        ++x_count;
        for (int t = 0; t < it.ntile && !fail; ++t, ++ntile) {
          const uint32_t buf = ntile & 1;
          const unsigned char* yop =
              smem + Sm::kYop + (size_t)(Lay::kYBufs == 2 ? buf : 0) * Lay::kTileBytes;
          fail |= !tc::mbar_wait_sleep(tile_ready + buf, (ntile >> 1) & 1, g.wait_seg);
          if (ntile >= 2)
            fail |= !tc::mbar_wait_sleep(tmem_free + buf, ((ntile - 2) >> 1) & 1, g.wait_seg);
          if (fail) break;
          tc::fence_after_sync();
          gemm_issue<FMT>(tmem + kColMf + 128 * buf, yop, cc,
                          tc::instr_desc(FMT, kRows, 2 * NXP), mf_bar + buf);
          ++mf_count[buf];
        }
      }
      if (fail && err) atomicAdd(err, 1u);
      // MMAs still running (only after a timeout) must finish before tensor memory is released
      if (x_count) tc::mbar_wait_sleep(x_bar, (x_count - 1) & 1, kWaitIters);
      for (int b = 0; b < 2; ++b)
        if (mf_count[b]) tc::mbar_wait_sleep(mf_bar + b, (mf_count[b] - 1) & 1, kWaitIters);
    }
    __syncwarp();
  } else {
    uint32_t nitem = 0, ntile = 0;
    unsigned* err = nullptr;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
      const TcView v = src.at(w);
      const Geo& g = *v.g;
      const Item it = item_of(g, v.w, v.cell0);
      const int nds = g.n_dsym;
      float4* ygg = v.ygg;
      cf* bvec = v.bvec;
      err = v.err;
      // ---- X -> shared memory (after every drain warp is done with the previous item's X)
      fail |= !tc::mbar_wait_sleep(x_bar, nitem & 1, g.wait_seg);
      tc::fence_after_sync();
      tc::bar_sync<2, 128>();
      {
        const int row = 32 * quarter + lane;
#pragma unroll
        for (int c0 = 0; c0 < NXP; c0 += 32) {
          float v[32];
          tc::tmem_ld32(tmem + lane_base + kColX + c0, v);
          if (row < 2 * NXP) {
            const int c = row % NXP, part = row / NXP;
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (c0 + q <= c)  // lower triangle, packed by rows
                reinterpret_cast<float*>(Xs + c * (c + 1) / 2 + c0 + q)[part] = v[q];
          }
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(x_free);
      stop = tc::bar_or<2, 128>(fail);
      if (stop) break;
      // ---- per-symbol Gram blocks
      auto Xget = [&](int i, int k) -> cf {  // X is Hermitian
        if (i >= k) return Xs[i * (i + 1) / 2 + k];
        const cf v = Xs[k * (k + 1) / 2 + i];
        return mk(v.x, -v.y);
      };
      form_gram_blocks<NL, 128>(g, Xget,
                                ygg + (((size_t)it.lc * g.n_seg + it.j) * nds) * NTRI * 2, gtid);
      // ---- matched filter of each RE tile: this thread's TMEM lane is its RE row
      for (int t = 0; t < it.ntile; ++t, ++ntile) {
        const uint32_t buf = ntile & 1;
        fail |= !tc::mbar_wait_sleep(mf_bar + buf, (ntile >> 1) & 1, g.wait_seg);
        tc::fence_after_sync();
        const int row = 32 * quarter + lane;
        const int nrow = tile_syms(g, it, t) * it.W;
        const bool valid = row < nrow;
        const int jj = t * it.spt + (valid ? row / it.W : 0);
        const int k = it.lo + (valid ? row % it.W : 0);
        const float t1 = g.tw[jj], t0 = 1.f - t1;
        const float be0 = seg_beta(g, it.j, k, 0), be1 = seg_beta(g, it.j, k, 1);
        // weight of corner (d, g) for a layer on comb p: tau_d (1 - beta_p or beta_p)
        float wc[2][4];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const float be = p ? be1 : be0;
          wc[p][0] = t0 * (1.f - be);
          wc[p][1] = t0 * be;
          wc[p][2] = t1 * (1.f - be);
          wc[p][3] = t1 * be;
        }
        float bre[NL], bim[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) bre[l] = bim[l] = 0.f;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
#pragma unroll
          for (int c0 = 0; c0 < NXP; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + lane_base + kColMf + 128 * buf + part * NXP + c0, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              const int c = c0 + q;
              if (c < NX) {
                const int corner = c / NL, l = c % NL;
                const float wt = wc[l & 1][corner];
                if (part == 0)
                  bre[l] = fmaf(wt, v[q], bre[l]);
                else
                  bim[l] = fmaf(wt, v[q], bim[l]);
              }
            }
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(tmem_free + buf);
        if (valid) {
          float4* bo = reinterpret_cast<float4*>(bvec +
                                                 ((size_t)(it.lc * nds + jj) * g.n_sc + k) * NL);
#pragma unroll
          for (int l = 0; l < NL; l += 2)
            bo[l / 2] = make_float4(bre[l], bim[l], bre[l + 1], bim[l + 1]);
        }
      }
      ++nitem;
      stop = tc::bar_or<2, 128>(fail);
      if (stop) break;
    }
    if (gtid == 0 && stop && err) atomicAdd(err, 1u);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <int NL, int NC, uint32_t FMT, int RS>
__global__ void __launch_bounds__(kTcThreads, 1)
    seg_prep_tc_kernel(const __grid_constant__ CUtensorMap tmY,
                       const __grid_constant__ CUtensorMap tmA, const __grid_constant__ Geo g,
                       int cell0, int nc, float4* __restrict__ ygg, cf* __restrict__ bvec,
                       unsigned* __restrict__ err) {
  const TcSingle src{&g, &tmY, &tmA, ygg, bvec, err, cell0, nc};
  seg_prep_tc_body<NL, NC, FMT, RS>(src);
}

// Batched form: the FP16 tensor-core jobs of one layer class (two DMRS symbols) in the table.
template <int NL>
__global__ void __launch_bounds__(kTcThreads, 1)
    seg_prep_tc_batch_kernel(const BatchTable* __restrict__ t) {
  const TcBatch src{t, batch_class(NL)};
  seg_prep_tc_body<NL, 4, tc::kFmtF16, Layout<tc::kFmtF16>::kStages>(src);
}

// ---------------------------------------------------------------- host side
}  // namespace

// Received grid: (2 n_sc floats, n_rx, n_cells n_sym), box = kBoxSc subcarriers x all antennas.
// Anchors: (2 n_rx floats, n_layers, n_cells n_dmrs G), box = one corner's [layer][antenna].
bool encode_tc_maps(const Geo& g, const phy_c32* anchors, const phy_c32* Y, CUtensorMap* tmY,
                    CUtensorMap* tmA) {
  const cuuint64_t ydim[3] = {(cuuint64_t)2 * g.n_sc, (cuuint64_t)g.n_rx,
                              (cuuint64_t)g.n_cells * g.n_sym};
  const cuuint64_t ystr[2] = {(cuuint64_t)8 * g.n_sc, (cuuint64_t)8 * g.n_sc * g.n_rx};
  const cuuint32_t ybox[3] = {2 * kBoxSc, (cuuint32_t)g.n_rx, 1};
  const cuuint64_t adim[3] = {(cuuint64_t)2 * g.n_rx, (cuuint64_t)g.n_layers,
                              (cuuint64_t)g.n_cells * g.n_dmrs * g.G};
  const cuuint64_t astr[2] = {(cuuint64_t)8 * g.n_rx, (cuuint64_t)8 * g.n_rx * g.n_layers};
  const cuuint32_t abox[3] = {(cuuint32_t)2 * g.n_rx, (cuuint32_t)g.n_layers, 1};
  return make_map(tmY, Y, ydim, ystr, ybox) && make_map(tmA, anchors, adim, astr, abox);
}

namespace {

template <int NL, int NC, uint32_t FMT, int RS>
cudaError_t launch_one(const Geo& g, int c0, int nc, const phy_c32* anchors, const phy_c32* Y,
                       float4* ygg, cf* bvec, unsigned* err, cudaStream_t st) {
  constexpr size_t smem = Smem<NL, NC, FMT, RS>::kTotal;
  static bool configured_on[kMaxDevices] = {};
  bool& configured = configured_on[current_device()];
  const int num_sms = device_sm_count();
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(seg_prep_tc_kernel<NL, NC, FMT, RS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (std::getenv("PHY_DEBUG"))
      std::fprintf(stderr, "seg_prep_tc<%d,%d,%u,%d>: smem %zu, SMs %d\n", NL, NC, FMT, RS, smem,
                   num_sms);
    configured = true;
  }
  // Received grid: (2 n_sc floats, n_rx, n_cells n_sym), box = kBoxSc subcarriers x all antennas.
  // Anchors: (2 n_rx floats, n_layers, n_cells n_dmrs G), box = one corner's [layer][antenna].
  CUtensorMap tmY, tmA;
  if (!encode_tc_maps(g, anchors, Y, &tmY, &tmA)) return cudaErrorInvalidValue;
  const int n_work = g.n_seg * nc;
  const int grid = std::min(n_work, num_sms);
  seg_prep_tc_kernel<NL, NC, FMT, RS><<<grid, kTcThreads, smem, st>>>(tmY, tmA, g, c0, nc, ygg,
                                                                      bvec, err);
  return cudaGetLastError();
}

// Ring depth: the format's default, or a deeper ring of kDeepRing stages (more box bytes in
// flight per SM) where the shared-memory map still fits; the autotuner picks.
constexpr int kDeepRing = 12;

template <int NL, int NC, uint32_t FMT>
cudaError_t launch_ring(const Geo& g, int c0, int nc, const phy_c32* anchors, const phy_c32* Y,
                        float4* ygg, cf* bvec, unsigned* err, cudaStream_t st) {
  constexpr int kDef = Layout<FMT>::kStages;
  if constexpr (FMT != tc::kFmtTF32 && Smem<NL, NC, FMT, kDeepRing>::kTotal <= 227 * 1024) {
    if (tuned_tile(g).ring == kDeepRing)
      return launch_one<NL, NC, FMT, kDeepRing>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
  }
  return launch_one<NL, NC, FMT, kDef>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
}

template <int NL, uint32_t FMT>
cudaError_t launch_nc(const Geo& g, int c0, int nc, const phy_c32* anchors, const phy_c32* Y,
                      float4* ygg, cf* bvec, unsigned* err, cudaStream_t st) {
  if (g.n_dmrs == 2) return launch_ring<NL, 4, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
  return launch_ring<NL, 2, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
}

template <uint32_t FMT>
cudaError_t launch_fmt(const Geo& g, int NL, int c0, int nc, const phy_c32* anchors,
                       const phy_c32* Y, float4* ygg, cf* bvec, unsigned* err, cudaStream_t st) {
  switch (NL) {
    case 2: return launch_nc<2, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
    case 4: return launch_nc<4, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
    case 8: return launch_nc<8, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
    default: return launch_nc<16, FMT>(g, c0, nc, anchors, Y, ygg, bvec, err, st);
  }
}

template <int NL>
cudaError_t launch_tc_batch_nl(const BatchTable* t, cudaStream_t st) {
  constexpr size_t smem = Smem<NL, 4, tc::kFmtF16, Layout<tc::kFmtF16>::kStages>::kTotal;
  static bool configured_on[kMaxDevices] = {};
  bool& configured = configured_on[current_device()];
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(seg_prep_tc_batch_kernel<NL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  seg_prep_tc_batch_kernel<NL><<<device_sm_count(), kTcThreads, smem, st>>>(t);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_seg_prep_tc_batch(const BatchTable* t, int nl_cls, cudaStream_t st) {
  switch (nl_cls) {
    case 2: return launch_tc_batch_nl<2>(t, st);
    case 4: return launch_tc_batch_nl<4>(t, st);
    case 8: return launch_tc_batch_nl<8>(t, st);
    default: return launch_tc_batch_nl<16>(t, st);
  }
}

bool tc_deep_ring_fits(const Geo& g) {
  if (g.prec != PHY_PREC_TC_FP16 && g.prec != PHY_PREC_TC_BF16) return false;
  const int nc = g.n_dmrs == 2 ? 4 : 2;
  auto fits = [](size_t total) { return total <= 227 * 1024; };
  switch (nl_class_of(g.n_layers)) {
    case 2: return fits(nc == 4 ? Smem<2, 4, tc::kFmtF16, kDeepRing>::kTotal
                                : Smem<2, 2, tc::kFmtF16, kDeepRing>::kTotal);
    case 4: return fits(nc == 4 ? Smem<4, 4, tc::kFmtF16, kDeepRing>::kTotal
                                : Smem<4, 2, tc::kFmtF16, kDeepRing>::kTotal);
    case 8: return fits(nc == 4 ? Smem<8, 4, tc::kFmtF16, kDeepRing>::kTotal
                                : Smem<8, 2, tc::kFmtF16, kDeepRing>::kTotal);
    default: return fits(nc == 4 ? Smem<16, 4, tc::kFmtF16, kDeepRing>::kTotal
                                 : Smem<16, 2, tc::kFmtF16, kDeepRing>::kTotal);
  }
}

bool seg_prep_tc_supported(const Geo& g) {
  // tensor-map rules: 16-byte strides and inner box extents (even antenna count); tiles of
  // whole data symbols (segments of at most 64 subcarriers, always the case for covers <= 16)
  return g.n_rx % 2 == 0 && host_max_segment_width(g) <= 64;
}

cudaError_t launch_seg_prep_tc(const Geo& g, int NL, int c0, int nc, const phy_c32* anchors,
                               const phy_c32* Y, float4* ygg, cf* bvec, unsigned* err,
                               cudaStream_t st) {
  if (!seg_prep_tc_supported(g) || (reinterpret_cast<uintptr_t>(anchors) % 16) ||
      (reinterpret_cast<uintptr_t>(Y) % 16))
    return cudaErrorInvalidValue;
  switch (g.prec) {
    case PHY_PREC_TC_TF32:
      return launch_fmt<tc::kFmtTF32>(g, NL, c0, nc, anchors, Y, ygg, bvec, err, st);
    case PHY_PREC_TC_BF16:
      return launch_fmt<tc::kFmtBF16>(g, NL, c0, nc, anchors, Y, ygg, bvec, err, st);
    default:
      return launch_fmt<tc::kFmtF16>(g, NL, c0, nc, anchors, Y, ygg, bvec, err, st);
  }
}

}  // namespace phy
