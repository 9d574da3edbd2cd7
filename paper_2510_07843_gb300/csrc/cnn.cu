// Learned channel denoiser: a residual CNN on 12-subcarrier x 14-symbol tiles of the interpolated
// LS estimate (one tile per PRB, Rx antenna and layer), trained and run by the kernels below. The
// paper has no learned part; this is the step between channel estimation and detection.
//
// Network: 3x3 cross-correlations with zero padding, channels 2 -> 32 -> 32 -> 32 -> 2, ReLU after
// the first three, input added to the output. Parameters, one flat FP32 vector: W1 [32][2][3][3],
// b1 [32], W2 [32][32][3][3], b2, W3, b3, W4 [2][32][3][3], b4. Tiles: [n][C][14][12] FP32.
// Loss: mean over tiles and positions of |out - label|^2. Optimiser: Adam.
//
// Kernels (FP32 on the CUDA cores):
//  - conv3x3_kernel<CIN, COUT, MODE, BWD>: persistent CTAs, the layer's weights staged in shared
//    memory once per CTA as [cin][tap][cout], then per tile the input staged zero-padded
//    ([cin][16][14]) and each thread computing 4 output channels x 3 neighbouring columns of one
//    row (the 5 input values of a row segment and the 4 weights of a tap are reused 3 and 4
//    times). With BWD the same kernel is the backward pass to the layer's input: weights read
//    transposed and flipped, W'[ci][co][tap] = W[co][ci][8 - tap].
//  - conv3x3_wgrad_kernel<CIN, COUT>: persistent CTAs accumulate dW and db over their tiles in
//    registers (each thread 2 output x 2 input channels x 9 taps) and write one partial per CTA;
//    reduce_partials sums them in a fixed order, so gradients do not depend on scheduling.
//  - loss_grad_kernel, adam_kernel: elementwise, with fixed-order partial sums for the loss.
#include <algorithm>
#include <cmath>

#include "launch.h"
#include "segment.cuh"

namespace phy {

namespace {

constexpr int kTR = 14, kTC = 12, kTP = kTR * kTC;  // tile rows (symbols), columns, positions
constexpr int kPR = kTR + 2, kPC = kTC + 2;         // zero-padded staging
constexpr int kCnnThreads = 256;
constexpr int kOffW1 = 0, kOffB1 = 576, kOffW2 = 608, kOffB2 = 9824, kOffW3 = 9856,
              kOffB3 = 19072, kOffW4 = 19104, kOffB4 = 19680, kParams = 19682;

enum { kRelu = 0, kResid = 1, kMask = 2 };

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return ((size_t)CIN * 9 * COUT + COUT + (size_t)CIN * kPR * kPC) * sizeof(float);
}

template <int CIN, int COUT, int MODE, bool BWD>
__global__ void __launch_bounds__(kCnnThreads)
    conv3x3_kernel(int n, const float* __restrict__ in, const float* __restrict__ W,
                   const float* __restrict__ bias, const float* __restrict__ aux,
                   float* __restrict__ out) {
  constexpr int CG = COUT < 4 ? COUT : 4;  // output channels per thread
  constexpr int NG = COUT / CG;
  constexpr int ITEMS = NG * kTR * (kTC / 3);
  extern __shared__ __align__(16) float cnn_smem[];
  float* s_w = cnn_smem;                   // [CIN][9][COUT]
  float* s_b = s_w + CIN * 9 * COUT;       // [COUT]
  float* s_in = s_b + COUT;                // [CIN][kPR][kPC]
  for (int e = threadIdx.x; e < CIN * 9 * COUT; e += kCnnThreads) {
    const int co = e % COUT, tap = (e / COUT) % 9, ci = e / (9 * COUT);
    s_w[e] = BWD ? W[(ci * COUT + co) * 9 + (8 - tap)]   // W_orig[ci][co][flip]
                 : W[(co * CIN + ci) * 9 + tap];
  }
  for (int e = threadIdx.x; e < COUT; e += kCnnThreads) s_b[e] = bias ? bias[e] : 0.f;
  for (int e = threadIdx.x; e < CIN * kPR * kPC; e += kCnnThreads) s_in[e] = 0.f;  // borders
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    __syncthreads();  // weights staged / the previous tile's outputs done with s_in
    const float* src = in + (size_t)t * CIN * kTP;
    for (int e = threadIdx.x; e < CIN * kTP; e += kCnnThreads) {
      const int ci = e / kTP, p = e % kTP;
      s_in[(ci * kPR + p / kTC + 1) * kPC + p % kTC + 1] = __ldg(src + e);
    }
    __syncthreads();
    for (int it = threadIdx.x; it < ITEMS; it += kCnnThreads) {
      // consecutive lanes: consecutive row segments of one channel group (contiguous stores,
      // broadcast weight reads)
      const int seg = it % (kTR * (kTC / 3)), cgi = it / (kTR * (kTC / 3));
      const int row = seg / (kTC / 3), c0 = (seg % (kTC / 3)) * 3;
      const int co0 = cgi * CG;
      float acc[CG][3];
#pragma unroll
      for (int g = 0; g < CG; ++g)
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[g][q] = 0.f;
#pragma unroll 2
      for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
        for (int di = 0; di < 3; ++di) {
          const float* r = s_in + (ci * kPR + row + di) * kPC + c0;  // padded: columns c0-1 ..
          float v[5];
#pragma unroll
          for (int q = 0; q < 5; ++q) v[q] = r[q];
#pragma unroll
          for (int dj = 0; dj < 3; ++dj) {
            const float* w = s_w + (ci * 9 + di * 3 + dj) * COUT + co0;
            float wv[CG];
#pragma unroll
            for (int g = 0; g < CG; ++g) wv[g] = w[g];
#pragma unroll
            for (int g = 0; g < CG; ++g)
#pragma unroll
              for (int q = 0; q < 3; ++q) acc[g][q] = fmaf(wv[g], v[q + dj], acc[g][q]);
          }
        }
      }
#pragma unroll
      for (int g = 0; g < CG; ++g) {
        const size_t o = ((size_t)t * COUT + co0 + g) * kTP + row * kTC + c0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          float z = acc[g][q] + s_b[co0 + g];
          if (MODE == kRelu) z = fmaxf(z, 0.f);
          if (MODE == kResid) z += aux[o + q];
          if (MODE == kMask) z = aux[o + q] > 0.f ? z : 0.f;
          out[o + q] = z;
        }
      }
    }
  }
}

// Partial weight and bias gradients over this CTA's tiles: part[blockIdx.x][COUT*CIN*9 + COUT].
template <int CIN, int COUT>
__global__ void __launch_bounds__(kCnnThreads)
    conv3x3_wgrad_kernel(int n, const float* __restrict__ a, const float* __restrict__ dz,
                         float* __restrict__ part) {
  constexpr int CP = CIN / 2, OP = COUT / 2;  // channel pairs
  // channel stride of the staged activations padded by one word: the lanes of a warp read 16
  // different channel pairs at once, which an unpadded stride (448 words) puts in one bank
  constexpr int kCS = kPR * kPC + 1;
  extern __shared__ __align__(16) float cnn_smem[];
  float* s_a = cnn_smem;                 // [CIN][kCS] zero-padded
  float* s_d = s_a + CIN * kCS;          // [COUT][kTP]
  const int op = threadIdx.x / CP, cp = threadIdx.x % CP;
  const bool active = threadIdx.x < CP * OP;
  float acc[2][2][9], bacc[2] = {0.f, 0.f};
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[x][y][k] = 0.f;
  for (int e = threadIdx.x; e < CIN * kCS; e += kCnnThreads) s_a[e] = 0.f;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    __syncthreads();
    for (int e = threadIdx.x; e < CIN * kTP; e += kCnnThreads) {
      const int ci = e / kTP, p = e % kTP;
      s_a[ci * kCS + (p / kTC + 1) * kPC + p % kTC + 1] = __ldg(a + (size_t)t * CIN * kTP + e);
    }
    for (int e = threadIdx.x; e < COUT * kTP; e += kCnnThreads)
      s_d[e] = __ldg(dz + (size_t)t * COUT * kTP + e);
    __syncthreads();
    if (!active) continue;
#pragma unroll 1
    for (int row = 0; row < kTR; ++row) {
      float d[2][kTC];
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int j = 0; j < kTC; ++j) d[x][j] = s_d[(2 * op + x) * kTP + row * kTC + j];
      if (cp == 0) {
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int j = 0; j < kTC; ++j) bacc[x] += d[x][j];
      }
#pragma unroll
      for (int di = 0; di < 3; ++di) {
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          const float* r = s_a + (2 * cp + y) * kCS + (row + di) * kPC;
          float v[kPC];
#pragma unroll
          for (int j = 0; j < kPC; ++j) v[j] = r[j];
#pragma unroll
          for (int x = 0; x < 2; ++x)
#pragma unroll
            for (int dj = 0; dj < 3; ++dj) {
              float s = acc[x][y][di * 3 + dj];
#pragma unroll
              for (int j = 0; j < kTC; ++j) s = fmaf(d[x][j], v[j + dj], s);
              acc[x][y][di * 3 + dj] = s;
            }
        }
      }
    }
  }
  if (!active) return;
  float* p = part + (size_t)blockIdx.x * (COUT * CIN * 9 + COUT);
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int k = 0; k < 9; ++k) p[((2 * op + x) * CIN + 2 * cp + y) * 9 + k] = acc[x][y][k];
  if (cp == 0) {
    p[COUT * CIN * 9 + 2 * op] = bacc[0];
    p[COUT * CIN * 9 + 2 * op + 1] = bacc[1];
  }
}

// grad[k] = sum over the CTAs' partials, in CTA order.
__global__ void reduce_partials(const float* __restrict__ part, int n_part, int len,
                                float* __restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= len) return;
  float s = 0.f;
  for (int c = 0; c < n_part; ++c) s += part[(size_t)c * len + k];
  grad[k] = s;
}

// dout = 2 (out - label) / (n P); per-CTA partial sums of (out - label)^2 / (n P).
__global__ void __launch_bounds__(kCnnThreads)
    loss_grad_kernel(long long total, float inv_np, const float* __restrict__ out,
                     const float* __restrict__ label, float* __restrict__ dout,
                     float* __restrict__ loss_part) {
  float s = 0.f;
  for (long long i = (long long)blockIdx.x * kCnnThreads + threadIdx.x; i < total;
       i += (long long)gridDim.x * kCnnThreads) {
    const float e = out[i] - label[i];
    dout[i] = 2.f * e * inv_np;
    s = fmaf(e, e, s);
  }
  __shared__ float red[kCnnThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kCnnThreads / 32; ++w) t += red[w];
    loss_part[blockIdx.x] = t * inv_np;
  }
}

__global__ void adam_kernel(int len, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= len) return;
  const float gk = g[k];
  const float mk_ = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk_;
  v[k] = vk;
  p[k] -= lr * (mk_ * c1) / (sqrtf(vk * c2) + eps);
}

constexpr int kMaxCnnGrid = 512;  // persistent CTAs at most (bounds the gradient partials)
constexpr size_t kPartFloats = (size_t)kMaxCnnGrid * (9216 + 32);
int cnn_grid(int n) {
  return std::max(1, std::min(std::min(n, 3 * device_sm_count()), kMaxCnnGrid));
}

template <int CIN, int COUT, int MODE, bool BWD>
cudaError_t conv(int n, const float* in, const float* W, const float* b, const float* aux,
                 float* out, cudaStream_t st) {
  constexpr size_t smem = conv_smem<CIN, COUT>();
  static bool set_on[kMaxDevices] = {};
  bool& set = set_on[current_device()];
  if (!set) {
    cudaError_t e = cudaFuncSetAttribute(conv3x3_kernel<CIN, COUT, MODE, BWD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    set = true;
  }
  conv3x3_kernel<CIN, COUT, MODE, BWD><<<cnn_grid(n), kCnnThreads, smem, st>>>(n, in, W, b, aux,
                                                                              out);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad(int n, const float* a, const float* dz, float* part, float* grad_w,
                  float* grad_b, cudaStream_t st) {
  constexpr size_t smem = ((size_t)CIN * (kPR * kPC + 1) + (size_t)COUT * kTP) * sizeof(float);
  static bool set_on[kMaxDevices] = {};
  bool& set = set_on[current_device()];
  if (!set) {
    cudaError_t e = cudaFuncSetAttribute(conv3x3_wgrad_kernel<CIN, COUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    set = true;
  }
  // at least four tiles per CTA: fewer partials to write and sum
  const int grid = std::max(1, std::min(cnn_grid(n), n / 4));
  conv3x3_wgrad_kernel<CIN, COUT><<<grid, kCnnThreads, smem, st>>>(n, a, dz, part);
  constexpr int len = COUT * CIN * 9 + COUT;  // W then b, as in the flat parameter vector
  reduce_partials<<<(len + 255) / 256, 256, 0, st>>>(part, grid, len, grad_w);
  (void)grad_b;  // the biases follow their weights in the flat vector
  return cudaGetLastError();
}

// Interpolated LS channel at every symbol (DMRS symbols included): H[cell][t][k][r][l].
__global__ void interp_all_kernel(Geo g, const phy_c32* __restrict__ anchors,
                                  phy_c32* __restrict__ H) {
  const int nl = g.n_layers, nr = g.n_rx;
  const long long total = (long long)g.n_cells * g.n_sym * g.n_sc * nr * nl;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(i % nl);
    long long q = i / nl;
    const int r = (int)(q % nr);
    q /= nr;
    const int k = (int)(q % g.n_sc);
    q /= g.n_sc;
    const int t = (int)(q % g.n_sym), cell = (int)(q / g.n_sym);
    const int j = seg_of(g, k), j1 = seg_g1(g, j);
    const float b = seg_beta(g, j, k, l & 1);
    float a = 0.f;  // weight of the second DMRS symbol
    if (g.n_dmrs == 2)
      a = fminf(fmaxf((float)(t - g.dmrs0) / (float)(g.dmrs1 - g.dmrs0), 0.f), 1.f);
    cf h = mk(0.f, 0.f);
    for (int d = 0; d < g.n_dmrs; ++d) {
      const phy_c32* A = anchors + ((size_t)(cell * g.n_dmrs + d) * g.G) * nl * nr;
      const cf h0 = ld(A + ((size_t)j * nl + l) * nr + r);
      const cf h1 = ld(A + ((size_t)j1 * nl + l) * nr + r);
      const cf hf = (1.f - b) * h0 + b * h1;
      h = h + (d == 0 ? (g.n_dmrs == 2 ? 1.f - a : 1.f) : a) * hf;
    }
    st(H + i, h);
  }
}

// Tiles [tile][2][14][12] from H[cell][t][k][r][l], tile = ((cell n_prb + prb) n_rx + r) nl + l.
__global__ void tiles_from_h_kernel(Geo g, const phy_c32* __restrict__ H,
                                    float* __restrict__ tiles) {
  const int nl = g.n_layers, nr = g.n_rx, n_prb = g.n_sc / 12;
  const long long total = (long long)g.n_cells * n_prb * nr * nl * kTP;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i % kTP);
    const long long tile = i / kTP;
    const int l = (int)(tile % nl);
    long long q = tile / nl;
    const int r = (int)(q % nr);
    q /= nr;
    const int prb = (int)(q % n_prb), cell = (int)(q / n_prb);
    const int t = p / kTC, k = 12 * prb + p % kTC;
    const cf h = ld(H + ((((size_t)cell * g.n_sym + t) * g.n_sc + k) * nr + r) * nl + l);
    tiles[tile * 2 * kTP + p] = h.x;
    tiles[tile * 2 * kTP + kTP + p] = h.y;
  }
}

// Data symbols of the tiles into Hd[cell][dsym][k][r][l] (the explicit-channel detector's input).
__global__ void tiles_to_h_kernel(Geo g, const float* __restrict__ tiles,
                                  phy_c32* __restrict__ Hd) {
  const int nl = g.n_layers, nr = g.n_rx, n_prb = g.n_sc / 12;
  const long long total = (long long)g.n_cells * g.n_dsym * g.n_sc * nr * nl;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(i % nl);
    long long q = i / nl;
    const int r = (int)(q % nr);
    q /= nr;
    const int k = (int)(q % g.n_sc);
    q /= g.n_sc;
    const int jj = (int)(q % g.n_dsym), cell = (int)(q / g.n_dsym);
    const long long tile = (((long long)cell * n_prb + k / 12) * nr + r) * nl + l;
    const int p = g.dsym[jj] * kTC + k % 12;
    st(Hd + i, mk(tiles[tile * 2 * kTP + p], tiles[tile * 2 * kTP + kTP + p]));
  }
}

int elementwise_grid(long long total) {
  return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 65535LL * 8));
}

}  // namespace

int cnn_param_count() { return kParams; }

cudaError_t launch_interp_all(const Geo& g, const phy_c32* anchors, phy_c32* H,
                              cudaStream_t st) {
  const long long total = (long long)g.n_cells * g.n_sym * g.n_sc * g.n_rx * g.n_layers;
  interp_all_kernel<<<elementwise_grid(total), 256, 0, st>>>(g, anchors, H);
  return cudaGetLastError();
}

cudaError_t launch_tiles_from_h(const Geo& g, const phy_c32* H, float* tiles, cudaStream_t st) {
  const long long total = (long long)g.n_cells * (g.n_sc / 12) * g.n_rx * g.n_layers * kTP;
  tiles_from_h_kernel<<<elementwise_grid(total), 256, 0, st>>>(g, H, tiles);
  return cudaGetLastError();
}

cudaError_t launch_tiles_to_h(const Geo& g, const float* tiles, phy_c32* Hd, cudaStream_t st) {
  const long long total = (long long)g.n_cells * g.n_dsym * g.n_sc * g.n_rx * g.n_layers;
  tiles_to_h_kernel<<<elementwise_grid(total), 256, 0, st>>>(g, tiles, Hd);
  return cudaGetLastError();
}

// Scratch floats for n tiles: activations a1..a3, output, dout, two dz buffers, the gradient
// partials of the persistent CTAs and the loss partials.
size_t cnn_scratch_floats(int n) {
  const size_t big = (size_t)n * 32 * kTP, small = (size_t)n * 2 * kTP;
  return 3 * big + 2 * small + 2 * big + kPartFloats + 1024 + 64;  // + the error word's block
}

size_t cnn_train_error_float(int n) { return cnn_scratch_floats(n) - 64; }

cudaError_t cnn_forward(int n, const float* P, const float* x, float* out, float* ws,
                        cudaStream_t st) {
  const size_t big = (size_t)n * 32 * kTP;
  float *a1 = ws, *a2 = a1 + big, *a3 = a2 + big;
  cudaError_t e;
  if ((e = conv<2, 32, kRelu, false>(n, x, P + kOffW1, P + kOffB1, nullptr, a1, st))) return e;
  if ((e = conv<32, 32, kRelu, false>(n, a1, P + kOffW2, P + kOffB2, nullptr, a2, st))) return e;
  if ((e = conv<32, 32, kRelu, false>(n, a2, P + kOffW3, P + kOffB3, nullptr, a3, st))) return e;
  return conv<32, 2, kResid, false>(n, a3, P + kOffW4, P + kOffB4, x, out, st);
}

cudaError_t cnn_train_step(int n, float* P, float* m, float* v, int step, float lr,
                           const float* x, const float* label, float* grad_out, float* dx_out,
                           float* loss_out, float* ws, cudaStream_t st, bool tc_forward) {
  const size_t big = (size_t)n * 32 * kTP, small = (size_t)n * 2 * kTP;
  float *a1 = ws, *a2 = a1 + big, *a3 = a2 + big;
  float* out = a3 + big;
  float* dout = out + small;
  float *dzA = dout + small, *dzB = dzA + big;
  float* part = dzB + big;
  float* lpart = part + kPartFloats;
  float* g = grad_out;
  // forward: FP32 on the CUDA cores, or BF16 operands on the tensor cores (the activations it
  // keeps are the BF16 values the next layer read; the backward pass stays FP32 on the FP32
  // master weights)
  cudaError_t e =
      tc_forward ? cnn_forward_tc(n, P, x, out,
                                  reinterpret_cast<unsigned*>(ws + cnn_train_error_float(n)), st,
                                  a1)
                 : cnn_forward(n, P, x, out, ws, st);
  if (e) return e;
  const long long total = (long long)small;
  const int lg = (int)std::min<long long>(1024, (total + kCnnThreads - 1) / kCnnThreads);
  loss_grad_kernel<<<lg, kCnnThreads, 0, st>>>(total, 1.f / ((float)n * kTP), out, label, dout,
                                               lpart);
  if (loss_out) reduce_partials<<<1, 32, 0, st>>>(lpart, lg, 1, loss_out);
  // layer 4, then back through the ReLUs
  if ((e = wgrad<32, 2>(n, a3, dout, part, g + kOffW4, g + kOffB4, st))) return e;
  if ((e = conv<2, 32, kMask, true>(n, dout, P + kOffW4, nullptr, a3, dzA, st))) return e;
  if ((e = wgrad<32, 32>(n, a2, dzA, part, g + kOffW3, g + kOffB3, st))) return e;
  if ((e = conv<32, 32, kMask, true>(n, dzA, P + kOffW3, nullptr, a2, dzB, st))) return e;
  if ((e = wgrad<32, 32>(n, a1, dzB, part, g + kOffW2, g + kOffB2, st))) return e;
  if ((e = conv<32, 32, kMask, true>(n, dzB, P + kOffW2, nullptr, a1, dzA, st))) return e;
  if ((e = wgrad<2, 32>(n, x, dzA, part, g + kOffW1, g + kOffB1, st))) return e;
  if (dx_out) {  // d loss / d x: through the first layer, plus the residual path
    if ((e = conv<32, 2, kResid, true>(n, dzA, P + kOffW1, nullptr, dout, dx_out, st))) return e;
  }
  if (step > 0) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, step)));
    adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(kParams, P, g, m, v, lr, b1, b2, eps, c1,
                                                       c2);
  }
  return cudaGetLastError();
}

}  // namespace phy
