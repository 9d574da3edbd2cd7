// phy_slot_run_noalloc: the whole receiver with its scratch in a fixed device array.
//
// phy_slot_run keeps its scratch (the LS anchors, the noise-estimate partial sums, the error
// word and the Gram-block and matched-filter intermediates of a chunk of cells) in a
// caller-provided workspace. This variant keeps all of it in the file-scope array below
// instead, so the caller passes only inputs and outputs and nothing is allocated, ever.
#include <mutex>

#include "../../include/phy.h"
#include "launch.h"

namespace {

constexpr size_t kScratchBytes = PHY_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

}  // namespace

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device. The host-side name of the array
// is a stand-in, not a device address, so it is resolved once per device (with that device
// current) and cached for the life of the process: the cached address belongs to the device's
// primary context and is stale after cudaDeviceReset (documented in the header).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" phy_status phy_slot_run_noalloc(const phy_slot_cfg* cfg, const phy_c32* Y,
                                           const phy_c32* pilots, const float* sigma2,
                                           phy_c32* x_hat, float* sinr, float* llr,
                                           uint8_t* flags, void* stream) {
  // the work runs in chunks of cells sized to fit the array
  const size_t need = phy::min_workspace_bytes(cfg);
  if (need == 0) return PHY_ERR_INVALID_ARG;
  if (need > kScratchBytes) return PHY_ERR_NO_MEMORY;
  if (!Y || !pilots || !sigma2 || !flags) return PHY_ERR_INVALID_ARG;
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return PHY_ERR_CUDA;
  // Validation of the rest and the kernels are phy_slot_run's. Every value the kernels read from
  // the array is written earlier in the same call, so nothing needs clearing between calls.
  return phy::slot_run_fit(cfg, Y, pilots, sigma2, x_hat, sinr, llr, flags, scratch,
                           kScratchBytes, (cudaStream_t)stream);
}
