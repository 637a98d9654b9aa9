// noalloc.cu -- gpma_export_sorted_noalloc: the sorted-edge export with its
// look-back scratch in a fixed, file-scope device array, so the call itself
// allocates no device memory.  The paper has no counterpart: this serves callers
// that must not allocate device memory when they query the graph.
#include <mutex>

#include "gpma.h"
#include "gpma_launch.h"

namespace {

// Look-back status words of the single-pass compaction: one per tile of 2,048
// slots (the export scans one column), plus a margin.  Sized for arrays of up
// to 2^27 slots (about 512 KiB, held by every GPU that loads the library until
// the process exits).
constexpr uint64_t kMaxSlots = 1ull << 27;
constexpr uint64_t kStatusWords = kMaxSlots / 2048 + 64;
static __device__ __align__(256) uint64_t g_export_status[kStatusWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
uint64_t *g_status_addr[kMaxDevices] = {};

// Device address of g_export_status on the current device, looked up once per
// device (the host-side name of the array is not a device address).
int status_address(uint64_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GPMA_EDEVICE;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_status_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_export_status) != cudaSuccess || !p) {
      cudaGetLastError();
      return GPMA_EDEVICE;
    }
    g_status_addr[dev] = static_cast<uint64_t *>(p);
  }
  *out = g_status_addr[dev];
  return GPMA_OK;
}

}  // namespace

extern "C" int gpma_export_sorted_noalloc(gpma_t h, uint64_t *d_out, uint64_t cap, uint64_t *n_out,
                                          void *stream) {
  if (!h || !n_out || (cap && !d_out)) return GPMA_EINVAL;
  const gpk::HandleView v = gpk::handle_view(h, (cudaStream_t)stream);
  if (v.poisoned) return v.poisoned;
  if (v.geo->C > kMaxSlots) return GPMA_EINVAL;  // larger than the fixed scratch
  uint64_t *status = nullptr;
  int rc = status_address(&status);
  if (rc) return gpk::poison_handle(h, rc);
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's words (maybe another handle's): clear
  // the part this call uses so no stale word can pass for this call's
  const uint64_t words = (uint64_t)gpk::comp_tiles(v.geo->C) + 64;
  if (cudaMemsetAsync(status, 0, words * sizeof(uint64_t), s) != cudaSuccess) {
    cudaGetLastError();
    return gpk::poison_handle(h, GPMA_EDEVICE);
  }
  gpk::launch_export(*v.geo, v.ctl, d_out, nullptr, cap, status, s);
  if (cudaMemcpyAsync(v.h_ctl, v.ctl, sizeof(gpk::Ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return gpk::poison_handle(h, GPMA_EDEVICE);
  }
  // a look-back wait that gave up leaves the count and keys wrong
  if ((rc = gpk::export_status(h, v.h_ctl->err))) return rc;
  *n_out = v.h_ctl->gen_count;
  return *n_out > cap ? GPMA_ECAP : GPMA_OK;
}
