// hyrf_bin_sort_noalloc: the binning and depth sort of hyrf_bin_sort with its
// temporary storage in a fixed device array owned by this library, for
// callers that cannot hand the library a device workspace (see hyrf.h).
#include <mutex>

#include "common.cuh"

namespace hyrf {

size_t bin_sort_workspace(int n, int64_t cap);
hyrf_status bin_sort_check(const hyrf_bin_sort_args* a);
hyrf_status launch_bin_sort(const hyrf_bin_sort_args& a, void* ws, cudaStream_t s);

// The scratch array. Every GPU that loads the library holds it until the
// process exits. In host code this name is only a stand-in for the device
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_sort_scratch[HYRF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).
hyrf_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HYRF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HYRF_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return HYRF_OK;
}
}  // namespace

}  // namespace hyrf

extern "C" hyrf_status hyrf_bin_sort_noalloc(const hyrf_bin_sort_args* a, void* stream) {
  using namespace hyrf;
  if (!a) return HYRF_ERR_INVALID_ARG;
  if (a->n > HYRF_NOALLOC_MAX_GAUSSIANS || a->capacity > HYRF_NOALLOC_MAX_INSTANCES)
    return HYRF_ERR_INVALID_ARG;
  hyrf_status st = bin_sort_check(a);  // host-side argument checks, no device work
  if (st != HYRF_OK) return st;
  if (bin_sort_workspace(a->n, a->capacity) > (size_t)HYRF_NOALLOC_SCRATCH_BYTES)
    return HYRF_ERR_INVALID_ARG;
  void* scratch = nullptr;
  st = scratch_address(&scratch);
  if (st != HYRF_OK) return st;
  // No part of the scratch is read before this call writes it, so nothing
  // is cleared here.
  return launch_bin_sort(*a, scratch, static_cast<cudaStream_t>(stream));
}
