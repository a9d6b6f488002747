// Internal definitions shared by the libhyrf translation units.
#pragma once
#include <atomic>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hyrf.h"

namespace hyrf {

constexpr int kTile = 16;        // tile edge (pixels); one CTA of 256 threads per tile
constexpr int kMaxLevels = 16;   // hash-grid levels supported by the kernels
constexpr int kPEPad = 32;       // width of the positional-encoding block of the colour input

// ---------------------------------------------------------------- device params

// One hash grid as the kernels see it (built on the host from hyrf_grid).
struct GridDev {
  const void* table;   // [L][T][2] float, bf16 or uint8 codes
  uint32_t T;          // entries per level (power of two)
  uint32_t mask;       // T - 1
  uint32_t dense;      // bit l: level l is stored densely
  int L;
  int bf16;
  int f16;
  int u8;              // uint8 codes with per-level (lo, step) in q
  int log2T;
  const float* q;
  int res[kMaxLevels]; // level resolution floor(base * growth^l)
};

// One decoder. Weights [out][in] row-major (float or bf16), biases float.
struct MlpDev {
  const void* W[3];
  const float* b[3];
  int n_in, width, n_hidden, n_out;
  int bf16;            // 16-bit weights: bf16, or f16 when f16 is set (render only)
  int f16;
};

struct FieldsDev {
  float lo[3], sx[3];  // App. A.1 normalisation x = (p - lo) * sx - 1, sx = 2 / (hi - lo)
  GridDev geo, rad;
  MlpDev gm, cm;
  int pe_freq, pe_pad;
};

struct CamDev {
  float R[9], t[3];
  float fx, fy, cx, cy;
  int W, H;
  float z_near, tol;
};

inline CamDev to_dev(const hyrf_camera& c) {
  CamDev d;
  for (int i = 0; i < 9; ++i) d.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) d.t[i] = c.t[i];
  d.fx = c.fx;
  d.fy = c.fy;
  d.cx = c.cx;
  d.cy = c.cy;
  d.W = c.width;
  d.H = c.height;
  d.z_near = c.z_near;
  d.tol = c.cull_tol;
  return d;
}

__device__ __forceinline__ void set_status(int32_t* st, int flag) {
  if (st) atomicOr(st, flag);
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// ---------------------------------------------------------------- host helpers

// Launch accounting (host counter, read by hyrf_launch_count).
void count_launch(int n = 1);

// Convert the public field description into device params; false if unsupported.
bool make_fields(const hyrf_fields& f, FieldsDev& d, bool need_geo);

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Carve sub-buffers out of a caller workspace.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* p) : base(static_cast<char*>(p)) {}
  template <class T>
  T* take(size_t count) {
    off = align_up(off);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t size() const { return align_up(off); }
};

int num_sms();

// Order `after` behind the work issued so far on `before` (an event from a
// small library pool, recorded on `before`, waited on by `after`); works
// during CUDA graph capture, where it forks `after` into the graph.
hyrf_status fork_stream(cudaStream_t before, cudaStream_t after);

// Raise a kernel's dynamic shared-memory limit once per device: the
// attribute persists, so later calls (for instance during CUDA graph
// capture) make no API call.
template <auto Kern>
inline void set_smem_limit(int bytes) {
  static std::atomic<uint64_t> done{0};  // bit d: set on device d
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  done.fetch_or(bit, std::memory_order_release);
}

// Records a CUDA event pair on `s` around the launches in its scope while the
// kernel timer is enabled (hyrf_timer_enable); otherwise does nothing.
class KernelTimer {
 public:
  KernelTimer(const char* name, cudaStream_t s);
  ~KernelTimer();
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

}  // namespace hyrf

#define HYRF_LAUNCH_CHECK()                                 \
  do {                                                      \
    ::hyrf::count_launch();                                 \
    if (cudaPeekAtLastError() != cudaSuccess) {             \
      cudaGetLastError();                                   \
      return HYRF_ERR_CUDA;                                 \
    }                                                       \
  } while (0)

// One kernel launch (the variadic tail, so the launch may hold commas):
// optionally timed under `name`, counted and checked.
#define HYRF_LAUNCH(name, stream, ...)                      \
  do {                                                      \
    {                                                       \
      ::hyrf::KernelTimer hyrf_kt_(name, stream);           \
      __VA_ARGS__;                                          \
    }                                                       \
    HYRF_LAUNCH_CHECK();                                    \
  } while (0)
