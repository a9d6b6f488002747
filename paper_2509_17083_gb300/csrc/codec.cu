// 8-bit min-max codec of the hash tables (hyrf_quantize_grid; the grids of
// the compressed model, Sec. 4.4): per level, codes 0..255 between the
// level's minimum and maximum. Decoding happens inside the gathers
// (load_entry); this file only encodes. The range and the codes use explicit
// round-to-nearest float operations, so a float replay reproduces them.
#include <cfloat>

#include "common.cuh"

namespace hyrf {
namespace {

// dt: HYRF_F32, HYRF_BF16 or HYRF_F16
__device__ __forceinline__ float tab_value(const void* t, int dt, size_t i) {
  if (dt == HYRF_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(t)[i]);
  if (dt == HYRF_F16) return __half2float(static_cast<const __half*>(t)[i]);
  return static_cast<const float*>(t)[i];
}

// One CTA per level: minimum and maximum of its 2T values -> (lo, step).
__global__ void __launch_bounds__(1024) k_grid_range(const void* __restrict__ t, int dt, size_t per_level,
                                                     float* __restrict__ q) {
  __shared__ float smin[32], smax[32];
  const size_t base = (size_t)blockIdx.x * per_level;
  float lo = FLT_MAX, hi = -FLT_MAX;
  for (size_t i = threadIdx.x; i < per_level; i += blockDim.x) {
    const float v = tab_value(t, dt, base + i);
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    smin[threadIdx.x >> 5] = lo;
    smax[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = fminf(lo, smin[w]);
      hi = fmaxf(hi, smax[w]);
    }
    q[2 * blockIdx.x] = lo;
    q[2 * blockIdx.x + 1] = __fdiv_rn(__fsub_rn(hi, lo), 255.0f);
  }
}

__global__ void __launch_bounds__(256) k_grid_encode(const void* __restrict__ t, int dt, int log2T,
                                                     size_t total, const float* __restrict__ q,
                                                     uint8_t* __restrict__ codes) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t l = (i >> 1) >> log2T;
    const float lo = q[2 * l], step = q[2 * l + 1];
    float c = 0.0f;
    if (step > 0.0f) c = rintf(__fdiv_rn(__fsub_rn(tab_value(t, dt, i), lo), step));
    codes[i] = (uint8_t)fminf(fmaxf(c, 0.0f), 255.0f);
  }
}

}  // namespace
}  // namespace hyrf

using namespace hyrf;

extern "C" hyrf_status hyrf_quantize_grid(const void* table, int32_t dtype, int32_t n_levels, int32_t log2_T,
                                          uint8_t* codes, float* qparams, void* stream) {
  if (!table || !codes || !qparams || n_levels < 1 || n_levels > kMaxLevels || log2_T < 4 || log2_T > 26 ||
      (dtype != HYRF_F32 && dtype != HYRF_BF16 && dtype != HYRF_F16))
    return HYRF_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t per_level = (size_t)2 << log2_T;
  const int dt = dtype;
  HYRF_LAUNCH("k_grid_range", s, k_grid_range<<<n_levels, 1024, 0, s>>>(table, dt, per_level, qparams));
  const size_t total = per_level * n_levels;
  int blocks = (int)((total + 255) / 256);
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  HYRF_LAUNCH("k_grid_encode", s, k_grid_encode<<<blocks, 256, 0, s>>>(table, dt, log2_T, total, qparams, codes));
  return HYRF_OK;
}
