// Adaptive density control (hyrf_densify_stats / _plan / _apply; see
// hyrf.h): the view-space gradient statistics, the per-Gaussian decision
// (keep / prune / clone / split) with the exclusive scan of the output
// multiplicities, and the rewrite of every per-Gaussian array.
//
// The statistics and the decision are computed with explicit round-to-
// nearest float operations (no contraction), so a float replay of the same
// operations reproduces them bit for bit.
#include "common.cuh"

namespace hyrf {
namespace {

constexpr int kChunk = 2048;  // elements per scan CTA (256 threads x 8)

__global__ void __launch_bounds__(256) k_dens_stats(hyrf_densify_stats_args a) {
  const int nv = min(*a.n_vis, a.n);
  const float hw = 0.5f * (float)a.width, hh = 0.5f * (float)a.height;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    if (a.ntiles[i] <= 0) continue;
    const int g = a.vis_ids[i];
    if (g < 0 || g >= a.n) continue;
    const float gx = __fmul_rn(a.d_mean2d[2 * i], hw), gy = __fmul_rn(a.d_mean2d[2 * i + 1], hh);
    const float norm = sqrtf(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
    a.accum[g] = __fadd_rn(a.accum[g], norm);
    a.count[g] += 1;
  }
}

__global__ void __launch_bounds__(256) k_dens_rows(const int32_t* __restrict__ vis_ids,
                                                   const int32_t* __restrict__ n_vis, int n,
                                                   int32_t* __restrict__ row) {
  const int nv = min(*n_vis, n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int g = vis_ids[i];
    if (g >= 0 && g < n) row[g] = i;
  }
}

__device__ __forceinline__ int dens_action(const hyrf_densify_plan_args& a, int g) {
  const int r = a.row[g];
  if (r < 0) return HYRF_DENSIFY_KEEP;
  if (a.alpha[r] < a.min_opacity) return HYRF_DENSIFY_PRUNE;
  const int c = a.count[g];
  if (c <= 0 || __fdiv_rn(a.accum[g], (float)c) < a.grad_threshold) return HYRF_DENSIFY_KEEP;
  const float s = fmaxf(fmaxf(a.scale[3 * r], a.scale[3 * r + 1]), a.scale[3 * r + 2]);
  return s > a.dense_scale ? HYRF_DENSIFY_SPLIT : HYRF_DENSIFY_CLONE;
}

__device__ __forceinline__ int multiplicity(int act) { return act == HYRF_DENSIFY_PRUNE ? 0 : (act == HYRF_DENSIFY_KEEP ? 1 : 2); }

// Pass 1: actions and the per-chunk sums of the multiplicities.
__global__ void __launch_bounds__(256) k_dens_plan(hyrf_densify_plan_args a, int64_t* __restrict__ sums) {
  __shared__ int64_t red[8];
  const int64_t start = (int64_t)blockIdx.x * kChunk;
  int64_t s = 0;
  for (int k = 0; k < kChunk / 256; ++k) {
    const int64_t g = start + k * 256 + threadIdx.x;
    if (g < a.n) {
      const int act = dens_action(a, (int)g);
      a.action[g] = (uint8_t)act;
      s += multiplicity(act);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    sums[blockIdx.x] = t;
  }
}

// Pass 2 (one CTA): exclusive scan of the chunk sums; total to *n_out.
__global__ void __launch_bounds__(1024) k_dens_scan(int64_t* __restrict__ sums, int m, int64_t* __restrict__ n_out) {
  __shared__ int64_t ws[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < m; base += 1024) {
    const int i = base + threadIdx.x;
    const int64_t v = i < m ? sums[i] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      int64_t t = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      ws[lane] = t;
    }
    __syncthreads();
    const int64_t incl = x + (w > 0 ? ws[w - 1] : 0) + carry;
    if (i < m) sums[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_out = carry;
}

// Pass 3: per-Gaussian exclusive offsets; offset[n] = total.
__global__ void __launch_bounds__(256) k_dens_offsets(const uint8_t* __restrict__ action, int n,
                                                      const int64_t* __restrict__ sums, int m,
                                                      int64_t* __restrict__ offset) {
  __shared__ int64_t ws[8];
  const int64_t start = (int64_t)blockIdx.x * kChunk;
  int64_t run = sums[blockIdx.x];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int k = 0; k < kChunk / 256; ++k) {
    const int64_t g = start + k * 256 + t;
    const int c = g < n ? multiplicity(action[g]) : 0;
    int64_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int64_t before = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      before += q < w ? ws[q] : 0;
      tot += ws[q];
    }
    if (g < n) offset[g] = run + before + x - c;
    run += tot;
    __syncthreads();
  }
  if (blockIdx.x == m - 1 && t == 0) offset[n] = run;
}

// One thread per old Gaussian: its 0, 1 or 2 output rows in every array.
__global__ void __launch_bounds__(256) k_dens_apply(const hyrf_densify_apply_args a) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n; g += gridDim.x * blockDim.x) {
    const int act = a.action[g];
    if (act == HYRF_DENSIFY_PRUNE) continue;
    const int64_t o = a.offset[g];
    float sample[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    const bool split = act == HYRF_DENSIFY_SPLIT && a.row[g] >= 0 && a.scale && a.quat && a.noise;
    if (split) {
      const int r = a.row[g];
      const float w = a.quat[4 * r], x = a.quat[4 * r + 1], y = a.quat[4 * r + 2], z = a.quat[4 * r + 3];
      const float R[9] = {1.0f - 2.0f * (y * y + z * z), 2.0f * (x * y - w * z), 2.0f * (x * z + w * y),
                          2.0f * (x * y + w * z), 1.0f - 2.0f * (x * x + z * z), 2.0f * (y * z - w * x),
                          2.0f * (x * z - w * y), 2.0f * (y * z + w * x), 1.0f - 2.0f * (x * x + y * y)};
      for (int k = 0; k < 2; ++k) {
        float u[3];
        for (int j = 0; j < 3; ++j) u[j] = a.scale[3 * r + j] * a.noise[6 * (int64_t)g + 3 * k + j];
        for (int i = 0; i < 3; ++i) sample[k][i] = R[3 * i] * u[0] + R[3 * i + 1] * u[1] + R[3 * i + 2] * u[2];
      }
    }
    for (int j = 0; j < a.n_arrays; ++j) {
      const hyrf_remap_array& A = a.arrays[j];
      const float* src = A.src + (int64_t)g * A.width;
      float* d0 = A.dst + o * A.width;
      if (act == HYRF_DENSIFY_KEEP) {
        for (int c = 0; c < A.width; ++c) d0[c] = src[c];
        continue;
      }
      float* d1 = d0 + A.width;
      for (int c = 0; c < A.width; ++c) {
        const float v = src[c];
        if (act == HYRF_DENSIFY_CLONE || !split) {  // clone (a split without its row clones)
          d0[c] = v;
          d1[c] = A.kind == HYRF_REMAP_STATE ? 0.0f : v;
        } else if (A.kind == HYRF_REMAP_STATE) {
          d0[c] = d1[c] = 0.0f;
        } else if (A.kind == HYRF_REMAP_POSITION) {
          d0[c] = v + sample[0][c];
          d1[c] = v + sample[1][c];
        } else if (A.kind == HYRF_REMAP_SCALE_LOGIT) {
          d0[c] = d1[c] = v - a.split_log_scale;
        } else {
          d0[c] = d1[c] = v;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_reset_opacity(float* __restrict__ a, int64_t n, float vmax,
                                                       float* __restrict__ m, float* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a[i] = fminf(a[i], vmax);
    if (m) m[i] = 0.0f;
    if (v) v[i] = 0.0f;
  }
}

int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace
}  // namespace hyrf

using namespace hyrf;

extern "C" {

hyrf_status hyrf_densify_stats(const hyrf_densify_stats_args* a, void* stream) {
  if (!a || a->n < 0 || a->width <= 0 || a->height <= 0) return HYRF_ERR_INVALID_ARG;
  if (a->n == 0) return HYRF_OK;
  if (!a->vis_ids || !a->n_vis || !a->d_mean2d || !a->ntiles || !a->accum || !a->count)
    return HYRF_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HYRF_LAUNCH("k_dens_stats", s, k_dens_stats<<<grid_of(a->n), 256, 0, s>>>(*a));
  return HYRF_OK;
}

size_t hyrf_densify_plan_workspace_size(const hyrf_densify_plan_args* a) {
  if (!a || a->n < 0) return 0;
  return align_up(((size_t)a->n + kChunk - 1) / kChunk * sizeof(int64_t) + sizeof(int64_t));
}

hyrf_status hyrf_densify_plan(const hyrf_densify_plan_args* a, void* ws, size_t ws_bytes, void* stream) {
  if (!a || a->n < 0 || !a->offset || !a->n_out) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->vis_ids || !a->n_vis || !a->alpha || !a->scale || !a->accum || !a->count ||
                   !a->action || !a->row))
    return HYRF_ERR_INVALID_ARG;
  const size_t need = hyrf_densify_plan_workspace_size(a);
  if (ws_bytes < need || !ws) return HYRF_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (a->n == 0) {
    cudaMemsetAsync(a->offset, 0, sizeof(int64_t), s);
    cudaMemsetAsync(a->n_out, 0, sizeof(int64_t), s);
    return cudaPeekAtLastError() == cudaSuccess ? HYRF_OK : HYRF_ERR_CUDA;
  }
  int64_t* sums = static_cast<int64_t*>(ws);
  const int m = (a->n + kChunk - 1) / kChunk;
  cudaMemsetAsync(a->row, 0xff, (size_t)a->n * sizeof(int32_t), s);  // -1: not visible
  HYRF_LAUNCH("k_dens_rows", s, k_dens_rows<<<grid_of(a->n), 256, 0, s>>>(a->vis_ids, a->n_vis, a->n, a->row));
  HYRF_LAUNCH("k_dens_plan", s, k_dens_plan<<<m, 256, 0, s>>>(*a, sums));
  HYRF_LAUNCH("k_dens_scan", s, k_dens_scan<<<1, 1024, 0, s>>>(sums, m, a->n_out));
  HYRF_LAUNCH("k_dens_offsets", s, k_dens_offsets<<<m, 256, 0, s>>>(a->action, a->n, sums, m, a->offset));
  return HYRF_OK;
}

hyrf_status hyrf_reset_opacity(float* alpha_e, int64_t n, float max_logit, float* m, float* v, void* stream) {
  if (n < 0 || (n > 0 && !alpha_e)) return HYRF_ERR_INVALID_ARG;
  if (n == 0) return HYRF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HYRF_LAUNCH("k_reset_opacity", s, k_reset_opacity<<<grid_of(n), 256, 0, s>>>(alpha_e, n, max_logit, m, v));
  return HYRF_OK;
}

hyrf_status hyrf_densify_apply(const hyrf_densify_apply_args* a, void* stream) {
  if (!a || a->n < 0 || a->n_arrays < 0 || a->n_arrays > HYRF_REMAP_MAX) return HYRF_ERR_INVALID_ARG;
  if (a->n == 0) return HYRF_OK;
  if (!a->action || !a->row || !a->offset) return HYRF_ERR_INVALID_ARG;
  bool need_split = false;
  for (int j = 0; j < a->n_arrays; ++j) {
    const hyrf_remap_array& A = a->arrays[j];
    if (!A.src || !A.dst || A.width < 1 || A.width > 4 || A.kind < 0 || A.kind > 3) return HYRF_ERR_INVALID_ARG;
    if (A.kind == HYRF_REMAP_POSITION && A.width != 3) return HYRF_ERR_INVALID_ARG;
    if (A.kind == HYRF_REMAP_SCALE_LOGIT && A.width != 1) return HYRF_ERR_INVALID_ARG;
    need_split |= A.kind == HYRF_REMAP_POSITION;
  }
  if (need_split && (!a->scale || !a->quat || !a->noise)) return HYRF_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HYRF_LAUNCH("k_dens_apply", s, k_dens_apply<<<grid_of(a->n), 256, 0, s>>>(*a));
  return HYRF_OK;
}

}  // extern "C"
