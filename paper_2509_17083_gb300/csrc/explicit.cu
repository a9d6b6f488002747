// Ablation paths of Tab. 5: explicit-only aggregation ("w/o Neural": Eq. 7
// with the neural terms removed, i.e. isotropic, diffuse 3DGS Gaussians) and
// compositing without the neural background ("w/o Background": C = C_fg).
#include "common.cuh"

namespace hyrf {

__global__ void __launch_bounds__(256) k_query_explicit(hyrf_query_fields_args a) {
  const int nv = min(*a.n_vis, a.n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int g = a.vis_ids[i];
    if (g < 0 || g >= a.n) {
      set_status(a.status, HYRF_ERR_BOUNDS);
      continue;
    }
    a.alpha[i] = sigmoidf_(a.alpha_e ? a.alpha_e[g] : 0.0f);
    const float s = sigmoidf_(a.scale_e ? a.scale_e[g] : 0.0f);
#pragma unroll
    for (int k = 0; k < 3; ++k) a.scale[3 * i + k] = s;
    a.quat[4 * i] = 1.0f;
    a.quat[4 * i + 1] = a.quat[4 * i + 2] = a.quat[4 * i + 3] = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) a.color[3 * i + k] = sigmoidf_(a.color_e ? a.color_e[3 * (int64_t)g + k] : 0.0f);
  }
}

__global__ void __launch_bounds__(256) k_query_explicit_bwd(hyrf_query_fields_backward_args a) {
  const int nv = min(*a.n_vis, a.n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int g = a.vis_ids[i];
    if (g < 0 || g >= a.n) {
      set_status(a.status, HYRF_ERR_BOUNDS);
      continue;
    }
    if (a.d_alpha_e) {
      const float al = sigmoidf_(a.alpha_e ? a.alpha_e[g] : 0.0f);
      a.d_alpha_e[g] += a.d_alpha[i] * al * (1.0f - al);
    }
    if (a.d_scale_e) {
      const float s = sigmoidf_(a.scale_e ? a.scale_e[g] : 0.0f);
      a.d_scale_e[g] += (a.d_scale[3 * i] + a.d_scale[3 * i + 1] + a.d_scale[3 * i + 2]) * s * (1.0f - s);
    }
    if (a.d_color_e) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float c = sigmoidf_(a.color_e ? a.color_e[3 * (int64_t)g + k] : 0.0f);
        a.d_color_e[3 * (int64_t)g + k] += a.d_color[3 * i + k] * c * (1.0f - c);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_bg_none(int64_t m, const float* __restrict__ C_fg, float* __restrict__ C) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    C[i] = C_fg[i];
}

__global__ void __launch_bounds__(256) k_bg_none_bwd(int64_t P, const float* __restrict__ dC,
                                                     float* __restrict__ dC_fg, float* __restrict__ dT) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    if (dT) dT[i] = 0.0f;
    if (dC_fg) {
#pragma unroll
      for (int k = 0; k < 3; ++k) dC_fg[3 * i + k] = dC[3 * i + k];
    }
  }
}

static int grid_for(int n) {
  int b = (n + 255) / 256;
  const int cap = num_sms() * 8;
  return b < 1 ? 1 : (b > cap ? cap : b);
}

hyrf_status launch_query_explicit(const hyrf_query_fields_args& a, cudaStream_t s) {
  if (a.n == 0) return HYRF_OK;
  HYRF_LAUNCH("k_query_explicit", s, k_query_explicit<<<grid_for(a.n), 256, 0, s>>>(a));
  return HYRF_OK;
}

hyrf_status launch_query_explicit_bwd(const hyrf_query_fields_backward_args& a, cudaStream_t s) {
  if (a.n == 0) return HYRF_OK;
  HYRF_LAUNCH("k_query_explicit_bwd", s, k_query_explicit_bwd<<<grid_for(a.n), 256, 0, s>>>(a));
  return HYRF_OK;
}

hyrf_status launch_bg_none(const hyrf_composite_background_args& a, cudaStream_t s) {
  const int64_t P = (int64_t)a.cam.width * a.cam.height;
  HYRF_LAUNCH("k_bg_none", s, k_bg_none<<<grid_for((int)((3 * P + 3) / 4)), 256, 0, s>>>(3 * P, a.C_fg, a.C));
  return HYRF_OK;
}

hyrf_status launch_bg_none_bwd(const hyrf_composite_background_backward_args& b, cudaStream_t s) {
  const int64_t P = (int64_t)b.fwd.cam.width * b.fwd.cam.height;
  HYRF_LAUNCH("k_bg_none_bwd", s, k_bg_none_bwd<<<grid_for((int)P), 256, 0, s>>>(P, b.d_C, b.d_C_fg, b.d_T_final));
  return HYRF_OK;
}

}  // namespace hyrf
