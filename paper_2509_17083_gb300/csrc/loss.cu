// Training loss of Sec. 3.4 (Eq. 12): L = (1 - lambda) mean|C - target|
// + lambda (1 - SSIM(C, target)), SSIM with an 11x11 Gaussian window
// (sigma 1.5, zero padding) per channel, mean over pixels and channels,
// and its gradient dL/dC in the same pass.
#include <cmath>

#include "common.cuh"

namespace hyrf {

__constant__ float c_win[11];

__device__ __forceinline__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.0f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(256) k_l1(const float* __restrict__ C, const float* __restrict__ tgt,
                                            int64_t n, float w_l1, float gscale,
                                            float* __restrict__ loss, float* __restrict__ dC) {
  __shared__ float red[8];
  float acc = 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = C[e] - tgt[e];
    acc += fabsf(d);
    if (dC) dC[e] = gscale * w_l1 * (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f)) / (float)n;
  }
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(loss, w_l1 * s / (float)n);
}

// Per pixel and channel: SSIM map value and its partial derivatives w.r.t.
// the windowed mean of C, the windowed second moment of C and the windowed
// cross moment.
__global__ void __launch_bounds__(256) k_ssim_maps(const float* __restrict__ X, const float* __restrict__ Y,
                                                   int W, int H, float lam, float* __restrict__ loss,
                                                   float* __restrict__ dmu, float* __restrict__ dsxx,
                                                   float* __restrict__ dsxy) {
  __shared__ float red[8];
  const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
  const int64_t n = (int64_t)W * H * 3;
  float acc = 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(e % 3);
    const int64_t pix = e / 3;
    const int px = (int)(pix % W), py = (int)(pix / W);
    float mx = 0, my = 0, sxx = 0, syy = 0, sxy = 0;
    for (int dy = -5; dy <= 5; ++dy) {
      const int qy = py + dy;
      if (qy < 0 || qy >= H) continue;
      for (int dx = -5; dx <= 5; ++dx) {
        const int qx = px + dx;
        if (qx < 0 || qx >= W) continue;
        const float w = c_win[dy + 5] * c_win[dx + 5];
        const int64_t q = ((int64_t)qy * W + qx) * 3 + ch;
        const float a = X[q], b = Y[q];
        mx += w * a;
        my += w * b;
        sxx += w * a * a;
        syy += w * b * b;
        sxy += w * a * b;
      }
    }
    const float vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
    const float A1 = 2.f * mx * my + C1, A2 = 2.f * cxy + C2;
    const float B1 = mx * mx + my * my + C1, B2 = vx + vy + C2;
    const float S = (A1 * A2) / (B1 * B2);
    acc += S;
    dmu[e] = S * (2.f * my / A1 - 2.f * my / A2 - 2.f * mx / B1 + 2.f * mx / B2);
    dsxx[e] = -S / B2;
    dsxy[e] = 2.f * S / A2;
  }
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(loss, lam * (1.0f / (float)gridDim.x - s / (float)n));
}

__global__ void __launch_bounds__(256) k_ssim_grad(const float* __restrict__ X, const float* __restrict__ Y,
                                                   int W, int H, float scale,
                                                   const float* __restrict__ dmu,
                                                   const float* __restrict__ dsxx,
                                                   const float* __restrict__ dsxy,
                                                   float* __restrict__ dC) {
  const int64_t n = (int64_t)W * H * 3;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(e % 3);
    const int64_t pix = e / 3;
    const int qx = (int)(pix % W), qy = (int)(pix / W);
    const float a = X[e], b = Y[e];
    float acc = 0.0f;
    for (int dy = -5; dy <= 5; ++dy) {
      const int py = qy + dy;
      if (py < 0 || py >= H) continue;
      for (int dx = -5; dx <= 5; ++dx) {
        const int px = qx + dx;
        if (px < 0 || px >= W) continue;
        const float w = c_win[dy + 5] * c_win[dx + 5];
        const int64_t p = ((int64_t)py * W + px) * 3 + ch;
        acc += w * (dmu[p] + 2.f * a * dsxx[p] + b * dsxy[p]);
      }
    }
    dC[e] += scale * acc;
  }
}

size_t loss_workspace(const hyrf_loss_args& a) {
  if (a.lambda == 0.0f) return 0;
  Carver c(nullptr);
  for (int k = 0; k < 3; ++k) c.take<float>((size_t)a.width * a.height * 3);
  return c.size();
}

static bool g_win_ready = false;

hyrf_status launch_loss(const hyrf_loss_args& a, void* ws, cudaStream_t s) {
  if (!g_win_ready) {
    float w[11];
    double t = 0;
    for (int i = 0; i < 11; ++i) t += std::exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
    for (int i = 0; i < 11; ++i) w[i] = (float)(std::exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)) / t);
    if (cudaMemcpyToSymbol(c_win, w, sizeof(w)) != cudaSuccess) return HYRF_ERR_CUDA;
    g_win_ready = true;
  }
  const int64_t n = (int64_t)a.width * a.height * 3;
  cudaMemsetAsync(a.loss, 0, sizeof(float), s);
  int blocks = (int)((n + 255) / 256);
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  if (blocks < 1) blocks = 1;
  HYRF_LAUNCH("k_l1", s,
              k_l1<<<blocks, 256, 0, s>>>(a.C, a.target, n, 1.0f - a.lambda, a.grad_scale, a.loss, a.d_C));
  if (a.lambda != 0.0f) {
    Carver c(ws);
    float* dmu = c.take<float>(n);
    float* dsxx = c.take<float>(n);
    float* dsxy = c.take<float>(n);
    HYRF_LAUNCH("k_ssim_maps", s,
                k_ssim_maps<<<blocks, 256, 0, s>>>(a.C, a.target, a.width, a.height, a.lambda, a.loss, dmu, dsxx,
                                       dsxy));
    if (a.d_C) {
      HYRF_LAUNCH("k_ssim_grad", s,
                  k_ssim_grad<<<blocks, 256, 0, s>>>(a.C, a.target, a.width, a.height,
                                         -a.lambda * a.grad_scale / (float)n, dmu, dsxx, dsxy, a.d_C));
    }
  }
  return HYRF_OK;
}

}  // namespace hyrf
