// Visibility pre-culling with ascending compaction (Sec. 3.3, Eqs. 8-9) and
// the EWA projection of the visible Gaussians (the 3DGS rasterizer of
// Sec. 3.2). This file is compiled with -fmad=false: every product and sum
// below is rounded on its own, in source order, so that visibility, tile
// rectangles and depth keys are reproducible bit for bit. The operation
// order is part of the library's contract.
#include "footprint.cuh"

namespace hyrf {

constexpr int kChunk = 1024;  // elements per pre-cull CTA (256 threads x 4)

// x_c = R p + t, each row summed left to right.
__device__ __forceinline__ void cam_point(const CamDev& c, const float p[3], float tc[3]) {
  tc[0] = c.R[0] * p[0] + c.R[1] * p[1] + c.R[2] * p[2] + c.t[0];
  tc[1] = c.R[3] * p[0] + c.R[4] * p[1] + c.R[5] * p[2] + c.t[1];
  tc[2] = c.R[6] * p[0] + c.R[7] * p[1] + c.R[8] * p[2] + c.t[2];
}

// Eq. 9 on normalised device coordinates, plus the near test z > z_near.
__device__ __forceinline__ bool visible(const CamDev& c, const float* __restrict__ pos, int64_t g) {
  float p[3] = {pos[3 * g], pos[3 * g + 1], pos[3 * g + 2]};
  float tc[3];
  cam_point(c, p, tc);
  if (!(tc[2] > c.z_near)) return false;
  float u = c.fx * tc[0] / tc[2] + c.cx;
  float v = c.fy * tc[1] / tc[2] + c.cy;
  float xn = 2.0f * u / (float)c.W - 1.0f;
  float yn = 2.0f * v / (float)c.H - 1.0f;
  float lim = 1.0f + c.tol;
  return fabsf(xn) <= lim && fabsf(yn) <= lim;
}

__global__ void __launch_bounds__(256) k_precull_count(CamDev cam, const float* __restrict__ pos,
                                                       int n, int32_t* __restrict__ counts) {
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  int c = 0;
  for (int k = 0; k < kChunk / 256; ++k) {
    int64_t g = base + k * 256 + threadIdx.x;
    if (g < n) c += visible(cam, pos, g) ? 1 : 0;
  }
  // block sum
  __shared__ int red[8];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < 8; ++w) s += red[w];
    counts[blockIdx.x] = s;
  }
}

// Exclusive scan of `m` counts by one CTA of 1024 threads; total to *total.
__global__ void __launch_bounds__(1024) k_scan_small(int32_t* __restrict__ counts, int m,
                                                     int32_t* __restrict__ total) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < m; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < m ? counts[i] : 0;
    int x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      int s = warp_sums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    int incl = x + (w > 0 ? warp_sums[w - 1] : 0) + carry;
    if (i < m) counts[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Ordered compaction: visible ids of chunk b land at offsets[b] + rank.
__global__ void __launch_bounds__(256) k_precull_scatter(CamDev cam, const float* __restrict__ pos,
                                                         int n, const int32_t* __restrict__ offsets,
                                                         int32_t* __restrict__ vis_ids) {
  __shared__ int wsum[8];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  int run = offsets[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < kChunk / 256; ++k) {
    int64_t g = base + k * 256 + threadIdx.x;
    bool f = g < n && visible(cam, pos, g);
    unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    int before = 0, tot = 0;
    for (int j = 0; j < 8; ++j) {
      before += j < w ? wsum[j] : 0;
      tot += wsum[j];
    }
    if (f) vis_ids[run + before + __popc(m & ((1u << lane) - 1u))] = (int32_t)g;
    run += tot;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- projection

struct ProjOut {
  float* mean2d;
  float* conic;
  float* depth;
  int32_t* rect;
  int32_t* ntiles;
  uint8_t* flag;
  const float* alpha;  // opacity for the footprint (NULL: 1)
  float4* foot;        // footprint records out (footprint.cuh; NULL: whole rectangles)
};

// FP64 recomputation of Sigma' and its inverse for near-singular Gaussians.
__device__ __noinline__ void conic_fp64(const CamDev& c, const float p[3], const float s[3],
                                        const float q[4], float out[3]) {
  double tc[3];
  for (int i = 0; i < 3; ++i)
    tc[i] = (double)c.R[3 * i] * p[0] + (double)c.R[3 * i + 1] * p[1] +
            (double)c.R[3 * i + 2] * p[2] + (double)c.t[i];
  const double z = tc[2];
  const double limx = 1.3 * (0.5 * c.W / (double)c.fx), limy = 1.3 * (0.5 * c.H / (double)c.fy);
  double mx = fmin(limx, fmax(-limx, tc[0] / z)), my = fmin(limy, fmax(-limy, tc[1] / z));
  const double J[6] = {c.fx / z, 0.0, -c.fx * mx / z, 0.0, c.fy / z, -c.fy * my / z};
  double T[6];
  for (int i = 0; i < 2; ++i)
    for (int k = 0; k < 3; ++k)
      T[3 * i + k] = J[3 * i] * c.R[k] + J[3 * i + 1] * c.R[3 + k] + J[3 * i + 2] * c.R[6 + k];
  const double w = q[0], x = q[1], y = q[2], zq = q[3];
  const double r[9] = {1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y),
                       2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x),
                       2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)};
  double M[9], S[9];
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) M[3 * a + k] = r[3 * a + k] * (double)s[k];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      S[3 * a + b] = M[3 * a] * M[3 * b] + M[3 * a + 1] * M[3 * b + 1] + M[3 * a + 2] * M[3 * b + 2];
  double A = 0.3, B = 0.0, C = 0.3;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A += T[i] * S[3 * i + j] * T[j];
      B += T[i] * S[3 * i + j] * T[3 + j];
      C += T[3 + i] * S[3 * i + j] * T[3 + j];
    }
  const double det = A * C - B * B;
  out[0] = (float)(C / det);
  out[1] = (float)(-B / det);
  out[2] = (float)(A / det);
}

__global__ void __launch_bounds__(256) k_project(CamDev c, int n, const float* __restrict__ pos,
                                                 const int32_t* __restrict__ vis_ids,
                                                 const int32_t* __restrict__ n_vis,
                                                 const float* __restrict__ scale,
                                                 const float* __restrict__ quat, int TX, int TY,
                                                 ProjOut o, int32_t* status) {
  const int nv = min(*n_vis, n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int g = vis_ids[i];
    if (g < 0 || g >= n) {
      set_status(status, HYRF_ERR_BOUNDS);
      o.ntiles[i] = 0;
      o.rect[4 * i] = o.rect[4 * i + 1] = o.rect[4 * i + 2] = o.rect[4 * i + 3] = 0;
      o.depth[i] = 0.0f;
      continue;
    }
    const float p[3] = {pos[3 * (int64_t)g], pos[3 * (int64_t)g + 1], pos[3 * (int64_t)g + 2]};
    const float s[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
    const float q[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
    float tc[3];
    cam_point(c, p, tc);
    const float x = tc[0], y = tc[1], z = tc[2];
    if (!(z > c.z_near)) {  // behind the near plane (rows kept without the pre-cull): no footprint
      o.ntiles[i] = 0;
      o.rect[4 * i] = o.rect[4 * i + 1] = o.rect[4 * i + 2] = o.rect[4 * i + 3] = 0;
      o.depth[i] = z;
      if (o.flag) o.flag[i] = 0;
      continue;
    }
    const float u = c.fx * x / z + c.cx;
    const float v = c.fy * y / z + c.cy;
    const float limx = 1.3f * (0.5f * (float)c.W / c.fx);
    const float limy = 1.3f * (0.5f * (float)c.H / c.fy);
    const float mx = fminf(limx, fmaxf(-limx, x / z));
    const float my = fminf(limy, fmaxf(-limy, y / z));
    const float j00 = c.fx / z, j02 = -(c.fx * mx) / z;
    const float j11 = c.fy / z, j12 = -(c.fy * my) / z;
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = j00 * c.R[k] + j02 * c.R[6 + k];
      T1[k] = j11 * c.R[3 + k] + j12 * c.R[6 + k];
    }
    const float w = q[0], qx = q[1], qy = q[2], qz = q[3];
    const float r[9] = {1.0f - 2.0f * (qy * qy + qz * qz), 2.0f * (qx * qy - w * qz),
                        2.0f * (qx * qz + w * qy),         2.0f * (qx * qy + w * qz),
                        1.0f - 2.0f * (qx * qx + qz * qz), 2.0f * (qy * qz - w * qx),
                        2.0f * (qx * qz - w * qy),         2.0f * (qy * qz + w * qx),
                        1.0f - 2.0f * (qx * qx + qy * qy)};
    float M[9], S[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) M[3 * a + k] = r[3 * a + k] * s[k];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        S[3 * a + b] = M[3 * a] * M[3 * b] + M[3 * a + 1] * M[3 * b + 1] + M[3 * a + 2] * M[3 * b + 2];
    float U0[3], U1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      U0[k] = T0[0] * S[k] + T0[1] * S[3 + k] + T0[2] * S[6 + k];
      U1[k] = T1[0] * S[k] + T1[1] * S[3 + k] + T1[2] * S[6 + k];
    }
    const float a = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2] + 0.3f;
    const float b = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
    const float cc = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2] + 0.3f;
    const float det = a * cc - b * b;
    const float mid = 0.5f * (a + cc);
    const float disc = fmaxf(mid * mid - det, 0.0f);
    const float lam = mid + sqrtf(disc);
    const float rad = ceilf(3.0f * sqrtf(lam));
    const float tw = (float)kTile;
    float x0 = floorf((u - rad) / tw), x1 = floorf((u + rad) / tw) + 1.0f;
    float y0 = floorf((v - rad) / tw), y1 = floorf((v + rad) / tw) + 1.0f;
    x0 = fminf(fmaxf(x0, 0.0f), (float)TX);
    x1 = fminf(fmaxf(x1, 0.0f), (float)TX);
    y0 = fminf(fmaxf(y0, 0.0f), (float)TY);
    y1 = fminf(fmaxf(y1, 0.0f), (float)TY);
    const int ix0 = (int)x0, ix1 = (int)x1, iy0 = (int)y0, iy1 = (int)y1;
    const bool near_singular = fabsf(det) < 1e-2f * a * cc;
    float con[3];
    if (near_singular) {
      conic_fp64(c, p, s, q, con);
    } else {
      const float inv = 1.0f / det;
      con[0] = cc * inv;
      con[1] = -b * inv;
      con[2] = a * inv;
    }
    o.mean2d[2 * i] = u;
    o.mean2d[2 * i + 1] = v;
    o.conic[3 * i] = con[0];
    o.conic[3 * i + 1] = con[1];
    o.conic[3 * i + 2] = con[2];
    o.depth[i] = z;
    o.rect[4 * i] = ix0;
    o.rect[4 * i + 1] = iy0;
    o.rect[4 * i + 2] = ix1;
    o.rect[4 * i + 3] = iy1;
    int nt = (ix1 > ix0 && iy1 > iy0) ? (ix1 - ix0) * (iy1 - iy0) : 0;
    if (o.foot) {
      // the footprint (footprint.cuh); near-singular Gaussians keep their
      // rectangle (their conic comes from an FP64 recomputation of Sigma')
      float t = fp_qlimit(o.alpha ? o.alpha[i] : 1.0f);
      if (near_singular && t >= 0.0f) t = INFINITY;
      uint32_t w[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
      nt = 0;
      if (t >= 0.0f && iy1 > iy0 && ix1 > ix0) {
        const FootRows fr = fp_rows(a, b, cc, t);
        if (fp_packed(iy1 - iy0, ix1 - ix0)) {
#pragma unroll
          for (int j = 0; j < kSpanRows; ++j) {
            if (iy0 + j < iy1) {
              int t0, t1;
              fp_row_span(fr, u, v, cc, t, iy0 + j, ix0, ix1, t0, t1);
              nt += t1 - t0;
              w[j >> 1] |= (uint32_t)((t0 - ix0) | ((t1 - t0) << 8)) << (16 * (j & 1));
            }
          }
        } else {
          for (int ty = iy0; ty < iy1; ++ty) {
            int t0, t1;
            fp_row_span(fr, u, v, cc, t, ty, ix0, ix1, t0, t1);
            nt += t1 - t0;
          }
        }
      }
      o.foot[kFootVec * i] = make_float4(a, b, cc, t);
      reinterpret_cast<uint4*>(o.foot)[kFootVec * i + 1] = make_uint4(w[0], w[1], w[2], w[3]);
      reinterpret_cast<uint4*>(o.foot)[kFootVec * i + 2] = make_uint4(w[4], w[5], w[6], w[7]);
    }
    o.ntiles[i] = nt;
    if (o.flag) o.flag[i] = near_singular ? 1 : 0;
  }
}

// ---------------------------------------------------------------- launchers

// Exclusive scan of m per-chunk counts in place, total to *total (one CTA).
hyrf_status launch_scan_small(int32_t* counts, int m, int32_t* total, cudaStream_t s) {
  HYRF_LAUNCH("k_scan_small", s, k_scan_small<<<1, 1024, 0, s>>>(counts, m, total));
  return HYRF_OK;
}

size_t precull_workspace(int n) {
  Carver c(nullptr);
  c.take<int32_t>((n + kChunk - 1) / kChunk + 1);
  return c.size();
}

hyrf_status launch_precull(const CamDev& cam, const float* pos, int n, int32_t* vis_ids,
                           int32_t* n_vis, void* ws, cudaStream_t s) {
  const int chunks = (n + kChunk - 1) / kChunk;
  Carver c(ws);
  int32_t* counts = c.take<int32_t>(chunks + 1);
  if (chunks == 0) {
    cudaMemsetAsync(n_vis, 0, sizeof(int32_t), s);
    return cudaPeekAtLastError() == cudaSuccess ? HYRF_OK : HYRF_ERR_CUDA;
  }
  HYRF_LAUNCH("k_precull_count", s,
              k_precull_count<<<chunks, 256, 0, s>>>(cam, pos, n, counts));
  HYRF_LAUNCH("k_scan_small", s,
              k_scan_small<<<1, 1024, 0, s>>>(counts, chunks, n_vis));
  HYRF_LAUNCH("k_precull_scatter", s,
              k_precull_scatter<<<chunks, 256, 0, s>>>(cam, pos, n, counts, vis_ids));
  return HYRF_OK;
}

// Camera-space depth z of every visible row: the z of cam_point, as in
// k_project (this file's operation order), so that the depth keys of
// hyrf_depth_order and of hyrf_project agree bit for bit.
__global__ void __launch_bounds__(256) k_depth_of(CamDev c, int n, const float* __restrict__ pos,
                                                  const int32_t* __restrict__ vis_ids,
                                                  const int32_t* __restrict__ n_vis, float* __restrict__ depth,
                                                  int32_t* status) {
  const int nv = min(*n_vis, n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int g = vis_ids[i];
    if (g < 0 || g >= n) {
      set_status(status, HYRF_ERR_BOUNDS);
      depth[i] = 0.0f;
      continue;
    }
    const float p[3] = {pos[3 * (int64_t)g], pos[3 * (int64_t)g + 1], pos[3 * (int64_t)g + 2]};
    float tc[3];
    cam_point(c, p, tc);
    depth[i] = tc[2];
  }
}

hyrf_status launch_depth_of(const CamDev& cam, int n, const float* pos, const int32_t* vis_ids,
                            const int32_t* n_vis, float* depth, int32_t* status, cudaStream_t s) {
  if (n == 0) return HYRF_OK;
  int blocks = (n + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  HYRF_LAUNCH("k_depth_of", s, k_depth_of<<<blocks, 256, 0, s>>>(cam, n, pos, vis_ids, n_vis, depth, status));
  return HYRF_OK;
}

hyrf_status launch_project(const CamDev& cam, int n, const float* pos, const int32_t* vis_ids,
                           const int32_t* n_vis, const float* scale, const float* quat, float* mean2d,
                           float* conic, float* depth, int32_t* rect, int32_t* ntiles, uint8_t* flag,
                           int32_t* status, const float* alpha, float* footprint, cudaStream_t s) {
  if (n == 0) return HYRF_OK;
  const int TX = (cam.W + kTile - 1) / kTile, TY = (cam.H + kTile - 1) / kTile;
  ProjOut o{mean2d, conic, depth, rect, ntiles, flag, alpha, reinterpret_cast<float4*>(footprint)};
  int blocks = (n + 255) / 256;
  blocks = blocks < num_sms() * 8 ? blocks : num_sms() * 8;
  HYRF_LAUNCH("k_project", s,
              k_project<<<blocks, 256, 0, s>>>(cam, n, pos, vis_ids, n_vis, scale, quat, TX, TY, o, status));
  return HYRF_OK;
}

}  // namespace hyrf
