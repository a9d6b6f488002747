// Front-to-back alpha compositing of Eq. 1 per 16x16 tile, and its reverse.
// One CTA of 256 threads per tile, one pixel per thread. The visible
// Gaussians' screen-space records are first packed into 48-byte rows
// (three float4: {u, v, conic a, conic b}, {conic c, opacity, r, g}, {b})
// so that a tile stages a batch of 256 of them into shared memory with
// three vector loads per thread. The forward ends a tile early once every
// pixel has stopped (CTA-wide vote). The reverse walks each pixel's list
// back to front, recovering T from the stored T_final by division, reduces
// the per-Gaussian gradients across each warp and adds them with atomics.
#include "common.cuh"

namespace hyrf {

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

__global__ void __launch_bounds__(256) k_pack(const int32_t* __restrict__ n_vis, int n,
                                              const float* __restrict__ mean2d,
                                              const float* __restrict__ conic,
                                              const float* __restrict__ alpha,
                                              const float* __restrict__ color,
                                              float4* __restrict__ rec) {
  const int nv = min(*n_vis, n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    rec[3 * i] = make_float4(mean2d[2 * i], mean2d[2 * i + 1], conic[3 * i], conic[3 * i + 1]);
    rec[3 * i + 1] = make_float4(conic[3 * i + 2], alpha[i], color[3 * i], color[3 * i + 1]);
    rec[3 * i + 2] = make_float4(color[3 * i + 2], 0.0f, 0.0f, 0.0f);
  }
}

// exp of the (non-positive) splat exponent with the hardware exponential
// (relative error ~1e-6 here, far inside the compositing tolerances); the
// forward and the reverse pass evaluate it identically, so their
// threshold decisions agree bit for bit.
__device__ __forceinline__ float splat_exp(float power) { return __expf(power); }

// Exponent of the 2D Gaussian at offset (dx, dy) = mean - pixel centre, with
// a fixed multiply-add order shared by the forward and the reverse pass.
__device__ __forceinline__ float splat_power(float ca, float cb, float cc, float dx, float dy) {
  const float q = fmaf(cc * dy, dy, ca * dx * dx);
  return fmaf(-0.5f, q, -(cb * dx * dy));
}

__global__ void __launch_bounds__(256) k_raster_fwd(const int32_t* __restrict__ ranges,
                                                    const int32_t* __restrict__ vals, int n,
                                                    const float4* __restrict__ rec, int W, int H,
                                                    int TX, float* __restrict__ C_fg,
                                                    float* __restrict__ T_final,
                                                    int32_t* __restrict__ n_contrib,
                                                    int32_t* status) {
  __shared__ float4 s0[256], s1[256], s2[256];
  const int tile = blockIdx.x;
  const int t = threadIdx.x;
  const int px = (tile % TX) * kTile + (t % kTile);
  const int py = (tile / TX) * kTile + (t / kTile);
  const bool inside = px < W && py < H;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const int start = ranges[2 * tile], end = ranges[2 * tile + 1];
  float T = 1.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
  int last = 0;
  bool done = !inside;
  for (int b0 = start; b0 < end; b0 += 256) {
    if (__syncthreads_count(done) == 256) break;
    const int k = b0 + t;
    if (k < end) {
      int g = vals[k];
      if (g < 0 || g >= n) {
        set_status(status, HYRF_ERR_BOUNDS);
        s0[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        s1[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // opacity 0: never contributes
      } else {
        s0[t] = rec[3 * g];
        s1[t] = rec[3 * g + 1];
        s2[t] = rec[3 * g + 2];
      }
    }
    __syncthreads();
    const int cnt = min(256, end - b0);
    for (int j = 0; j < cnt && !done; ++j) {
      const float4 r0 = s0[j], r1 = s1[j];
      const float dx = r0.x - fx, dy = r0.y - fy;
      const float power = splat_power(r0.z, r0.w, r1.x, dx, dy);
      if (power > 0.0f) continue;
      const float alpha = fminf(kAlphaMax, r1.y * splat_exp(power));
      if (alpha < kAlphaMin) continue;
      const float test_T = T * (1.0f - alpha);
      if (test_T < kTMin) {
        done = true;
        break;
      }
      const float w = alpha * T;
      c0 = fmaf(r1.z, w, c0);
      c1 = fmaf(r1.w, w, c1);
      c2 = fmaf(s2[j].x, w, c2);
      T = test_T;
      last = b0 - start + j + 1;
    }
  }
  if (inside) {
    const int p = py * W + px;
    C_fg[3 * p] = c0;
    C_fg[3 * p + 1] = c1;
    C_fg[3 * p + 2] = c2;
    T_final[p] = T;
    n_contrib[p] = last;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums of 8 values over the 32 lanes by recursive halving (9 shuffles
// instead of 8 x 5): each step a lane keeps half of its partial sums and
// adds its partner's copy of that half. On return the lanes with
// (lane & 3) == 0 hold the sum of value col8(lane), one value each.
__device__ __forceinline__ float reduce8(float* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 4, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = up ? v[j] : v[j + h];
      const float keep = up ? v[j + h] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float s = v[0];
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  return s;
}

__device__ __forceinline__ int col8(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// State of one pixel's back-to-front walk: T before the current Gaussian
// (recovered from T_final), the colour composited behind it (normalised by T
// after it), the previous contributor, and the pixel's upstream gradients.
struct PixBack {
  float fx, fy, Tf, T, g0, g1, g2, gT, a0, a1, a2, la, lc0, lc1, lc2;
  int last;
};

__device__ __forceinline__ void pix_init(PixBack& q, int px, int py, int W, int H,
                                         const float* __restrict__ T_final,
                                         const int32_t* __restrict__ n_contrib,
                                         const float* __restrict__ dC, const float* __restrict__ dT) {
  const bool inside = px < W && py < H;
  const int p = inside ? py * W + px : 0;
  q.fx = (float)px + 0.5f;
  q.fy = (float)py + 0.5f;
  q.Tf = inside ? T_final[p] : 1.0f;
  q.T = q.Tf;
  q.last = inside ? n_contrib[p] : 0;
  q.g0 = inside ? dC[3 * p] : 0.0f;
  q.g1 = inside ? dC[3 * p + 1] : 0.0f;
  q.g2 = inside ? dC[3 * p + 2] : 0.0f;
  q.gT = inside ? dT[p] : 0.0f;
  q.a0 = q.a1 = q.a2 = q.la = q.lc0 = q.lc1 = q.lc2 = 0.0f;
}

// Reverse of one (pixel, Gaussian) compositing step at list position pos:
// adds dL/d(mean2d u, v, conic a, b, c, opacity, colour r, g, b) of this
// pixel to acc; false if the Gaussian did not contribute to the pixel.
__device__ __forceinline__ bool pix_step(PixBack& q, int pos, const float4& r0, const float4& r1, float cb,
                                         float* acc) {
  if (pos >= q.last) return false;
  const float dx = r0.x - q.fx, dy = r0.y - q.fy;
  const float power = splat_power(r0.z, r0.w, r1.x, dx, dy);
  if (power > 0.0f) return false;
  const float G = splat_exp(power);
  const float oG = r1.y * G;
  const float alpha = fminf(kAlphaMax, oG);
  if (alpha < kAlphaMin) return false;
  const float inv = __fdividef(1.0f, 1.0f - alpha);  // 1 - alpha >= 0.01
  q.T = q.T * inv;                                   // T before this Gaussian
  q.a0 = q.la * q.lc0 + (1.0f - q.la) * q.a0;
  q.a1 = q.la * q.lc1 + (1.0f - q.la) * q.a1;
  q.a2 = q.la * q.lc2 + (1.0f - q.la) * q.a2;
  q.la = alpha;
  q.lc0 = r1.z;
  q.lc1 = r1.w;
  q.lc2 = cb;
  const float w = alpha * q.T;
  acc[6] += w * q.g0;
  acc[7] += w * q.g1;
  acc[8] += w * q.g2;
  float dal = ((r1.z - q.a0) * q.g0 + (r1.w - q.a1) * q.g1 + (cb - q.a2) * q.g2) * q.T;
  dal -= q.gT * q.Tf * inv;
  if (oG <= kAlphaMax) {
    acc[5] += dal * G;
    const float dp = dal * alpha;
    acc[0] += dp * (-(r0.z * dx) - r0.w * dy);
    acc[1] += dp * (-(r1.x * dy) - r0.w * dx);
    acc[2] += dp * (-0.5f * dx * dx);
    acc[3] += dp * (-(dx * dy));
    acc[4] += dp * (-0.5f * dy * dy);
  }
  return true;
}

// Two pixels per thread, (x, y) and (x, y + 2): a warp covers four rows of the
// tile, so each warp-level reduction of a Gaussian's gradient sums 64 pixels.
constexpr int kBwdRasterThreads = 128;

__global__ void __launch_bounds__(kBwdRasterThreads) k_raster_bwd(
    const int32_t* __restrict__ ranges, const int32_t* __restrict__ vals, int n,
    const float4* __restrict__ rec, int W, int H, int TX, const float* __restrict__ T_final,
    const int32_t* __restrict__ n_contrib, const float* __restrict__ dC,
    const float* __restrict__ dT, float* __restrict__ d_mean2d, float* __restrict__ d_conic,
    float* __restrict__ d_alpha, float* __restrict__ d_color) {
  constexpr int B = 256;  // Gaussians staged per batch
  __shared__ float4 s0[B], s1[B], s2[B];
  __shared__ int sg[B];
  __shared__ int max_last;
  const int tile = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int px = (tile % TX) * kTile + (lane & 15);
  const int py = (tile / TX) * kTile + 4 * wp + (lane >> 4);
  const int start = ranges[2 * tile], end = ranges[2 * tile + 1];
  PixBack A, Bq;
  pix_init(A, px, py, W, H, T_final, n_contrib, dC, dT);
  pix_init(Bq, px, py + 2, W, H, T_final, n_contrib, dC, dT);
  const int mylast = max(A.last, Bq.last);
  if (t == 0) max_last = 0;
  __syncthreads();
  atomicMax(&max_last, mylast);
  __syncthreads();
  const int stop = min(end, start + max_last);  // no pixel of the tile used positions >= stop
  // nor did any pixel of this warp use positions >= wstop (warp-uniform bound)
  const int wstop = start + __reduce_max_sync(0xffffffffu, mylast);
  for (int b1 = stop; b1 > start; b1 -= B) {
    const int b0 = max(start, b1 - B);
    __syncthreads();
    for (int e = t; e < b1 - b0; e += kBwdRasterThreads) {
      int g = vals[b0 + e];
      if (g < 0 || g >= n) {
        g = -1;
        s1[e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // opacity 0: never contributes
      } else {
        s0[e] = rec[3 * g];
        s1[e] = rec[3 * g + 1];
        s2[e] = rec[3 * g + 2];
      }
      sg[e] = g;
    }
    __syncthreads();
    for (int j = min(b1, wstop) - b0 - 1; j >= 0; --j) {
      const int pos = b0 - start + j;  // list position
      const float4 r0 = s0[j], r1 = s1[j];
      const float cb = s2[j].x;
      float acc[9] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      const bool ca = pix_step(A, pos, r0, r1, cb, acc);
      const bool cbq = pix_step(Bq, pos, r0, r1, cb, acc);
      if (__any_sync(0xffffffffu, ca || cbq)) {
        // mean2d (2), conic (3), opacity, colour r, g: one sum per lane group
        const float s8 = reduce8(acc);
        const float sb = warp_sum(acc[8]);
        const int g = sg[j];
        if (g >= 0) {
          if ((lane & 3) == 0) {
            const int c = col8(lane);
            float* dst = c < 2 ? d_mean2d + 2 * g + c
                         : c < 5 ? d_conic + 3 * g + (c - 2)
                         : c == 5 ? d_alpha + g
                                  : d_color + 3 * g + (c - 6);
            atomicAdd(dst, s8);
          }
          if (lane == 1) atomicAdd(d_color + 3 * g + 2, sb);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- host side

size_t raster_workspace(int n) {
  Carver c(nullptr);
  c.take<float4>((size_t)3 * (n > 0 ? n : 1));
  return c.size();
}

static hyrf_status pack(const hyrf_rasterize_args& a, float4* rec, cudaStream_t s) {
  int blocks = (a.n + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  if (blocks < 1) blocks = 1;
  HYRF_LAUNCH("k_pack", s,
              k_pack<<<blocks, 256, 0, s>>>(a.n_vis, a.n, a.mean2d, a.conic, a.alpha, a.color, rec));
  return HYRF_OK;
}

hyrf_status launch_raster_fwd(const hyrf_rasterize_args& a, void* ws, cudaStream_t s) {
  const int TX = (a.width + kTile - 1) / kTile, TY = (a.height + kTile - 1) / kTile;
  Carver c(ws);
  float4* rec = c.take<float4>((size_t)3 * (a.n > 0 ? a.n : 1));
  hyrf_status st = pack(a, rec, s);
  if (st != HYRF_OK) return st;
  HYRF_LAUNCH("k_raster_fwd", s,
              k_raster_fwd<<<TX * TY, 256, 0, s>>>(a.ranges, a.vals, a.n, rec, a.width, a.height, TX, a.C_fg,
                                       a.T_final, a.n_contrib, a.status));
  return HYRF_OK;
}

hyrf_status launch_raster_bwd(const hyrf_rasterize_backward_args& b, void* ws, cudaStream_t s) {
  const hyrf_rasterize_args& a = b.fwd;
  const int TX = (a.width + kTile - 1) / kTile, TY = (a.height + kTile - 1) / kTile;
  Carver c(ws);
  float4* rec = c.take<float4>((size_t)3 * (a.n > 0 ? a.n : 1));
  hyrf_status st = pack(a, rec, s);
  if (st != HYRF_OK) return st;
  HYRF_LAUNCH("k_raster_bwd", s,
              k_raster_bwd<<<TX * TY, kBwdRasterThreads, 0, s>>>(a.ranges, a.vals, a.n, rec, a.width, a.height, TX, a.T_final,
                                       a.n_contrib, b.d_C_fg, b.d_T_final, b.d_mean2d, b.d_conic,
                                       b.d_alpha, b.d_color));
  return HYRF_OK;
}

}  // namespace hyrf
