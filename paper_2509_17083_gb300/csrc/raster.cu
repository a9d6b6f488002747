// Front-to-back alpha compositing of Eq. 1 per 16x16 tile, and its reverse.
// The forward runs one CTA of 256 threads per tile, one pixel per thread.
// The visible Gaussians' screen-space records are first packed into
// 48-byte rows (three float4: {u, v, conic a, conic b}, {conic c, opacity,
// r, g}, {b, p_min}) so that a tile stages a batch of 256 of them into
// shared memory with three vector loads per thread; p_min is a lower bound
// of the exponent below which the opacity test must fail, so most
// (pixel, Gaussian) pairs are rejected before the exponential. The forward
// ends a tile early once every pixel has stopped (CTA-wide vote). The
// reverse walks each pixel's list back to front, recovering T from the
// stored T_final by division, with several pixels of one column per thread,
// reduces the per-Gaussian gradients across each warp and adds them with
// atomics. Both passes can take the tiles in decreasing order of their
// longest pixel list (k_tile_work / k_tile_order: a previous frame's for
// the forward, the current one for the reverse), so that the last CTAs to
// run on each SM are short ones.
#include "common.cuh"

namespace hyrf {

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// exp of the (non-positive) splat exponent with the hardware exponential
// (relative error ~1e-6 here, far inside the compositing tolerances); the
// forward and the reverse pass evaluate it identically, so their
// threshold decisions agree bit for bit.
__device__ __forceinline__ float splat_exp(float power) { return __expf(power); }

// Exponent of the 2D Gaussian at offset (dx, dy) = mean - pixel centre,
// from the pixel-independent parts (conic a) dx dx and (conic b) dx of the
// column, with a fixed operation order shared by the forward and the
// reverse pass.
__device__ __forceinline__ float splat_power(float cadx2, float cbdx, float cc, float dy) {
  const float q = fmaf(cc * dy, dy, cadx2);
  return fmaf(-0.5f, q, -(cbdx * dy));
}

// p_min of a Gaussian with opacity o: for an exponent below it,
// o exp(power) < 1/255 holds with a margin (1e-3 in the exponent, three
// orders above the error of the hardware exponential and of the products),
// so the opacity test of Eq. 1 fails and the exponential is not needed.
// +inf when no exponent can pass (o <= 1/255 or o not a number).
__device__ __forceinline__ float splat_pmin(float o) {
  return o > kAlphaMin ? logf(kAlphaMin / o) - 1e-3f : INFINITY;
}

// Opacity test of Eq. 1 at one pixel: alpha = min(0.99, o G) with
// G = exp(power); false when power > 0 or alpha < 1/255 (exactly the
// decision of the unscreened test: p_min only skips certain failures).
__device__ __forceinline__ bool splat_alpha(float power, float pmin, float o, float& G, float& alpha) {
  if (!(power >= pmin && power <= 0.0f)) return false;
  G = splat_exp(power);
  alpha = fminf(kAlphaMax, o * G);
  return alpha >= kAlphaMin;
}

// Paired FP32 arithmetic (two independent round-to-nearest operations per
// instruction, the same values as the scalar ones): the compositing reverse
// runs two pixels per thread through one instruction stream.
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  float2 d;
  asm("{\n.reg .b64 p, q;\nmov.b64 p, {%2, %3};\nmov.b64 q, {%4, %5};\nadd.rn.f32x2 p, p, q;\n"
      "mov.b64 {%0, %1}, p;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  float2 d;
  asm("{\n.reg .b64 p, q;\nmov.b64 p, {%2, %3};\nmov.b64 q, {%4, %5};\nsub.rn.f32x2 p, p, q;\n"
      "mov.b64 {%0, %1}, p;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  float2 d;
  asm("{\n.reg .b64 p, q;\nmov.b64 p, {%2, %3};\nmov.b64 q, {%4, %5};\nmul.rn.f32x2 p, p, q;\n"
      "mov.b64 {%0, %1}, p;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// a b + c
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n.reg .b64 p, q, r;\nmov.b64 p, {%2, %3};\nmov.b64 q, {%4, %5};\nmov.b64 r, {%6, %7};\n"
      "fma.rn.f32x2 p, p, q, r;\nmov.b64 {%0, %1}, p;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 pbc(float s) { return make_float2(s, s); }

// Asynchronous global -> shared copies (cp.async, L1-allocating): a batch
// of records lands in shared memory while the previous batch is composited.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// 16 bytes through L2 only (no L1 line allocated).
__device__ __forceinline__ void cp_async16_l2(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's most recent groups are in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Records of 256 Gaussians per CTA and pass: the inputs are read
// coalesced into shared memory, the 48-byte records written coalesced as
// consecutive float4.
__global__ void __launch_bounds__(256) k_pack(const int32_t* __restrict__ n_vis, int n,
                                              const float* __restrict__ mean2d,
                                              const float* __restrict__ conic,
                                              const float* __restrict__ alpha,
                                              const float* __restrict__ color,
                                              float4* __restrict__ rec) {
  __shared__ float sm2[2 * 256], sc3[3 * 256], sa[256], scl[3 * 256];
  const int nv = min(*n_vis, n);
  const int t = threadIdx.x;
  for (int i0 = blockIdx.x * 256; i0 < nv; i0 += gridDim.x * 256) {
    const int m = min(256, nv - i0);
    for (int k = t; k < 2 * m; k += 256) sm2[k] = mean2d[2 * (size_t)i0 + k];
    for (int k = t; k < 3 * m; k += 256) {
      sc3[k] = conic[3 * (size_t)i0 + k];
      scl[k] = color[3 * (size_t)i0 + k];
    }
    if (t < m) sa[t] = alpha[i0 + t];
    __syncthreads();
    for (int k = t; k < 3 * m; k += 256) {
      const int i = k / 3, part = k % 3;
      float4 v;
      if (part == 0) v = make_float4(sm2[2 * i], sm2[2 * i + 1], sc3[3 * i], sc3[3 * i + 1]);
      else if (part == 1) v = make_float4(sc3[3 * i + 2], sa[i], scl[3 * i], scl[3 * i + 1]);
      else v = make_float4(scl[3 * i + 2], splat_pmin(sa[i]), 0.0f, 0.0f);
      rec[3 * (size_t)i0 + k] = v;
    }
    __syncthreads();
  }
}

// One CTA per tile, one pixel per thread. The tile's list is taken in
// batches of 256 records (cp.async, one record per thread, into a double
// buffer). Most tiles stop within their first batch or two, so the first
// batch is loaded alone; from the second on, batch b + 1 is copied into the
// other half of the buffer while batch b is composited.
__global__ void __launch_bounds__(256) k_raster_fwd(const int32_t* __restrict__ ranges,
                                                    const int32_t* __restrict__ vals, int n,
                                                    const float4* __restrict__ rec, int W, int H,
                                                    int TX, const int32_t* __restrict__ order,
                                                    float* __restrict__ C_fg,
                                                    float* __restrict__ T_final,
                                                    int32_t* __restrict__ n_contrib,
                                                    int32_t* status) {
  __shared__ float4 s0[2][256], s1[2][256], s2[2][256];
  const int tile = order ? order[blockIdx.x] : (int)blockIdx.x;
  if (tile < 0 || tile >= gridDim.x) {  // CTA-uniform
    if (threadIdx.x == 0) set_status(status, HYRF_ERR_BOUNDS);
    return;
  }
  const int t = threadIdx.x;
  const int px = (tile % TX) * kTile + (t % kTile);
  const int py = (tile / TX) * kTile + (t / kTile);
  const bool inside = px < W && py < H;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const int start = ranges[2 * tile], end = ranges[2 * tile + 1];
  const int nb = (end - start + 255) / 256;
  // record of list position start + 256 b + t into buffer b & 1; g is its
  // Gaussian (from vals), or -1 past the end of the list
  auto stage = [&](int b, int g) {
    const int buf = b & 1;
    if (g < 0) return;
    if (g >= n) {
      set_status(status, HYRF_ERR_BOUNDS);
      s0[buf][t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      s1[buf][t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // opacity 0: never contributes
      s2[buf][t] = make_float4(0.0f, INFINITY, 0.0f, 0.0f);
      return;
    }
    cp_async16(&s0[buf][t], rec + 3 * (size_t)g);
    cp_async16(&s1[buf][t], rec + 3 * (size_t)g + 1);
    cp_async16(&s2[buf][t], rec + 3 * (size_t)g + 2);
  };
  auto index = [&](int b) {
    const int k = start + 256 * b + t;
    if (b >= nb || k >= end) return -1;
    const int g = vals[k];
    return g < 0 ? n : g;  // out of range either way: stage() reports it
  };
  auto fetch = [&](int b) {
    stage(b, index(b));
    cp_async_commit();
  };
  float T = 1.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
  int last = 0;
  bool done = !inside;
  fetch(0);
  for (int b = 0; b < nb; ++b) {
    // also: every thread is done with batch b - 1, whose buffer the copies
    // of batch b + 1 overwrite
    if (__syncthreads_count(done) == 256) break;
    if (b == 1) fetch(1);
    if (b >= 1) fetch(b + 1);
    if (b == 0) cp_async_wait<0>();
    else cp_async_wait<1>();  // this thread's copies of batch b have landed
    __syncthreads();          // and everyone's
    const int buf = b & 1, b0 = start + 256 * b;
    const int cnt = min(256, end - b0);
    for (int j = 0; j < cnt && !done; ++j) {
      const float4 r0 = s0[buf][j], r1 = s1[buf][j];
      const float dx = r0.x - fx, dy = r0.y - fy;
      const float power = splat_power(r0.z * dx * dx, r0.w * dx, r1.x, dy);
      float G, alpha;
      if (!splat_alpha(power, s2[buf][j].y, r1.y, G, alpha)) continue;
      const float test_T = T * (1.0f - alpha);
      if (test_T < kTMin) {
        done = true;
        break;
      }
      const float w = alpha * T;
      c0 = fmaf(r1.z, w, c0);
      c1 = fmaf(r1.w, w, c1);
      c2 = fmaf(s2[buf][j].x, w, c2);
      T = test_T;
      last = b0 - start + j + 1;
    }
  }
  cp_async_wait<0>();  // no copy outlives the CTA
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
    float keep[4], got[4];
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = up ? v[j] : v[j + h];
      keep[j] = up ? v[j + h] : v[j];
      got[j] = __shfl_xor_sync(0xffffffffu, send, o);
    }
    if (h >= 2) {  // the sums two at a time (paired adds, same values)
#pragma unroll
      for (int j = 0; j < h; j += 2) {
        const float2 s2 = padd(make_float2(keep[j], keep[j + 1]), make_float2(got[j], got[j + 1]));
        v[j] = s2.x;
        v[j + 1] = s2.y;
      }
    } else {
      v[0] = keep[0] + got[0];
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

// Reverse of Eq. 1 per tile: each pixel walks its list back to front from
// its last contributor, recovering T before each Gaussian from T after it
// (division by 1 - alpha) and the colour composited behind it through
// S = (colour behind) . dL/dC, so that
//   dL/dalpha = (c . dL/dC - S) T - dL/dT_final T_final / (1 - alpha).
// A thread holds P pixels of one column (rows r, r + 2, ..., r + 2(P - 1));
// a CTA of WARPS warps covers WARPS x 2P rows of a tile, so a tile takes
// 16 / (2 P WARPS) CTAs (smaller CTAs leave less work in the last ones to
// finish on each SM); the x offset dx of a Gaussian is common to
// the thread's pixels, so the conic and mean gradients are accumulated as
// sums D0 = sum dp, D1 = sum dp dy, D2 = sum dp dy^2 (dp = dL/dpower) and
// expanded once per Gaussian before the warp reduction.
#ifndef HYRF_RASTER_BWD_WARPS
#define HYRF_RASTER_BWD_WARPS 4
#endif
#ifndef HYRF_RASTER_BWD_PIXELS
#define HYRF_RASTER_BWD_PIXELS 2
#endif
constexpr int kBwdRasterWarps = HYRF_RASTER_BWD_WARPS;
constexpr int kBwdRasterPixels = HYRF_RASTER_BWD_PIXELS;
static_assert(kTile % (2 * kBwdRasterWarps * kBwdRasterPixels) == 0,
              "a CTA covers a whole number of row pairs of a tile");
constexpr int kBwdCtasPerTile = kTile / (2 * kBwdRasterWarps * kBwdRasterPixels);

template <int WARPS, int P>
__global__ void __launch_bounds__(32 * WARPS) k_raster_bwd(
    const int32_t* __restrict__ ranges, const int32_t* __restrict__ vals, int n,
    const float4* __restrict__ rec, int W, int H, int TX, const int32_t* __restrict__ order,
    const float* __restrict__ T_final, const int32_t* __restrict__ n_contrib, const float* __restrict__ dC,
    const float* __restrict__ dT, const float* __restrict__ Cimg, const float* __restrict__ C_fg,
    float* __restrict__ d_mean2d, float* __restrict__ d_conic, float* __restrict__ d_alpha,
    float* __restrict__ d_color, int32_t* status) {
  constexpr int NT = 32 * WARPS;     // threads per CTA
  constexpr int CPT = kTile / (2 * WARPS * P);  // CTAs per tile
  constexpr int B = 256;             // Gaussians staged per batch
  __shared__ float4 s0[2][B], s1[2][B];
  __shared__ float2 s2[2][B];
  __shared__ int sg[2][B];
  __shared__ int max_last;
  const int tile = order[blockIdx.x / CPT], sub = blockIdx.x % CPT;
  if (tile < 0 || tile >= (int)(gridDim.x / CPT)) {  // CTA-uniform
    if (threadIdx.x == 0) set_status(status, HYRF_ERR_BOUNDS);
    return;
  }
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int px = (tile % TX) * kTile + (lane & 15);
  const int py0 = (tile / TX) * kTile + (sub * WARPS + wp) * 2 * P + (lane >> 4);
  const int start = ranges[2 * tile], end = ranges[2 * tile + 1];
  const float fx = (float)px + 0.5f;
  float fy[P], T[P], g0[P], g1[P], g2[P], gTf[P], S[P], la[P], ls[P];
  int last[P];
  int mylast = 0;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int py = py0 + 2 * k;
    const bool inside = px < W && py < H;
    const int p = inside ? py * W + px : 0;
    fy[k] = (float)py + 0.5f;
    const float Tf = inside ? T_final[p] : 1.0f;
    T[k] = Tf;
    last[k] = inside ? n_contrib[p] : 0;
    g0[k] = inside ? dC[3 * p] : 0.0f;
    g1[k] = inside ? dC[3 * p + 1] : 0.0f;
    g2[k] = inside ? dC[3 * p + 2] : 0.0f;
    if (!inside) {
      gTf[k] = 0.0f;
    } else if (dT) {
      gTf[k] = dT[p] * Tf;
    } else {  // dL/dT_final T_final = dL/dC . (C - C_fg), Eq. 11
      gTf[k] = g0[k] * (Cimg[3 * p] - C_fg[3 * p]) + g1[k] * (Cimg[3 * p + 1] - C_fg[3 * p + 1]) +
               g2[k] * (Cimg[3 * p + 2] - C_fg[3 * p + 2]);
    }
    S[k] = la[k] = ls[k] = 0.0f;
    mylast = max(mylast, last[k]);
  }
  // no pixel of this warp used list positions >= wstop (warp-uniform)
  // the gradient this lane adds after each reduction: value col8(lane) of
  // (mean2d u, v, conic a, b, c, opacity, colour r, g) at base + stride g;
  // lane 1 adds colour b
  float* gbase;
  int gstride;
  {
    const int c = col8(lane);
    gbase = c < 2 ? d_mean2d + c : c < 5 ? d_conic + (c - 2) : c == 5 ? d_alpha : d_color + (c - 6);
    gstride = c < 2 ? 2 : c == 5 ? 1 : 3;
    if (lane == 1) {
      gbase = d_color + 2;
      gstride = 3;
    }
  }
  const bool adds = (lane & 3) == 0 || lane == 1;
  const int wlast = __reduce_max_sync(0xffffffffu, mylast);
  const int wstop = start + wlast;
  if (t == 0) max_last = 0;
  __syncthreads();
  if (lane == 0) atomicMax(&max_last, wlast);
  __syncthreads();
  const int stop = min(end, start + max_last);  // nor did any pixel of the tile use positions >= stop
  // batches of B list positions from the back: batch k is [b0, b1) with
  // b1 = stop - k B; batch k + 1 is copied into the other half of a double
  // buffer (cp.async, NT records at a time) while batch k is walked, and the
  // list indices of batch k + 2 are fetched meanwhile
  const int nbk = stop > start ? (stop - start + B - 1) / B : 0;
  constexpr int kNone = -2;  // no list position here
  constexpr int EPT = B / NT;  // records per thread and batch
  auto index = [&](int k, int* g) {
    const int b1 = stop - k * B, b0 = max(start, b1 - B);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = t + u * NT;
      g[u] = (k < nbk && e < b1 - b0) ? vals[b0 + e] : kNone;
    }
  };
  auto stage = [&](int k, const int* g) {
    const int buf = k & 1;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int e = t + u * NT;
      if (g[u] == kNone) continue;
      if (g[u] < 0 || g[u] >= n) {
        s1[buf][e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        s2[buf][e] = make_float2(0.0f, INFINITY);  // never contributes
        sg[buf][e] = -1;
      } else {
        cp_async16_l2(&s0[buf][e], rec + 3 * (size_t)g[u]);
        cp_async16_l2(&s1[buf][e], rec + 3 * (size_t)g[u] + 1);
        cp_async8(&s2[buf][e], rec + 3 * (size_t)g[u] + 2);
        sg[buf][e] = g[u];
      }
    }
  };
  int gn[EPT];
  index(0, gn);
  stage(0, gn);
  cp_async_commit();
  index(1, gn);
  for (int k = 0; k < nbk; ++k) {
    const int b1 = stop - k * B, b0 = max(start, b1 - B), buf = k & 1;
    __syncthreads();  // batch k - 1 is walked: its buffer takes batch k + 1
    stage(k + 1, gn);
    cp_async_commit();
    index(k + 2, gn);
    cp_async_wait<1>();  // this thread's copies of batch k have landed
    __syncthreads();     // and everyone's
    for (int j = min(b1, wstop) - b0 - 1; j >= 0; --j) {
      const int pos = b0 - start + j;  // list position
      const float4 r0 = s0[buf][j], r1 = s1[buf][j];
      const float2 r2 = s2[buf][j];
      const float dx = r0.x - fx;
      const float cadx2 = r0.z * dx * dx, cbdx = r0.w * dx;
      float D0 = 0.0f, D1 = 0.0f, D2 = 0.0f, dop = 0.0f, dc0 = 0.0f, dc1 = 0.0f, dc2 = 0.0f;
      bool any = false, warp_any;  // warp_any: some lane of the warp took the Gaussian
      if constexpr (P == 2) {
        // both pixels through one instruction stream (paired FP32 operations,
        // the same values as the per-pixel code below): a pixel that does
        // not take this Gaussian keeps its state (selects) and adds zeros
        const float2 dy = psub(pbc(r0.y), make_float2(fy[0], fy[1]));
        const float2 pw = pfma(pbc(-0.5f), pfma(pmul(pbc(r1.x), dy), dy, pbc(cadx2)), pmul(pbc(-cbdx), dy));
        float G0 = 0.0f, a0 = 0.0f, G1 = 0.0f, a1 = 0.0f;
        const bool c0 = pos < last[0] && splat_alpha(pw.x, r2.y, r1.y, G0, a0);
        const bool c1 = pos < last[1] && splat_alpha(pw.y, r2.y, r1.y, G1, a1);
        warp_any = __any_sync(0xffffffffu, c0 || c1);
        if (warp_any) {
          const float2 G = make_float2(c0 ? G0 : 0.0f, c1 ? G1 : 0.0f);
          const float2 al = make_float2(c0 ? a0 : 0.0f, c1 ? a1 : 0.0f);
          const float2 om = psub(pbc(1.0f), al);  // >= 0.01
          const float2 inv = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
          const float2 Tn = pmul(make_float2(T[0], T[1]), inv);  // T before this Gaussian
          T[0] = c0 ? Tn.x : T[0];
          T[1] = c1 ? Tn.y : T[1];
          const float2 T2 = make_float2(T[0], T[1]);
          const float2 So = make_float2(S[0], S[1]);
          const float2 Sn = pfma(make_float2(la[0], la[1]), psub(make_float2(ls[0], ls[1]), So), So);
          S[0] = c0 ? Sn.x : S[0];
          S[1] = c1 ? Sn.y : S[1];
          const float2 g0v = make_float2(g0[0], g0[1]), g1v = make_float2(g1[0], g1[1]),
                       g2v = make_float2(g2[0], g2[1]);
          const float2 cg = pfma(pbc(r2.x), g2v, pfma(pbc(r1.w), g1v, pmul(pbc(r1.z), g0v)));
          la[0] = c0 ? al.x : la[0];
          la[1] = c1 ? al.y : la[1];
          ls[0] = c0 ? cg.x : ls[0];
          ls[1] = c1 ? cg.y : ls[1];
          const float2 w = pmul(al, T2);
          dc0 = fmaf(w.y, g0v.y, w.x * g0v.x);
          dc1 = fmaf(w.y, g1v.y, w.x * g1v.x);
          dc2 = fmaf(w.y, g2v.y, w.x * g2v.x);
          const float2 dal =
              pfma(make_float2(-gTf[0], -gTf[1]), inv, pmul(psub(cg, make_float2(S[0], S[1])), T2));
          const float2 oG = pmul(pbc(r1.y), G);  // alpha not clamped where o G <= 0.99
          const float2 dm = make_float2(c0 && oG.x <= kAlphaMax ? dal.x : 0.0f,
                                        c1 && oG.y <= kAlphaMax ? dal.y : 0.0f);
          dop = fmaf(dm.y, G.y, dm.x * G.x);
          const float2 dp = pmul(dm, al);
          const float2 e = pmul(dp, dy);
          D0 = dp.x + dp.y;
          D1 = e.x + e.y;
          D2 = fmaf(e.y, dy.y, e.x * dy.x);
        }
      } else {
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const float dy = r0.y - fy[k];
          const float power = splat_power(cadx2, cbdx, r1.x, dy);
          float G = 0.0f, alpha = 0.0f;
          const bool c = pos < last[k] && splat_alpha(power, r2.y, r1.y, G, alpha);
          if (__any_sync(0xffffffffu, c) && c) {
            any = true;
            const float inv = __fdividef(1.0f, 1.0f - alpha);  // 1 - alpha >= 0.01
            T[k] *= inv;                                       // T before this Gaussian
            S[k] = fmaf(la[k], ls[k] - S[k], S[k]);            // behind: previous contributor over the rest
            const float cg = fmaf(r2.x, g2[k], fmaf(r1.w, g1[k], r1.z * g0[k]));
            la[k] = alpha;
            ls[k] = cg;
            const float w = alpha * T[k];
            dc0 = fmaf(w, g0[k], dc0);
            dc1 = fmaf(w, g1[k], dc1);
            dc2 = fmaf(w, g2[k], dc2);
            const float dal = fmaf(-gTf[k], inv, (cg - S[k]) * T[k]);
            if (r1.y * G <= kAlphaMax) {  // alpha not clamped
              dop = fmaf(dal, G, dop);
              const float dp = dal * alpha;
              const float e = dp * dy;
              D0 += dp;
              D1 += e;
              D2 = fmaf(e, dy, D2);
            }
          }
        }
        warp_any = __any_sync(0xffffffffu, any);
      }
      if (warp_any) {
        // mean2d (u, v), conic (a, b, c), opacity, colour r, g; colour b apart
        float v[8];
        v[0] = -(r0.z * dx) * D0 - r0.w * D1;
        v[1] = -(r1.x * D1) - cbdx * D0;
        v[2] = -0.5f * dx * dx * D0;
        v[3] = -dx * D1;
        v[4] = -0.5f * D2;
        v[5] = dop;
        v[6] = dc0;
        v[7] = dc1;
        const float s8 = reduce8(v);
        const float sb = warp_sum(dc2);
        const int g = sg[buf][j];
        if (g >= 0 && adds) atomicAdd(gbase + (size_t)gstride * g, lane == 1 ? sb : s8);
      }
    }
  }
  cp_async_wait<0>();  // no copy outlives the CTA
}

// ---------------------------------------------------------------- host side

size_t raster_workspace(int n, int width, int height, bool reverse) {
  Carver c(nullptr);
  c.take<float4>((size_t)3 * (n > 0 ? n : 1));
  if (reverse) {
    const int64_t tiles = (int64_t)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile);
    c.take<int32_t>(2 * (size_t)(tiles > 0 ? tiles : 1));  // work key, order
  }
  return c.size();
}

size_t tile_order_workspace(int width, int height) {
  const int64_t tiles = (int64_t)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile);
  Carver c(nullptr);
  c.take<int32_t>((size_t)(tiles > 0 ? tiles : 1));
  return c.size();
}

// Work class of each tile for the reverse: the bit length of its longest
// pixel list (the reverse walks every pixel's list from its end).
__global__ void __launch_bounds__(256) k_tile_work(const int32_t* __restrict__ n_contrib, int W, int H, int TX,
                                                   int32_t* __restrict__ key) {
  __shared__ int wmax[8];
  const int tile = blockIdx.x, t = threadIdx.x;
  const int px = (tile % TX) * kTile + (t % kTile), py = (tile / TX) * kTile + (t / kTile);
  const int v = (px < W && py < H) ? n_contrib[py * W + px] : 0;
  const int m = __reduce_max_sync(0xffffffffu, v);
  if ((t & 31) == 0) wmax[t >> 5] = m;
  __syncthreads();
  if (t == 0) {
    int mm = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) mm = max(mm, wmax[i]);
    key[tile] = mm > 0 ? __clz(mm) : 32;  // smaller key = more work
  }
}

// Tiles ordered by increasing key (bucket sort over 33 classes, one CTA;
// the order inside a class is that of the atomics and does not matter: the
// tiles are independent).
__global__ void __launch_bounds__(1024) k_tile_order(const int32_t* __restrict__ key, int ntiles,
                                                     int32_t* __restrict__ order) {
  __shared__ int cnt[33], off[33];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int rounds = (ntiles + 1023) / 1024;
  for (int r = 0; r < rounds; ++r) {
    const int t = r * 1024 + threadIdx.x;
    const bool ok = t < ntiles;
    const int k = ok ? min(max(key[t], 0), 32) : 0;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? k : 64 + lane) & act;
    if (ok && lane == __ffs(peers) - 1) atomicAdd(&cnt[k], __popc(peers));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < 33; ++k) {
      off[k] = run;
      run += cnt[k];
    }
  }
  __syncthreads();
  for (int r = 0; r < rounds; ++r) {
    const int t = r * 1024 + threadIdx.x;
    const bool ok = t < ntiles;
    const int k = ok ? min(max(key[t], 0), 32) : 0;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? k : 64 + lane) & act;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (ok && lane == leader) base = atomicAdd(&off[k], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, ok ? leader : lane);
    if (ok) order[base + __popc(peers & ((1u << lane) - 1u))] = t;
  }
}

static hyrf_status pack(const hyrf_rasterize_args& a, float4* rec, cudaStream_t s) {
  int blocks = (a.n + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  if (blocks < 1) blocks = 1;
  HYRF_LAUNCH("k_pack", s,
              k_pack<<<blocks, 256, 0, s>>>(a.n_vis, a.n, a.mean2d, a.conic, a.alpha, a.color, rec));
  return HYRF_OK;
}

hyrf_status launch_tile_order(const hyrf_tile_order_args& a, void* ws, cudaStream_t s) {
  const int TX = (a.width + kTile - 1) / kTile, TY = (a.height + kTile - 1) / kTile;
  Carver c(ws);
  int32_t* key = c.take<int32_t>((size_t)TX * TY);
  HYRF_LAUNCH("k_tile_work", s, k_tile_work<<<TX * TY, 256, 0, s>>>(a.n_contrib, a.width, a.height, TX, key));
  HYRF_LAUNCH("k_tile_order", s, k_tile_order<<<1, 1024, 0, s>>>(key, TX * TY, a.order));
  return HYRF_OK;
}

hyrf_status launch_raster_fwd(const hyrf_rasterize_args& a, void* ws, cudaStream_t s) {
  const int TX = (a.width + kTile - 1) / kTile, TY = (a.height + kTile - 1) / kTile;
  Carver c(ws);
  float4* rec = c.take<float4>((size_t)3 * (a.n > 0 ? a.n : 1));
  if (a.records) rec = reinterpret_cast<float4*>(a.records);  // kept for the reverse
  hyrf_status st = pack(a, rec, s);
  if (st != HYRF_OK) return st;
  HYRF_LAUNCH("k_raster_fwd", s,
              k_raster_fwd<<<TX * TY, 256, 0, s>>>(a.ranges, a.vals, a.n, rec, a.width, a.height, TX, a.tile_order,
                                                   a.C_fg,
                                       a.T_final, a.n_contrib, a.status));
  return HYRF_OK;
}

hyrf_status launch_raster_bwd(const hyrf_rasterize_backward_args& b, void* ws, cudaStream_t s) {
  const hyrf_rasterize_args& a = b.fwd;
  const int TX = (a.width + kTile - 1) / kTile, TY = (a.height + kTile - 1) / kTile;
  Carver c(ws);
  float4* rec = c.take<float4>((size_t)3 * (a.n > 0 ? a.n : 1));
  int32_t* key = c.take<int32_t>((size_t)TX * TY);
  int32_t* order = c.take<int32_t>((size_t)TX * TY);
  if (a.records) {  // the forward's records
    rec = reinterpret_cast<float4*>(a.records);
  } else {
    hyrf_status st = pack(a, rec, s);
    if (st != HYRF_OK) return st;
  }
  if (a.tile_order) {
    order = const_cast<int32_t*>(a.tile_order);
  } else {
    HYRF_LAUNCH("k_tile_work", s, k_tile_work<<<TX * TY, 256, 0, s>>>(a.n_contrib, a.width, a.height, TX, key));
    HYRF_LAUNCH("k_tile_order", s, k_tile_order<<<1, 1024, 0, s>>>(key, TX * TY, order));
  }
  HYRF_LAUNCH("k_raster_bwd", s,
              k_raster_bwd<kBwdRasterWarps, kBwdRasterPixels>
              <<<TX * TY * kBwdCtasPerTile, 32 * kBwdRasterWarps, 0, s>>>(a.ranges, a.vals, a.n, rec, a.width, a.height, TX, order, a.T_final,
                                       a.n_contrib, b.d_C_fg, b.d_T_final, b.C, a.C_fg, b.d_mean2d,
                                       b.d_conic, b.d_alpha, b.d_color, a.status));
  return HYRF_OK;
}

}  // namespace hyrf
