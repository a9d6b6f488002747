// Field query (Sec. 3.2, Eqs. 2-7) and neural background (Sec. 3.3,
// Eqs. 10-11, App. A.2): FP32 CUDA-core kernels, forward and backward.
// Forward: for 16-level grids with 2 x 64 decoders the hash gather runs in
// its own full-occupancy kernel (k_gather_f32, gather.cu) and the decoders
// here read its f32 features (k_query_dec_f32, k_bg_dec_f32: register-tiled
// CTA-wide products) and their reverses (k_bg_dec_bwd_f32,
// k_query_dec_bwd_f32) likewise; other shapes use the fused kernels (gather
// and decoders in one thread per point). Backward
// kernels recompute the decoder activations, keep them in shared memory as
// [feature][point] tiles, and reduce the weight gradients per CTA into a
// private float32 slab (no atomics); one reduction kernel adds the slabs
// into the caller's gradient buffers. The field-query reverse runs on the
// visible rows with a non-zero upstream gradient only.
#include <cmath>
#include <type_traits>

#include "tc_ops.cuh"

// This file is compiled several times: part 0 holds the host-side dispatch,
// the shape-independent kernels and their launch wrappers; parts 1-3 each
// instantiate the templated kernels for one (levels, width, hidden layers,
// weight type) combination, so the instantiations compile in parallel.
#ifndef HYRF_FIELDS_PART
#define HYRF_FIELDS_PART 0
#endif

namespace hyrf {

size_t slab_bytes(const FieldsDev& F, bool geo);

// gather.cu: the hash gather with f32 features out (the FP32 split path).
hyrf_status launch_gather_f32(const FieldsDev& F, const CamDev& cam, const RowSource& S, int rows, float* Xg,
                              float* Xr, cudaStream_t s);

struct QueryFwdIO {
  int n;
  const float* pos;
  const float* alpha_e;
  const float* scale_e;
  const float* color_e;
  const int32_t* vis_ids;
  const int32_t* n_vis;
  float* alpha;
  float* scale;
  float* quat;
  float* color;
  int32_t* status;
};

struct QueryBwdIO {
  int n;
  const float* pos;
  const float* alpha_e;
  const float* scale_e;
  const float* color_e;
  const int32_t* vis_ids;
  const int32_t* n_vis;
  const float* d_alpha;
  const float* d_scale;
  const float* d_quat;
  const float* d_color;
  float* d_pos;
  float* d_alpha_e;
  float* d_scale_e;
  float* d_color_e;
  float* g_geo_table;
  float* g_rad_table;
  float loss_scale;
  int32_t* status;
  // Optional list of the visible rows to process (those with a non-zero
  // upstream gradient; the others add exactly zero) and its device count.
  const int32_t* list;
  const int32_t* n_list;
};

__device__ __forceinline__ void cam_center(const CamDev& c, float pc[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) pc[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
}

constexpr int kFwdThreads = 128;
constexpr int kFwdPitch = kFwdThreads + 1;

// Eq. 7: the decoder outputs (go: alpha_n, s_n[3], r_n[4]; co: c_n[3])
// aggregated with the explicit parameters of Gaussian g into visible row i.
__device__ __forceinline__ void aggregate(const QueryFwdIO& io, int i, int g, const float* go, const float* co) {
  io.alpha[i] = sigmoidf_(go[0] + (io.alpha_e ? io.alpha_e[g] : 0.0f));
  const float se = io.scale_e ? io.scale_e[g] : 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) io.scale[3 * i + k] = sigmoidf_(go[1 + k] + se);
  const float rn = sqrtf(go[4] * go[4] + go[5] * go[5] + go[6] * go[6] + go[7] * go[7]);
  const float den = fmaxf(rn, 1e-12f);
#pragma unroll
  for (int k = 0; k < 4; ++k) io.quat[4 * i + k] = go[4 + k] / den;
#pragma unroll
  for (int k = 0; k < 3; ++k) io.color[3 * i + k] = sigmoidf_(co[k] + (io.color_e ? io.color_e[3 * (int64_t)g + k] : 0.0f));
}

// N consecutive floats (16-byte aligned) into registers.
template <int N>
__device__ __forceinline__ void load_row(const float* __restrict__ src, float* x) {
  static_assert(N % 4 == 0, "row length");
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int k = 0; k < N / 4; ++k) {
    const float4 v = __ldcs(s4 + k);
    x[4 * k] = v.x;
    x[4 * k + 1] = v.y;
    x[4 * k + 2] = v.z;
    x[4 * k + 3] = v.w;
  }
}

template <int NL, int WID, int NH, class WT>
__global__ void __launch_bounds__(kFwdThreads) k_query_fwd(FieldsDev F, CamDev cam, QueryFwdIO io) {
  constexpr int NG = 2 * NL, NC = 2 * NL + kPEPad;
  __shared__ float hid[WID * kFwdPitch];
  float* col = hid + threadIdx.x;
  const int nv = min(*io.n_vis, io.n);
  float pc[3];
  cam_center(cam, pc);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int g = io.vis_ids[i];
    if (g < 0 || g >= io.n) {
      set_status(io.status, HYRF_ERR_BOUNDS);
      continue;
    }
    const float p[3] = {io.pos[3 * (int64_t)g], io.pos[3 * (int64_t)g + 1], io.pos[3 * (int64_t)g + 2]};
    float y[3];
    contract_p(F, p, y, nullptr);
    float go[8];
    {
      float fg[NG];
      encode<NL>(F.geo, y, fg);
      mlp_fwd<NG, WID, NH, 8, WT>(F.gm, fg, col, kFwdPitch, go);
    }
    float co[3];
    {
      float fc[NC];
      encode<NL>(F.rad, y, fc);
      float v[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
      const float vn = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      const float dir[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
      pos_enc(dir, fc + NG);
      mlp_fwd<NC, WID, NH, 3, WT>(F.cm, fc, col, kFwdPitch, co);
    }
    aggregate(io, i, g, go, co);
  }
}

// Reverse of a decoder whose activations are in smem (act: input rows
// [0, IN), hidden rows after it) and whose output gradient dz_out is given;
// updates the CTA slab and returns dL/dinput in dx. All threads of the CTA
// must call it (it synchronises).
template <int IN, int WID, int NH, int OUT, class WT>
__device__ __forceinline__ void decoder_bwd(const MlpDev& m, const float* act, float* dzb,
                                            const float* dz_out, float* slab, const SlabLayout& SL,
                                            int dec, float* dx) {
  const int t = threadIdx.x;
  const float* hl = act + (IN + (NH - 1) * WID) * kActPitch;
#pragma unroll
  for (int r = 0; r < OUT; ++r) dzb[r * kActPitch + t] = dz_out[r];
  __syncthreads();
  cta_dw<OUT, WID>(dzb, hl, slab + SL.off_W[dec][NH], slab + SL.off_b[dec][NH]);
  float dh[WID];
  dense_dx_col<WID, OUT>(wptr<WT>(m, NH), dzb + t, kActPitch, dh);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < WID; ++r) dzb[r * kActPitch + t] = hl[r * kActPitch + t] > 0.0f ? dh[r] : 0.0f;
  __syncthreads();
  if constexpr (NH == 2) {
    const float* h1 = act + IN * kActPitch;
    cta_dw<WID, WID>(dzb, h1, slab + SL.off_W[dec][1], slab + SL.off_b[dec][1]);
    dense_dx_col<WID, WID>(wptr<WT>(m, 1), dzb + t, kActPitch, dh);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < WID; ++r) dzb[r * kActPitch + t] = h1[r * kActPitch + t] > 0.0f ? dh[r] : 0.0f;
    __syncthreads();
  }
  cta_dw<WID, IN>(dzb, act, slab + SL.off_W[dec][0], slab + SL.off_b[dec][0]);
  dense_dx_col<IN, WID>(wptr<WT>(m, 0), dzb + t, kActPitch, dx);
  __syncthreads();
}

// Forward of a decoder storing its input and hidden activations in smem.
template <int IN, int WID, int NH, int OUT, class WT>
__device__ __forceinline__ void decoder_fwd_store(const MlpDev& m, const float* x, float* act,
                                                  float* out) {
  const int t = threadIdx.x;
#pragma unroll
  for (int r = 0; r < IN; ++r) act[r * kActPitch + t] = x[r];
  float* h1 = act + IN * kActPitch + t;
  dense_col<IN, WID>(wptr<WT>(m, 0), m.b[0], x, h1, kActPitch);
  float h[WID];
  load_col<WID>(h1, kActPitch, h);
  if constexpr (NH == 2) {
    float* h2 = act + (IN + WID) * kActPitch + t;
    dense_col<WID, WID>(wptr<WT>(m, 1), m.b[1], h, h2, kActPitch);
    load_col<WID>(h2, kActPitch, h);
  }
  dense_out<WID, OUT>(wptr<WT>(m, NH), m.b[NH], h, out);
}

template <int NL, int WID, int NH>
constexpr int query_bwd_smem_floats() {
  return (2 * NL + kPEPad + NH * WID) * kActPitch + WID * kActPitch;
}

template <int NL, int WID, int NH, class WT>
__global__ void __launch_bounds__(kBwdThreads) k_query_bwd(FieldsDev F, CamDev cam, QueryBwdIO io,
                                                           SlabLayout SL, float* slabs) {
  extern __shared__ float sm[];
  constexpr int NG = 2 * NL, NC = 2 * NL + kPEPad;
  float* act = sm;
  float* dzb = sm + (NC + NH * WID) * kActPitch;
  float* slab = slabs + (size_t)blockIdx.x * SL.total;
  const int t = threadIdx.x;
  const int nv = min(*io.n_vis, io.n);
  const int nr = io.list ? min(*io.n_list, nv) : nv;
  const float ls = io.loss_scale, inv_ls = 1.0f / io.loss_scale;
  float pc[3];
  cam_center(cam, pc);
  for (int base = blockIdx.x * kBwdThreads; base < nr; base += gridDim.x * kBwdThreads) {
    bool ok = base + t < nr;
    const int i = ok ? (io.list ? io.list[base + t] : base + t) : 0;
    if (ok && (i < 0 || i >= nv)) {
      set_status(io.status, HYRF_ERR_BOUNDS);
      ok = false;
    }
    int g = ok ? io.vis_ids[i] : 0;
    if (ok && (g < 0 || g >= io.n)) {
      set_status(io.status, HYRF_ERR_BOUNDS);
      ok = false;
    }
    float p[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      p[k] = ok ? io.pos[3 * (int64_t)g + k] : F.lo[k] + 1.0f / F.sx[k];  // box centre when idle
    float y[3], J[9];
    contract_p(F, p, y, J);
    float da = 0.0f, ds[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dcol[3] = {0, 0, 0};
    float ae = 0.0f, se = 0.0f, ce[3] = {0, 0, 0};
    if (ok) {
      da = io.d_alpha[i] * ls;
#pragma unroll
      for (int k = 0; k < 3; ++k) ds[k] = io.d_scale[3 * i + k] * ls;
#pragma unroll
      for (int k = 0; k < 4; ++k) dq[k] = io.d_quat[4 * i + k] * ls;
#pragma unroll
      for (int k = 0; k < 3; ++k) dcol[k] = io.d_color[3 * i + k] * ls;
      ae = io.alpha_e ? io.alpha_e[g] : 0.0f;
      se = io.scale_e ? io.scale_e[g] : 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) ce[k] = io.color_e ? io.color_e[3 * (int64_t)g + k] : 0.0f;
    }
    float dy[3] = {0.0f, 0.0f, 0.0f};
    // ---------------- geometry decoder (Eq. 4) and the reverse of Eq. 7
    {
      float x0[NG], out[8], dz8[8];
      encode<NL>(F.geo, y, x0);
      decoder_fwd_store<NG, WID, NH, 8, WT>(F.gm, x0, act, out);
      const float a = sigmoidf_(out[0] + ae);
      dz8[0] = da * a * (1.0f - a);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float s = sigmoidf_(out[1 + k] + se);
        dz8[1 + k] = ds[k] * s * (1.0f - s);
      }
      const float rn = sqrtf(out[4] * out[4] + out[5] * out[5] + out[6] * out[6] + out[7] * out[7]);
      if (rn > 1e-12f) {
        float qd = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) qd += out[4 + k] / rn * dq[k];
#pragma unroll
        for (int k = 0; k < 4; ++k) dz8[4 + k] = (dq[k] - out[4 + k] / rn * qd) / rn;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) dz8[4 + k] = dq[k] / 1e-12f;
      }
      if (!ok) {
#pragma unroll
        for (int k = 0; k < 8; ++k) dz8[k] = 0.0f;
      }
      if (ok) {
        if (io.d_alpha_e) io.d_alpha_e[g] += dz8[0] * inv_ls;
        if (io.d_scale_e) io.d_scale_e[g] += (dz8[1] + dz8[2] + dz8[3]) * inv_ls;
      }
      float dx[NG];
      decoder_bwd<NG, WID, NH, 8, WT>(F.gm, act, dzb, dz8, slab, SL, 0, dx);
      if (ok) {
#pragma unroll
        for (int k = 0; k < NG; ++k) dx[k] *= inv_ls;
        encode_bwd<NL>(F.geo, y, dx, io.g_geo_table, dy);
      }
    }
    // ---------------- colour decoder (Eqs. 5-6) and the reverse of Eq. 7
    float v[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
    const float vn = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const float dir[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
    float dp[3] = {0.0f, 0.0f, 0.0f};
    {
      float x0[NC], out[3], dz3[3];
      encode<NL>(F.rad, y, x0);
      pos_enc(dir, x0 + NG);
      decoder_fwd_store<NC, WID, NH, 3, WT>(F.cm, x0, act, out);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float c = sigmoidf_(out[k] + ce[k]);
        dz3[k] = ok ? dcol[k] * c * (1.0f - c) : 0.0f;
      }
      if (ok) {
#pragma unroll
        if (io.d_color_e)
          for (int k = 0; k < 3; ++k) io.d_color_e[3 * (int64_t)g + k] += dz3[k] * inv_ls;
      }
      float dx[NC];
      decoder_bwd<NC, WID, NH, 3, WT>(F.cm, act, dzb, dz3, slab, SL, 1, dx);
      if (ok) {
#pragma unroll
        for (int k = 0; k < NC; ++k) dx[k] *= inv_ls;
        encode_bwd<NL>(F.rad, y, dx, io.g_rad_table, dy);
        float ddir[3];
        pos_enc_bwd(dir, dx + NG, ddir);
        const float dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) dp[k] = (ddir[k] - dir[k] * dd) / vn;
      }
    }
    if (ok) {
#pragma unroll
      for (int j = 0; j < 3; ++j)
        io.d_pos[3 * (int64_t)g + j] += dp[j] + J[j] * dy[0] + J[3 + j] * dy[1] + J[6 + j] * dy[2];
    }
  }
}


#if HYRF_FIELDS_PART == 0
// Element e of every slab, summed over the slab range of this CTA row
// (blockIdx.y of gridDim.y parts) and added atomically to the target: the
// parts and other reverse calls accumulating into the same weights add in
// any order.
__global__ void k_slab_reduce(const float* __restrict__ slabs, int nslabs, SlabLayout SL,
                              SlabTargets T, float scale) {
  const int per = (nslabs + gridDim.y - 1) / gridDim.y;
  const int c0 = blockIdx.y * per, c1 = min(nslabs, c0 + per);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < SL.total; e += gridDim.x * blockDim.x) {
    float* dst = nullptr;
    for (int d = 0; d < 2; ++d)
      for (int l = 0; l < 3; ++l) {
        if (e >= SL.off_W[d][l] && e < SL.off_W[d][l] + SL.n_W[d][l] && T.W[d][l])
          dst = T.W[d][l] + (e - SL.off_W[d][l]);
        if (e >= SL.off_b[d][l] && e < SL.off_b[d][l] + SL.n_b[d][l] && T.b[d][l])
          dst = T.b[d][l] + (e - SL.off_b[d][l]);
      }
    if (!dst) continue;
    float s = 0.0f;
    for (int c = c0; c < c1; ++c) s += slabs[(size_t)c * SL.total + e];
    if (c1 > c0) atomicAdd(dst, s * scale);
  }
}
#endif

// ---------------------------------------------------------------- background (Eqs. 10-11)

// Pixel (i, j): hit point p_s of the ray with the sphere |x| = r in the
// normalised box space (App. A.2, positive root) and the unit world-space
// ray direction.
__device__ __forceinline__ void bg_ray(const CamDev& c, const FieldsDev& F, float radius, int i, int j,
                                       float ps[3], float dirw[3]) {
  float oc[3];
  cam_center(c, oc);
  const float dc[3] = {((float)i + 0.5f - c.cx) / c.fx, ((float)j + 0.5f - c.cy) / c.fy, 1.0f};
  float on[3], dn[3], dw[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dw[k] = c.R[k] * dc[0] + c.R[3 + k] * dc[1] + c.R[6 + k] * dc[2];
    on[k] = (oc[k] - F.lo[k]) * F.sx[k] - 1.0f;
    dn[k] = dw[k] * F.sx[k];
  }
  const float A = dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2];
  const float B = 2.0f * (on[0] * dn[0] + on[1] * dn[1] + on[2] * dn[2]);
  const float C = on[0] * on[0] + on[1] * on[1] + on[2] * on[2] - radius * radius;
  const float t = (-B + sqrtf(B * B - 4.0f * A * C)) / (2.0f * A);
#pragma unroll
  for (int k = 0; k < 3; ++k) ps[k] = on[k] + t * dn[k];
  const float nd = sqrtf(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) dirw[k] = dw[k] / nd;
}

// Equirectangular texel (a, b): unit direction and contracted point r * dir.
__device__ __forceinline__ void texel_point(int a, int b, int Hb, int Wb, float radius, float y[3],
                                            float dir[3]) {
  const float phi = ((float)b + 0.5f) / (float)Wb * 6.28318530717959f - 3.14159265358979f;
  const float th = ((float)a + 0.5f) / (float)Hb * 3.14159265358979f - 1.57079632679490f;
  float sp, cp, st, ct;
  sincosf(phi, &sp, &cp);
  sincosf(th, &st, &ct);
  dir[0] = ct * sp;
  dir[1] = st;
  dir[2] = ct * cp;
  const float x[3] = {radius * dir[0], radius * dir[1], radius * dir[2]};
  contract_n(x, y);
}

// Bilinear footprint of the direction of p_s in the map (wrap in longitude,
// clamp in latitude).
struct MapTap {
  int a[2], b[2];
  float wa[2], wb[2];
};

__device__ __forceinline__ MapTap map_tap(const float ps[3], int Hb, int Wb) {
  const float n = sqrtf(ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2]);
  const float w1 = fminf(1.0f, fmaxf(-1.0f, ps[1] / n));
  const float th = asinf(w1);
  const float phi = atan2f(ps[0] / n, ps[2] / n);
  const float bf = (phi + 3.14159265358979f) / 6.28318530717959f * (float)Wb - 0.5f;
  const float af = (th + 1.57079632679490f) / 3.14159265358979f * (float)Hb - 0.5f;
  const float b0 = floorf(bf), a0 = floorf(af);
  MapTap m;
  m.wb[1] = bf - b0;
  m.wb[0] = 1.0f - m.wb[1];
  m.wa[1] = af - a0;
  m.wa[0] = 1.0f - m.wa[1];
  const int ib = (int)b0, ia = (int)a0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    m.b[k] = ((ib + k) % Wb + Wb) % Wb;
    m.a[k] = min(Hb - 1, max(0, ia + k));
  }
  return m;
}

// Background colour at contracted point y with view direction dir.
template <int NL, int WID, int NH, class WT>
__device__ __forceinline__ void bg_color(const FieldsDev& F, const float y[3], const float dir[3],
                                         float* col, float cs[3]) {
  constexpr int NG = 2 * NL, NC = NG + kPEPad;
  float x0[NC], out[3];
  encode<NL>(F.rad, y, x0);
  pos_enc(dir, x0 + NG);
  mlp_fwd<NC, WID, NH, 3, WT>(F.cm, x0, col, kFwdPitch, out);
#pragma unroll
  for (int k = 0; k < 3; ++k) cs[k] = sigmoidf_(out[k]);
}

template <int NL, int WID, int NH, class WT>
__global__ void __launch_bounds__(kFwdThreads) k_bg_exact_fwd(FieldsDev F, CamDev cam, float radius,
                                                              const float* __restrict__ C_fg,
                                                              const float* __restrict__ T_final,
                                                              float* __restrict__ C) {
  __shared__ float hid[WID * kFwdPitch];
  float* col = hid + threadIdx.x;
  const int P = cam.W * cam.H;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const int i = p % cam.W, j = p / cam.W;
    float ps[3], dir[3], y[3], cs[3];
    bg_ray(cam, F, radius, i, j, ps, dir);
    contract_n(ps, y);
    bg_color<NL, WID, NH, WT>(F, y, dir, col, cs);
    const float T = T_final[p];
#pragma unroll
    for (int k = 0; k < 3; ++k) C[3 * (int64_t)p + k] = C_fg[3 * (int64_t)p + k] + T * cs[k];
  }
}

// ---------------------------------------------------------------- FP32 decoders, register-tiled

// Decoders of the FP32 split path (2 x 64 hidden units) as a CTA-wide
// product: 256 threads take tiles of 256 rows; a tile's activations sit in
// shared memory feature-major (act[feature][row]) and the weights
// transposed (Wt[input][output]), staged once per CTA. A hidden layer is a
// 256 x 64 product in 8 x 8 register blocks: per input feature a thread
// reads 8 activations and 8 weights (four 16-byte loads) for 64 FMAs. Each
// output sums its products in input order from zero and then adds the
// bias, as dense_col and dot_row do, so the values equal those of the
// one-thread-per-row decoders bit for bit.
constexpr int kDecRows = 256;            // rows per tile = threads per CTA
constexpr int kDecPitch = kDecRows + 4;  // floats per feature row of act

template <int IN, int OP>
struct DecSmemF32 {
  static constexpr int act = 0, w0 = act + 64 * kDecPitch, w1 = w0 + IN * 64, w2 = w1 + 64 * 64,
                       b0 = w2 + 64 * OP, b1 = b0 + 64, b2 = b1 + 64, floats = b2 + OP;
};

// Wt[i][o] = W[o][i] (W row-major [rows_real][IN]), zero for o >= rows_real.
template <int OP, int IN>
__device__ __forceinline__ void stage_wt(float* Wt, const float* __restrict__ W, int rows_real) {
  for (int e = threadIdx.x; e < OP * IN; e += blockDim.x) {
    const int o = e / IN, i = e % IN;
    Wt[i * OP + o] = o < rows_real ? __ldg(W + o * IN + i) : 0.0f;
  }
}

// Stage a decoder's three layers (weights transposed, biases; output
// padded to OP) into the tile layout L.
template <int IN, int OP, int OUT>
__device__ __forceinline__ void stage_decoder(float* sm, const MlpDev& m) {
  using L = DecSmemF32<IN, OP>;
  stage_wt<64, IN>(sm + L::w0, static_cast<const float*>(m.W[0]), 64);
  stage_wt<64, 64>(sm + L::w1, static_cast<const float*>(m.W[1]), 64);
  stage_wt<OP, 64>(sm + L::w2, static_cast<const float*>(m.W[2]), OUT);
  for (int e = threadIdx.x; e < 64; e += blockDim.x) {
    sm[L::b0 + e] = m.b[0][e];
    sm[L::b1 + e] = m.b[1][e];
  }
  for (int e = threadIdx.x; e < OP; e += blockDim.x) sm[L::b2 + e] = e < OUT ? m.b[2][e] : 0.0f;
}

// act[o][r] = ReLU(sum_i Wt[i][o] act[i][r] + b[o]), o < 64, for the
// tile's 256 rows (in place: every thread reads the whole input first).
template <int IN>
__device__ __forceinline__ void dec_hidden(float* act, const float* Wt, const float* b) {
  const int t = threadIdx.x, r0 = 8 * (t & 31), o0 = 8 * (t >> 5);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 2
  for (int k = 0; k < IN; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(act + k * kDecPitch + r0);
    const float4 a1 = *reinterpret_cast<const float4*>(act + k * kDecPitch + r0 + 4);
    const float4 w0 = *reinterpret_cast<const float4*>(Wt + k * 64 + o0);
    const float4 w1 = *reinterpret_cast<const float4*>(Wt + k * 64 + o0 + 4);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(w[j], a[i], acc[i][j]);
  }
  __syncthreads();  // the whole input has been read
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bj = b[o0 + j];
    float* dst = act + (o0 + j) * kDecPitch + r0;
    *reinterpret_cast<float4*>(dst) =
        make_float4(fmaxf(acc[0][j] + bj, 0.0f), fmaxf(acc[1][j] + bj, 0.0f), fmaxf(acc[2][j] + bj, 0.0f),
                    fmaxf(acc[3][j] + bj, 0.0f));
    *reinterpret_cast<float4*>(dst + 4) =
        make_float4(fmaxf(acc[4][j] + bj, 0.0f), fmaxf(acc[5][j] + bj, 0.0f), fmaxf(acc[6][j] + bj, 0.0f),
                    fmaxf(acc[7][j] + bj, 0.0f));
  }
  __syncthreads();
}

// Output layer for this thread's row: out[o] = sum_k Wt2[k][o] act[k][r] + b[o].
template <int OP>
__device__ __forceinline__ void dec_out(const float* act, const float* Wt2, const float* b2, float* out) {
  const int r = threadIdx.x;
  float acc[OP];
#pragma unroll
  for (int o = 0; o < OP; ++o) acc[o] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < 64; ++k) {
    const float h = act[k * kDecPitch + r];
#pragma unroll
    for (int q = 0; q < OP / 4; ++q) {
      const float4 w = *reinterpret_cast<const float4*>(Wt2 + k * OP + 4 * q);
      acc[4 * q] = fmaf(w.x, h, acc[4 * q]);
      acc[4 * q + 1] = fmaf(w.y, h, acc[4 * q + 1]);
      acc[4 * q + 2] = fmaf(w.z, h, acc[4 * q + 2]);
      acc[4 * q + 3] = fmaf(w.w, h, acc[4 * q + 3]);
    }
  }
#pragma unroll
  for (int o = 0; o < OP; ++o) out[o] = acc[o] + b2[o];
}

// Field query, one decoder per launch (GEO: the geometry decoder -> alpha,
// scale, rotation; else the colour decoder -> colour), on the features
// k_gather_f32 wrote (X [n_vis][32]); Eq. 7 as aggregate().
template <bool GEO>
__global__ void __launch_bounds__(kDecRows, 2) k_query_dec_f32(FieldsDev F, CamDev cam, QueryFwdIO io,
                                                             const float* __restrict__ X) {
  constexpr int IN = GEO ? 32 : 32 + kPEPad, OP = GEO ? 8 : 4, OUT = GEO ? 8 : 3;
  using L = DecSmemF32<IN, OP>;
  extern __shared__ __align__(16) float smf[];
  float* act = smf + L::act;
  stage_decoder<IN, OP, OUT>(smf, GEO ? F.gm : F.cm);
  const int t = threadIdx.x;
  const int nv = min(*io.n_vis, io.n);
  const int ntile = (nv + kDecRows - 1) / kDecRows;
  float pc[3];
  cam_center(cam, pc);
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int i = tile * kDecRows + t;
    int g = i < nv ? io.vis_ids[i] : -1;
    if (i < nv && (g < 0 || g >= io.n)) {
      set_status(io.status, HYRF_ERR_BOUNDS);
      g = -1;
    }
    // this row's input -> column t of act (zeros for rows without a point)
    {
      float x[32];
      if (g >= 0) load_row<32>(X + (size_t)i * 32, x);
#pragma unroll
      for (int k = 0; k < 32; ++k) act[k * kDecPitch + t] = g >= 0 ? x[k] : 0.0f;
    }
    if constexpr (!GEO) {
      float pe[kPEPad];
      const float p[3] = {g >= 0 ? io.pos[3 * (int64_t)g] : pc[0] + 1.0f,
                          g >= 0 ? io.pos[3 * (int64_t)g + 1] : pc[1], g >= 0 ? io.pos[3 * (int64_t)g + 2] : pc[2]};
      float v[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
      const float vn = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      const float dir[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
      pos_enc(dir, pe);
#pragma unroll
      for (int k = 0; k < kPEPad; ++k) act[(32 + k) * kDecPitch + t] = pe[k];
    }
    __syncthreads();
    dec_hidden<IN>(act, smf + L::w0, smf + L::b0);
    dec_hidden<64>(act, smf + L::w1, smf + L::b1);
    float o[OP];
    dec_out<OP>(act, smf + L::w2, smf + L::b2, o);
    if (g >= 0) {
      if constexpr (GEO) {
        io.alpha[i] = sigmoidf_(o[0] + (io.alpha_e ? io.alpha_e[g] : 0.0f));
        const float se = io.scale_e ? io.scale_e[g] : 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) io.scale[3 * i + k] = sigmoidf_(o[1 + k] + se);
        const float rn = sqrtf(o[4] * o[4] + o[5] * o[5] + o[6] * o[6] + o[7] * o[7]);
        const float den = fmaxf(rn, 1e-12f);
#pragma unroll
        for (int k = 0; k < 4; ++k) io.quat[4 * i + k] = o[4 + k] / den;
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          io.color[3 * i + k] = sigmoidf_(o[k] + (io.color_e ? io.color_e[3 * (int64_t)g + k] : 0.0f));
      }
    }
    __syncthreads();  // act is rewritten by the next tile
  }
}

// Exact background (Eq. 11) on the features k_gather_f32 wrote at every
// pixel's sphere hit (Xb [W H][32]): C = C_fg + T_final sigmoid(decoder).
// NF: features per row (2 x 16 levels).
template <int NF>
__global__ void __launch_bounds__(kDecRows, 2) k_bg_dec_f32(FieldsDev F, CamDev cam, float radius,
                                                          const float* __restrict__ Xb,
                                                          const float* __restrict__ C_fg,
                                                          const float* __restrict__ T_final,
                                                          float* __restrict__ C) {
  static_assert(NF == 32, "16-level grids");
  constexpr int IN = NF + kPEPad, OP = 4;
  using L = DecSmemF32<IN, OP>;
  extern __shared__ __align__(16) float smf[];
  float* act = smf + L::act;
  stage_decoder<IN, OP, 3>(smf, F.cm);
  const int t = threadIdx.x;
  const int P = cam.W * cam.H;
  const int ntile = (P + kDecRows - 1) / kDecRows;
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int p = tile * kDecRows + t;
    const bool ok = p < P;
    {
      float x[32];
      if (ok) load_row<32>(Xb + (size_t)p * 32, x);
#pragma unroll
      for (int k = 0; k < 32; ++k) act[k * kDecPitch + t] = ok ? x[k] : 0.0f;
      float ps[3], dir[3], pe[kPEPad];
      const int q = ok ? p : 0;
      bg_ray(cam, F, radius, q % cam.W, q / cam.W, ps, dir);
      pos_enc(dir, pe);
#pragma unroll
      for (int k = 0; k < kPEPad; ++k) act[(32 + k) * kDecPitch + t] = pe[k];
    }
    __syncthreads();
    dec_hidden<IN>(act, smf + L::w0, smf + L::b0);
    dec_hidden<64>(act, smf + L::w1, smf + L::b1);
    float o[OP];
    dec_out<OP>(act, smf + L::w2, smf + L::b2, o);
    if (ok) {
      const float T = T_final[p];
#pragma unroll
      for (int k = 0; k < 3; ++k) C[3 * (int64_t)p + k] = C_fg[3 * (int64_t)p + k] + T * sigmoidf_(o[k]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- FP32 background reverse, register-tiled

// Reverse of the exact background's colour decoder on 128-pixel tiles
// (256 threads, one persistent CTA per SM): the forward is recomputed into
// shared memory (input X, H1, H2 feature-major), then dZ flows back layer by
// layer through the same tile; every product (forward, W^T dZ, dZ A^T) is a
// CTA-wide product in register blocks. The weight and bias gradients stay
// in registers over all of the CTA's tiles and are added to its slab once.
constexpr int kBgbRows = 128;             // pixels per tile
constexpr int kBgbPitch = kBgbRows + 4;   // floats per feature row of a tile buffer

struct BgbSmem {  // offsets in floats
  static constexpr int X = 0, H1 = X + 64 * kBgbPitch, H2 = H1 + 64 * kBgbPitch, DZ = H2 + 64 * kBgbPitch,
                       Wt0 = DZ + 64 * kBgbPitch, Wt1 = Wt0 + 64 * 64, W0 = Wt1 + 64 * 64, W1 = W0 + 64 * 64,
                       W2 = W1 + 64 * 64, Wt2 = W2 + 4 * 64, b0 = Wt2 + 64 * 4, b1 = b0 + 64, b2 = b1 + 64,
                       floats = b2 + 4;
};

// acc[i][j] = sum_k Wk[k][o0 + j] A[k][r0 + i], k < K (Wk row pitch WP, A row
// pitch kBgbPitch), in k order from zero.
template <int K, int BO, int WP = 64>
__device__ __forceinline__ void bgb_prod(const float* A, const float* Wk, int r0, int o0, float (&acc)[8][BO]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < BO; ++j) acc[i][j] = 0.0f;
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(A + k * kBgbPitch + r0);
    const float4 a1 = *reinterpret_cast<const float4*>(A + k * kBgbPitch + r0 + 4);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    float w[BO];
    if constexpr (BO == 4) {
      const float4 v = *reinterpret_cast<const float4*>(Wk + k * WP + o0);
      w[0] = v.x;
      w[1] = v.y;
      w[2] = v.z;
      w[3] = v.w;
    } else {
      const float2 v = *reinterpret_cast<const float2*>(Wk + k * WP + o0);
      w[0] = v.x;
      w[1] = v.y;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < BO; ++j) acc[i][j] = fmaf(w[j], a[i], acc[i][j]);
  }
}

// dW[o0 + a][i0 + c] += sum_r dZ[o0 + a][r] A[i0 + c][r] over the tile's rows.
template <int BA = 4, int BC = 4>
__device__ __forceinline__ void bgb_dw(const float* DZ, const float* A, int o0, int i0, float (&dw)[BA][BC]) {
#pragma unroll 2
  for (int r = 0; r < kBgbRows; r += 4) {
    float4 d[BA], x[BC];
#pragma unroll
    for (int a = 0; a < BA; ++a) d[a] = *reinterpret_cast<const float4*>(DZ + (o0 + a) * kBgbPitch + r);
#pragma unroll
    for (int c = 0; c < BC; ++c) x[c] = *reinterpret_cast<const float4*>(A + (i0 + c) * kBgbPitch + r);
#pragma unroll
    for (int a = 0; a < BA; ++a)
#pragma unroll
      for (int c = 0; c < BC; ++c) {
        dw[a][c] = fmaf(d[a].x, x[c].x, dw[a][c]);
        dw[a][c] = fmaf(d[a].y, x[c].y, dw[a][c]);
        dw[a][c] = fmaf(d[a].z, x[c].z, dw[a][c]);
        dw[a][c] = fmaf(d[a].w, x[c].w, dw[a][c]);
      }
  }
}

// sum_r buf[row][r] over the tile's rows.
__device__ __forceinline__ float bgb_rowsum(const float* buf, int row) {
  float s = 0.0f;
#pragma unroll 4
  for (int r = 0; r < kBgbRows; r += 4) {
    const float4 v = *reinterpret_cast<const float4*>(buf + row * kBgbPitch + r);
    s += (v.x + v.y) + (v.z + v.w);
  }
  return s;
}

// NF: features per pixel (2 x 16 levels). dXb receives dL/dX / loss_scale;
// the slab (colour decoder's entries, pre-zeroed) dL/dW * loss_scale.
template <int NF>
__global__ void __launch_bounds__(256, 1) k_bg_dec_bwd_f32(FieldsDev F, CamDev cam, float radius,
                                                         const float* __restrict__ T_final,
                                                         const float* __restrict__ dC, float* __restrict__ dC_fg,
                                                         float* __restrict__ dT, float loss_scale, SlabLayout SL,
                                                         float* __restrict__ slabs, const float* __restrict__ Xb,
                                                         float* __restrict__ dXb) {
  static_assert(NF == 32 && NF + kPEPad == 64, "16-level grids, 2 x 64 decoder");
  using L = BgbSmem;
  extern __shared__ __align__(16) float smf[];
  float *X = smf + L::X, *H1 = smf + L::H1, *H2 = smf + L::H2, *DZ = smf + L::DZ;
  const int t = threadIdx.x;
  {
    const float* W0g = static_cast<const float*>(F.cm.W[0]);
    const float* W1g = static_cast<const float*>(F.cm.W[1]);
    const float* W2g = static_cast<const float*>(F.cm.W[2]);
    for (int e = t; e < 64 * 64; e += 256) {
      const int o = e >> 6, i = e & 63;
      const float v0 = __ldg(W0g + e), v1 = __ldg(W1g + e);
      smf[L::W0 + e] = v0;
      smf[L::Wt0 + i * 64 + o] = v0;
      smf[L::W1 + e] = v1;
      smf[L::Wt1 + i * 64 + o] = v1;
    }
    {
      const int o = t >> 6, i = t & 63;
      const float v = o < 3 ? __ldg(W2g + o * 64 + i) : 0.0f;
      smf[L::W2 + t] = v;
      smf[L::Wt2 + i * 4 + o] = v;
    }
    if (t < 64) {
      smf[L::b0 + t] = F.cm.b[0][t];
      smf[L::b1 + t] = F.cm.b[1][t];
    }
    if (t < 4) smf[L::b2 + t] = t < 3 ? F.cm.b[2][t] : 0.0f;
  }
  const int P = cam.W * cam.H;
  const int ntile = (P + kBgbRows - 1) / kBgbRows;
  const float inv_ls = 1.0f / loss_scale;
  const int r0 = 8 * (t & 15), og = t >> 4;  // product blocks: rows r0.., outputs 4 og.. (2 og.. for dX)
  const int dob = t >> 4, dib = t & 15;      // weight-gradient blocks: outputs 4 dob.., inputs 4 dib..
  float dw0[4][4], dw1[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) dw0[a][c] = dw1[a][c] = 0.0f;
  float dw2 = 0.0f;  // output t >> 6, input t & 63
  float db = 0.0f;   // t < 64: b1[t]; t < 128: b0[t - 64]; t < 131: b2[t - 128]
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int pbase = tile * kBgbRows;
    // inputs: the pixel's features (threads < 128) and its direction's
    // positional encoding (threads >= 128)
    if (t < kBgbRows) {
      const int p = pbase + t;
      float x[32];
      if (p < P) load_row<32>(Xb + (size_t)p * 32, x);
#pragma unroll
      for (int k = 0; k < 32; ++k) X[k * kBgbPitch + t] = p < P ? x[k] : 0.0f;
    } else {
      const int r = t - kBgbRows, p = pbase + r, q = p < P ? p : 0;
      float ps[3], dir[3], pe[kPEPad];
      bg_ray(cam, F, radius, q % cam.W, q / cam.W, ps, dir);
      pos_enc(dir, pe);
#pragma unroll
      for (int k = 0; k < kPEPad; ++k) X[(32 + k) * kBgbPitch + r] = pe[k];
    }
    __syncthreads();
    // forward: H1 = ReLU(W0 X + b0), H2 = ReLU(W1 H1 + b1)
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
      const float* A = layer == 0 ? X : H1;
      float* Hout = layer == 0 ? H1 : H2;
      const float* b = smf + (layer == 0 ? L::b0 : L::b1);
      float acc[8][4];
      bgb_prod<64, 4>(A, smf + (layer == 0 ? L::Wt0 : L::Wt1), r0, 4 * og, acc);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float bj = b[4 * og + j];
        float* dst = Hout + (4 * og + j) * kBgbPitch + r0;
        *reinterpret_cast<float4*>(dst) = make_float4(fmaxf(acc[0][j] + bj, 0.0f), fmaxf(acc[1][j] + bj, 0.0f),
                                                      fmaxf(acc[2][j] + bj, 0.0f), fmaxf(acc[3][j] + bj, 0.0f));
        *reinterpret_cast<float4*>(dst + 4) = make_float4(fmaxf(acc[4][j] + bj, 0.0f), fmaxf(acc[5][j] + bj, 0.0f),
                                                          fmaxf(acc[6][j] + bj, 0.0f), fmaxf(acc[7][j] + bj, 0.0f));
      }
      __syncthreads();
    }
    // output layer, colour and dL/dz (Eq. 11; one thread per pixel)
    if (t < kBgbRows) {
      const int p = pbase + t;
      const bool ok = p < P;
      float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
      for (int k = 0; k < 64; ++k) {
        const float h = H2[k * kBgbPitch + t];
        const float4 w = *reinterpret_cast<const float4*>(smf + L::Wt2 + 4 * k);
        o[0] = fmaf(w.x, h, o[0]);
        o[1] = fmaf(w.y, h, o[1]);
        o[2] = fmaf(w.z, h, o[2]);
      }
      float cs[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) cs[k] = sigmoidf_(o[k] + smf[L::b2 + k]);
      const float T = ok ? T_final[p] : 0.0f;
      float dt = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float g = ok ? dC[3 * (int64_t)p + k] : 0.0f;
        dt += g * cs[k];
        if (ok && dC_fg) dC_fg[3 * (int64_t)p + k] = g;
        DZ[k * kBgbPitch + t] = g * T * loss_scale * cs[k] * (1.0f - cs[k]);
      }
      DZ[3 * kBgbPitch + t] = 0.0f;
      if (ok && dT) dT[p] = dt;
    }
    __syncthreads();
    // output layer's gradients; dH2 = W2^T dz masked by H2 > 0
    {
      const int o = t >> 6, i = t & 63;
#pragma unroll 4
      for (int r = 0; r < kBgbRows; r += 4) {
        const float4 d = *reinterpret_cast<const float4*>(DZ + o * kBgbPitch + r);
        const float4 h = *reinterpret_cast<const float4*>(H2 + i * kBgbPitch + r);
        dw2 = fmaf(d.x, h.x, dw2);
        dw2 = fmaf(d.y, h.y, dw2);
        dw2 = fmaf(d.z, h.z, dw2);
        dw2 = fmaf(d.w, h.w, dw2);
      }
      if (t >= 128 && t < 131) db += bgb_rowsum(DZ, t - 128);
    }
    {
      const int r = t & (kBgbRows - 1), half = t >> 7;
      float dh[32];
#pragma unroll
      for (int m = 0; m < 32; ++m) dh[m] = 0.0f;
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        const float d = DZ[o * kBgbPitch + r];
#pragma unroll
        for (int m = 0; m < 32; ++m) dh[m] = fmaf(smf[L::W2 + o * 64 + 32 * half + m], d, dh[m]);
      }
      __syncthreads();  // dz of the output layer has been read
#pragma unroll
      for (int m = 0; m < 32; ++m) {
        const int i = 32 * half + m;
        DZ[i * kBgbPitch + r] = H2[i * kBgbPitch + r] > 0.0f ? dh[m] : 0.0f;
      }
    }
    __syncthreads();
    // second hidden layer's gradients; dH1 = W1^T dZ masked by H1 > 0
    bgb_dw(DZ, H1, 4 * dob, 4 * dib, dw1);
    if (t < 64) db += bgb_rowsum(DZ, t);
    {
      float acc[8][4];
      bgb_prod<64, 4>(DZ, smf + L::W1, r0, 4 * og, acc);
      __syncthreads();  // dZ has been read
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = 4 * og + j;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float4 m = *reinterpret_cast<const float4*>(H1 + i * kBgbPitch + r0 + 4 * h);
          *reinterpret_cast<float4*>(DZ + i * kBgbPitch + r0 + 4 * h) =
              make_float4(m.x > 0.0f ? acc[4 * h][j] : 0.0f, m.y > 0.0f ? acc[4 * h + 1][j] : 0.0f,
                          m.z > 0.0f ? acc[4 * h + 2][j] : 0.0f, m.w > 0.0f ? acc[4 * h + 3][j] : 0.0f);
        }
      }
    }
    __syncthreads();
    // first layer's gradients; dX = W0^T dZ for the features (inputs < 32)
    bgb_dw(DZ, X, 4 * dob, 4 * dib, dw0);
    if (t >= 64 && t < 128) db += bgb_rowsum(DZ, t - 64);
    {
      float acc[8][2];
      bgb_prod<64, 2>(DZ, smf + L::W0, r0, 2 * og, acc);
      __syncthreads();  // X has been read
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h)
          *reinterpret_cast<float4*>(X + (2 * og + j) * kBgbPitch + r0 + 4 * h) =
              make_float4(acc[4 * h][j] * inv_ls, acc[4 * h + 1][j] * inv_ls, acc[4 * h + 2][j] * inv_ls,
                          acc[4 * h + 3][j] * inv_ls);
    }
    __syncthreads();
    if (t < kBgbRows && pbase + t < P) {
      float4* d4 = reinterpret_cast<float4*>(dXb + (size_t)(pbase + t) * 32);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        __stcs(d4 + k, make_float4(X[(4 * k) * kBgbPitch + t], X[(4 * k + 1) * kBgbPitch + t],
                                   X[(4 * k + 2) * kBgbPitch + t], X[(4 * k + 3) * kBgbPitch + t]));
    }
    __syncthreads();  // X is rewritten by the next tile
  }
  float* slab = slabs + (size_t)blockIdx.x * SL.total;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int e = (4 * dob + a) * 64 + 4 * dib + c;
      slab[SL.off_W[1][0] + e] += dw0[a][c];
      slab[SL.off_W[1][1] + e] += dw1[a][c];
    }
  if ((t >> 6) < 3) slab[SL.off_W[1][2] + t] += dw2;
  if (t < 64) slab[SL.off_b[1][1] + t] += db;
  else if (t < 128) slab[SL.off_b[1][0] + t - 64] += db;
  else if (t < 131) slab[SL.off_b[1][2] + t - 128] += db;
}

// ---------------------------------------------------------------- FP32 Gaussian reverse, register-tiled

// The field query's reverse for one decoder (GEO: geometry, else colour) on
// 128 listed rows per tile, as k_bg_dec_bwd_f32: the forward recomputed
// into shared memory, the reverse of Eq. 7 per row, W^T dZ and dZ A^T as
// CTA-wide products, the weight and bias gradients in registers over the
// CTA's tiles and added to its slab (slab index slab0 + CTA) once. Row k of
// the list takes its features from X[k] (k_gather_f32 over the listed rows)
// and leaves their gradients in dX[k] for the table scatter; the colour
// decoder adds the positional encoding's share of dL/dp here.
template <int IN, int OP>
struct QbSmem {  // offsets in floats
  static constexpr int X = 0, H1 = X + 64 * kBgbPitch, H2 = H1 + 64 * kBgbPitch, DZ = H2 + 64 * kBgbPitch,
                       Wt0 = DZ + 64 * kBgbPitch, Wt1 = Wt0 + IN * 64, W0 = Wt1 + 64 * 64, W1 = W0 + 64 * IN,
                       W2 = W1 + 64 * 64, Wt2 = W2 + OP * 64, b0 = Wt2 + 64 * OP, b1 = b0 + 64, b2 = b1 + 64,
                       floats = b2 + OP;
};

template <bool GEO>
__global__ void __launch_bounds__(256, 1) k_query_dec_bwd_f32(FieldsDev F, CamDev cam, QueryBwdIO io,
                                                            SlabLayout SL, float* __restrict__ slabs, int slab0,
                                                            const float* __restrict__ X_in,
                                                            float* __restrict__ dX_out) {
  constexpr int IN = GEO ? 32 : 32 + kPEPad, OUT = GEO ? 8 : 3, OP = GEO ? 8 : 4, DEC = GEO ? 0 : 1;
  using L = QbSmem<IN, OP>;
  extern __shared__ __align__(16) float smf[];
  float *X = smf + L::X, *H1 = smf + L::H1, *H2 = smf + L::H2, *DZ = smf + L::DZ;
  const int t = threadIdx.x;
  const MlpDev& m = GEO ? F.gm : F.cm;
  {
    const float* W0g = static_cast<const float*>(m.W[0]);
    const float* W1g = static_cast<const float*>(m.W[1]);
    const float* W2g = static_cast<const float*>(m.W[2]);
    for (int e = t; e < 64 * IN; e += 256) {  // W0 [64][IN]
      const int o = e / IN, i = e % IN;
      const float v = __ldg(W0g + e);
      smf[L::W0 + e] = v;
      smf[L::Wt0 + i * 64 + o] = v;
    }
    for (int e = t; e < 64 * 64; e += 256) {
      const float v = __ldg(W1g + e);
      smf[L::W1 + e] = v;
      smf[L::Wt1 + (e & 63) * 64 + (e >> 6)] = v;
    }
    for (int e = t; e < OP * 64; e += 256) {  // W2 [OUT][64], rows >= OUT zero
      const int o = e >> 6, i = e & 63;
      const float v = o < OUT ? __ldg(W2g + o * 64 + i) : 0.0f;
      smf[L::W2 + e] = v;
      smf[L::Wt2 + i * OP + o] = v;
    }
    if (t < 64) {
      smf[L::b0 + t] = m.b[0][t];
      smf[L::b1 + t] = m.b[1][t];
    }
    if (t < OP) smf[L::b2 + t] = t < OUT ? m.b[2][t] : 0.0f;
  }
  const int nv = min(*io.n_vis, io.n);
  const int nr = io.list ? min(*io.n_list, nv) : nv;
  const int ntile = (nr + kBgbRows - 1) / kBgbRows;
  const float ls = io.loss_scale, inv_ls = 1.0f / io.loss_scale;
  float pc[3];
  cam_center(cam, pc);
  const int r0 = 8 * (t & 15), og = t >> 4;
  const int dob = t >> 4, dib = t & 15;
  constexpr int BC0 = IN / 16;  // first layer's weight-gradient block: 4 outputs x BC0 inputs
  float dw0[4][BC0], dw1[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int c = 0; c < BC0; ++c) dw0[a][c] = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) dw1[a][c] = 0.0f;
  }
  constexpr int NW2 = OP * 64 / 256;  // output layer's weight gradients per thread
  float dw2[NW2];
#pragma unroll
  for (int q = 0; q < NW2; ++q) dw2[q] = 0.0f;
  float db = 0.0f;  // t < 64: b1[t]; t < 128: b0[t - 64]; t < 128 + OUT: b2[t - 128]
  __syncthreads();
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    // this thread's row (threads t and t + 128 take row t & 127 of the tile)
    const int rr = t & (kBgbRows - 1), krow = tile * kBgbRows + rr;
    bool ok = krow < nr;
    const int i = ok ? (io.list ? io.list[krow] : krow) : 0;
    if (ok && (i < 0 || i >= nv)) {
      set_status(io.status, HYRF_ERR_BOUNDS);
      ok = false;
    }
    const int g = ok ? io.vis_ids[i] : 0;
    if (ok && (g < 0 || g >= io.n)) {
      set_status(io.status, HYRF_ERR_BOUNDS);
      ok = false;
    }
    float dir[3] = {1.0f, 0.0f, 0.0f}, vn = 1.0f;
    if (t < kBgbRows) {  // features
      float x[32];
      load_row<32>(X_in + (size_t)(ok ? krow : 0) * 32, x);
#pragma unroll
      for (int k = 0; k < 32; ++k) X[k * kBgbPitch + rr] = ok ? x[k] : 0.0f;
    } else if (!GEO) {  // positional encoding of the direction from the camera
      float p[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) p[k] = ok ? io.pos[3 * (int64_t)g + k] : F.lo[k] + 1.0f / F.sx[k];
      float v[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
      vn = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) dir[k] = v[k] / vn;
      float pe[kPEPad];
      pos_enc(dir, pe);
#pragma unroll
      for (int k = 0; k < kPEPad; ++k) X[(32 + k) * kBgbPitch + rr] = pe[k];
    }
    __syncthreads();
    // forward: H1 = ReLU(W0 X + b0), H2 = ReLU(W1 H1 + b1)
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
      const float* A = layer == 0 ? X : H1;
      float* Hout = layer == 0 ? H1 : H2;
      const float* b = smf + (layer == 0 ? L::b0 : L::b1);
      float acc[8][4];
      if (layer == 0) bgb_prod<IN, 4>(A, smf + L::Wt0, r0, 4 * og, acc);
      else bgb_prod<64, 4>(A, smf + L::Wt1, r0, 4 * og, acc);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float bj = b[4 * og + j];
        float* dst = Hout + (4 * og + j) * kBgbPitch + r0;
        *reinterpret_cast<float4*>(dst) = make_float4(fmaxf(acc[0][j] + bj, 0.0f), fmaxf(acc[1][j] + bj, 0.0f),
                                                      fmaxf(acc[2][j] + bj, 0.0f), fmaxf(acc[3][j] + bj, 0.0f));
        *reinterpret_cast<float4*>(dst + 4) = make_float4(fmaxf(acc[4][j] + bj, 0.0f), fmaxf(acc[5][j] + bj, 0.0f),
                                                          fmaxf(acc[6][j] + bj, 0.0f), fmaxf(acc[7][j] + bj, 0.0f));
      }
      __syncthreads();
    }
    // output layer and the reverse of Eq. 7 (one thread per row)
    if (t < kBgbRows) {
      float out[OP];
#pragma unroll
      for (int o = 0; o < OP; ++o) out[o] = 0.0f;
#pragma unroll 4
      for (int k = 0; k < 64; ++k) {
        const float h = H2[k * kBgbPitch + t];
#pragma unroll
        for (int q = 0; q < OP / 4; ++q) {
          const float4 w = *reinterpret_cast<const float4*>(smf + L::Wt2 + k * OP + 4 * q);
          out[4 * q] = fmaf(w.x, h, out[4 * q]);
          out[4 * q + 1] = fmaf(w.y, h, out[4 * q + 1]);
          out[4 * q + 2] = fmaf(w.z, h, out[4 * q + 2]);
          out[4 * q + 3] = fmaf(w.w, h, out[4 * q + 3]);
        }
      }
#pragma unroll
      for (int o = 0; o < OP; ++o) out[o] += smf[L::b2 + o];
      float dz[OP];
#pragma unroll
      for (int o = 0; o < OP; ++o) dz[o] = 0.0f;
      if constexpr (GEO) {
        float da = 0.0f, ds[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, ae = 0.0f, se = 0.0f;
        if (ok) {
          da = io.d_alpha[i] * ls;
#pragma unroll
          for (int k = 0; k < 3; ++k) ds[k] = io.d_scale[3 * i + k] * ls;
#pragma unroll
          for (int k = 0; k < 4; ++k) dq[k] = io.d_quat[4 * i + k] * ls;
          ae = io.alpha_e ? io.alpha_e[g] : 0.0f;
          se = io.scale_e ? io.scale_e[g] : 0.0f;
        }
        const float a = sigmoidf_(out[0] + ae);
        dz[0] = da * a * (1.0f - a);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float sv = sigmoidf_(out[1 + k] + se);
          dz[1 + k] = ds[k] * sv * (1.0f - sv);
        }
        const float rn = sqrtf(out[4] * out[4] + out[5] * out[5] + out[6] * out[6] + out[7] * out[7]);
        if (rn > 1e-12f) {
          float qd = 0.0f;
#pragma unroll
          for (int k = 0; k < 4; ++k) qd += out[4 + k] / rn * dq[k];
#pragma unroll
          for (int k = 0; k < 4; ++k) dz[4 + k] = (dq[k] - out[4 + k] / rn * qd) / rn;
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) dz[4 + k] = dq[k] / 1e-12f;
        }
        if (!ok) {
#pragma unroll
          for (int k = 0; k < 8; ++k) dz[k] = 0.0f;
        } else {
          if (io.d_alpha_e) io.d_alpha_e[g] += dz[0] * inv_ls;
          if (io.d_scale_e) io.d_scale_e[g] += (dz[1] + dz[2] + dz[3]) * inv_ls;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float dcol = ok ? io.d_color[3 * i + k] * ls : 0.0f;
          const float ce = ok && io.color_e ? io.color_e[3 * (int64_t)g + k] : 0.0f;
          const float c = sigmoidf_(out[k] + ce);
          dz[k] = ok ? dcol * c * (1.0f - c) : 0.0f;
        }
        if (ok && io.d_color_e) {
#pragma unroll
          for (int k = 0; k < 3; ++k) io.d_color_e[3 * (int64_t)g + k] += dz[k] * inv_ls;
        }
      }
#pragma unroll
      for (int o = 0; o < OP; ++o) DZ[o * kBgbPitch + t] = dz[o];
    }
    __syncthreads();
    // output layer's gradients; dH2 = W2^T dz masked by H2 > 0
#pragma unroll
    for (int q = 0; q < NW2; ++q) {
      const int e = t + 256 * q, o = e >> 6, i2 = e & 63;
#pragma unroll 4
      for (int r = 0; r < kBgbRows; r += 4) {
        const float4 d = *reinterpret_cast<const float4*>(DZ + o * kBgbPitch + r);
        const float4 h = *reinterpret_cast<const float4*>(H2 + i2 * kBgbPitch + r);
        dw2[q] = fmaf(d.x, h.x, dw2[q]);
        dw2[q] = fmaf(d.y, h.y, dw2[q]);
        dw2[q] = fmaf(d.z, h.z, dw2[q]);
        dw2[q] = fmaf(d.w, h.w, dw2[q]);
      }
    }
    if (t >= 128 && t < 128 + OUT) db += bgb_rowsum(DZ, t - 128);
    {
      const int half = t >> 7;
      float dh[32];
#pragma unroll
      for (int mm = 0; mm < 32; ++mm) dh[mm] = 0.0f;
#pragma unroll
      for (int o = 0; o < OUT; ++o) {
        const float d = DZ[o * kBgbPitch + rr];
#pragma unroll
        for (int mm = 0; mm < 32; ++mm) dh[mm] = fmaf(smf[L::W2 + o * 64 + 32 * half + mm], d, dh[mm]);
      }
      __syncthreads();  // dz of the output layer has been read
#pragma unroll
      for (int mm = 0; mm < 32; ++mm) {
        const int i2 = 32 * half + mm;
        DZ[i2 * kBgbPitch + rr] = H2[i2 * kBgbPitch + rr] > 0.0f ? dh[mm] : 0.0f;
      }
    }
    __syncthreads();
    // second hidden layer's gradients; dH1 = W1^T dZ masked by H1 > 0
    bgb_dw(DZ, H1, 4 * dob, 4 * dib, dw1);
    if (t < 64) db += bgb_rowsum(DZ, t);
    {
      float acc[8][4];
      bgb_prod<64, 4>(DZ, smf + L::W1, r0, 4 * og, acc);
      __syncthreads();  // dZ has been read
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i2 = 4 * og + j;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float4 mk = *reinterpret_cast<const float4*>(H1 + i2 * kBgbPitch + r0 + 4 * h);
          *reinterpret_cast<float4*>(DZ + i2 * kBgbPitch + r0 + 4 * h) =
              make_float4(mk.x > 0.0f ? acc[4 * h][j] : 0.0f, mk.y > 0.0f ? acc[4 * h + 1][j] : 0.0f,
                          mk.z > 0.0f ? acc[4 * h + 2][j] : 0.0f, mk.w > 0.0f ? acc[4 * h + 3][j] : 0.0f);
        }
      }
    }
    __syncthreads();
    // first layer's gradients; dX = W0^T dZ (every input: features and, for
    // the colour decoder, the positional encoding)
    bgb_dw<4, BC0>(DZ, X, 4 * dob, BC0 * dib, dw0);
    if (t >= 64 && t < 128) db += bgb_rowsum(DZ, t - 64);
    {
      constexpr int BX = IN / 16;
      float acc[8][BX];
      bgb_prod<64, BX, IN>(DZ, smf + L::W0, r0, BX * og, acc);
      __syncthreads();  // X has been read
#pragma unroll
      for (int j = 0; j < BX; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h)
          *reinterpret_cast<float4*>(X + (BX * og + j) * kBgbPitch + r0 + 4 * h) =
              make_float4(acc[4 * h][j] * inv_ls, acc[4 * h + 1][j] * inv_ls, acc[4 * h + 2][j] * inv_ls,
                          acc[4 * h + 3][j] * inv_ls);
    }
    __syncthreads();
    if (ok) {
      if (t < kBgbRows) {
        float4* d4 = reinterpret_cast<float4*>(dX_out + (size_t)krow * 32);
#pragma unroll
        for (int k = 0; k < 8; ++k)
          __stcs(d4 + k, make_float4(X[(4 * k) * kBgbPitch + rr], X[(4 * k + 1) * kBgbPitch + rr],
                                     X[(4 * k + 2) * kBgbPitch + rr], X[(4 * k + 3) * kBgbPitch + rr]));
      } else if (!GEO) {  // dL/dp through the direction's positional encoding
        float dpe[kPEPad], ddir[3];
#pragma unroll
        for (int k = 0; k < kPEPad; ++k) dpe[k] = X[(32 + k) * kBgbPitch + rr];
        pos_enc_bwd(dir, dpe, ddir);
        const float dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) io.d_pos[3 * (int64_t)g + k] += (ddir[k] - dir[k] * dd) / vn;
      }
    }
    __syncthreads();  // X is rewritten by the next tile
  }
  float* slab = slabs + (size_t)(slab0 + blockIdx.x) * SL.total;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int c = 0; c < BC0; ++c) slab[SL.off_W[DEC][0] + (4 * dob + a) * IN + BC0 * dib + c] += dw0[a][c];
#pragma unroll
    for (int c = 0; c < 4; ++c) slab[SL.off_W[DEC][1] + (4 * dob + a) * 64 + 4 * dib + c] += dw1[a][c];
  }
#pragma unroll
  for (int q = 0; q < NW2; ++q) {
    const int e = t + 256 * q;
    if ((e >> 6) < OUT) slab[SL.off_W[DEC][2] + e] += dw2[q];
  }
  if (t < 64) slab[SL.off_b[DEC][1] + t] += db;
  else if (t < 128) slab[SL.off_b[DEC][0] + t - 64] += db;
  else if (t < 128 + OUT) slab[SL.off_b[DEC][2] + t - 128] += db;
}

template <int NL, int WID, int NH, class WT>
__global__ void __launch_bounds__(kFwdThreads) k_bg_map_texels(FieldsDev F, int Hb, int Wb, float radius,
                                                               float* __restrict__ map) {
  __shared__ float hid[WID * kFwdPitch];
  float* col = hid + threadIdx.x;
  const int n = Hb * Wb;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    float y[3], dir[3], cs[3];
    texel_point(e / Wb, e % Wb, Hb, Wb, radius, y, dir);
    bg_color<NL, WID, NH, WT>(F, y, dir, col, cs);
#pragma unroll
    for (int k = 0; k < 3; ++k) map[3 * e + k] = cs[k];
  }
}

#if HYRF_FIELDS_PART == 0
__global__ void __launch_bounds__(256) k_bg_map_fwd(FieldsDev F, CamDev cam, float radius, int Hb,
                                                    int Wb, const float* __restrict__ map,
                                                    const float* __restrict__ C_fg,
                                                    const float* __restrict__ T_final,
                                                    float* __restrict__ C) {
  const int P = cam.W * cam.H;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float ps[3], dir[3];
    bg_ray(cam, F, radius, p % cam.W, p / cam.W, ps, dir);
    const MapTap m = map_tap(ps, Hb, Wb);
    float cs[3] = {0, 0, 0};
#pragma unroll
    for (int ka = 0; ka < 2; ++ka)
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        const float w = m.wa[ka] * m.wb[kb];
        const float* t = map + 3 * (m.a[ka] * Wb + m.b[kb]);
#pragma unroll
        for (int k = 0; k < 3; ++k) cs[k] += w * t[k];
      }
    const float T = T_final[p];
#pragma unroll
    for (int k = 0; k < 3; ++k) C[3 * (int64_t)p + k] = C_fg[3 * (int64_t)p + k] + T * cs[k];
  }
}

// Map mode, reverse, per pixel: dL/dT_final, dL/dC_fg and the map gradient.
__global__ void __launch_bounds__(256) k_bg_map_bwd_pix(FieldsDev F, CamDev cam, float radius, int Hb,
                                                        int Wb, const float* __restrict__ map,
                                                        const float* __restrict__ T_final,
                                                        const float* __restrict__ dC,
                                                        float* __restrict__ dC_fg,
                                                        float* __restrict__ dT,
                                                        float* __restrict__ dmap) {
  const int P = cam.W * cam.H;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float ps[3], dir[3];
    bg_ray(cam, F, radius, p % cam.W, p / cam.W, ps, dir);
    const MapTap m = map_tap(ps, Hb, Wb);
    float cs[3] = {0, 0, 0};
#pragma unroll
    for (int ka = 0; ka < 2; ++ka)
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        const float w = m.wa[ka] * m.wb[kb];
        const float* t = map + 3 * (m.a[ka] * Wb + m.b[kb]);
#pragma unroll
        for (int k = 0; k < 3; ++k) cs[k] += w * t[k];
      }
    const float T = T_final[p];
    float g[3], dt = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      g[k] = dC[3 * (int64_t)p + k];
      dt += g[k] * cs[k];
      if (dC_fg) dC_fg[3 * (int64_t)p + k] = g[k];
    }
    if (dT) dT[p] = dt;
#pragma unroll
    for (int ka = 0; ka < 2; ++ka)
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        const float w = m.wa[ka] * m.wb[kb] * T;
        float* t = dmap + 3 * (m.a[ka] * Wb + m.b[kb]);
#pragma unroll
        for (int k = 0; k < 3; ++k) atomicAdd(t + k, w * g[k]);
      }
  }
}
#endif

// Reverse of the colour field at background points: MODE 0 = one point per
// pixel (exact mode, also writes dL/dT_final and dL/dC_fg), MODE 1 = one
// point per map texel with the texel gradient given in dmap.
template <int NL, int WID, int NH, int MODE, class WT>
__global__ void __launch_bounds__(kBwdThreads) k_bg_field_bwd(
    FieldsDev F, CamDev cam, float radius, int Hb, int Wb, const float* __restrict__ T_final,
    const float* __restrict__ dC, float* __restrict__ dC_fg, float* __restrict__ dT,
    const float* __restrict__ dmap, float* __restrict__ g_rad_table, float loss_scale,
    SlabLayout SL, float* slabs) {
  extern __shared__ float sm[];
  constexpr int NG = 2 * NL, NC = NG + kPEPad;
  float* act = sm;
  float* dzb = sm + (NC + NH * WID) * kActPitch;
  float* slab = slabs + (size_t)blockIdx.x * SL.total;
  const int t = threadIdx.x;
  const int P = MODE == 0 ? cam.W * cam.H : Hb * Wb;
  const float inv_ls = 1.0f / loss_scale;
  for (int base = blockIdx.x * kBwdThreads; base < P; base += gridDim.x * kBwdThreads) {
    const int e = base + t;
    const bool ok = e < P;
    const int ee = ok ? e : 0;
    float y[3], dir[3], dcs[3];
    if (MODE == 0) {
      float ps[3];
      bg_ray(cam, F, radius, ee % cam.W, ee / cam.W, ps, dir);
      contract_n(ps, y);
    } else {
      texel_point(ee / Wb, ee % Wb, Hb, Wb, radius, y, dir);
    }
    float x0[NC], out[3], dz3[3];
    encode<NL>(F.rad, y, x0);
    pos_enc(dir, x0 + NG);
    decoder_fwd_store<NC, WID, NH, 3, WT>(F.cm, x0, act, out);
    float cs[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) cs[k] = sigmoidf_(out[k]);
    if (MODE == 0) {
      const float T = ok ? T_final[ee] : 0.0f;
      float dt = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float g = ok ? dC[3 * (int64_t)ee + k] : 0.0f;
        dt += g * cs[k];
        dcs[k] = g * T;
        if (ok && dC_fg) dC_fg[3 * (int64_t)ee + k] = g;
      }
      if (ok && dT) dT[ee] = dt;
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) dcs[k] = ok ? dmap[3 * ee + k] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) dz3[k] = dcs[k] * loss_scale * cs[k] * (1.0f - cs[k]);
    float dx[NC];
    decoder_bwd<NC, WID, NH, 3, WT>(F.cm, act, dzb, dz3, slab, SL, 1, dx);
    if (ok) {
#pragma unroll
      for (int k = 0; k < NG; ++k) dx[k] *= inv_ls;
      encode_bwd<NL, true>(F.rad, y, dx, g_rad_table, nullptr);
    }
  }
}

// ---------------------------------------------------------------- host side

static int fwd_blocks(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

int bwd_ctas();
hyrf_status launch_slab_reduce(const float* slabs, int nslabs, const SlabLayout& SL,
                               const SlabTargets& T, float scale, cudaStream_t s);
hyrf_status launch_bg_map_fwd(const FieldsDev& F, const CamDev& cam, float radius, int Hb, int Wb,
                              const float* map, const float* C_fg, const float* T_final, float* C,
                              cudaStream_t s);
hyrf_status launch_bg_map_bwd_pix(const FieldsDev& F, const CamDev& cam, float radius, int Hb, int Wb,
                                  const float* map, const float* T_final, const float* dC,
                                  float* dC_fg, float* dT, float* dmap, cudaStream_t s);
SlabTargets slab_targets(const hyrf_field_grads& g, bool geo);


#if HYRF_FIELDS_PART == 0

bool make_fields(const hyrf_fields& f, FieldsDev& d, bool need_geo) {
  const hyrf_grid* gs[2] = {&f.geo, &f.rad};
  GridDev* gd[2] = {&d.geo, &d.rad};
  for (int k = 0; k < 2; ++k) {
    const hyrf_grid& g = *gs[k];
    if (k == 0 && !need_geo) {
      *gd[0] = GridDev{};
      continue;
    }
    if (!g.table || g.n_levels < 1 || g.n_levels > kMaxLevels || g.n_feat != 2 || g.log2_T < 4 ||
        g.log2_T > 26 || g.base_res < 1 || !(g.growth >= 1.0f) ||
        (g.dtype != HYRF_F32 && g.dtype != HYRF_BF16 && g.dtype != HYRF_U8 && g.dtype != HYRF_F16) ||
        (g.dtype == HYRF_U8 && !g.qparams))
      return false;
    GridDev& o = *gd[k];
    o.table = g.table;
    o.L = g.n_levels;
    o.T = 1u << g.log2_T;
    o.mask = o.T - 1u;
    o.bf16 = g.dtype == HYRF_BF16;
    o.f16 = g.dtype == HYRF_F16;
    o.u8 = g.dtype == HYRF_U8;
    o.q = g.qparams;
    o.log2T = g.log2_T;
    o.dense = 0;
    for (int l = 0; l < g.n_levels; ++l) {
      const double r = std::floor((double)g.base_res * std::pow((double)g.growth, (double)l));
      if (r > 1.0e6) return false;
      o.res[l] = (int)r;
      const uint64_t n1 = (uint64_t)o.res[l] + 1;
      if (n1 * n1 * n1 <= (uint64_t)o.T) o.dense |= 1u << l;
    }
  }
  for (int k = 0; k < 3; ++k) {
    d.lo[k] = f.box_lo[k];
    const float ext = f.box_hi[k] - f.box_lo[k];
    if (!(ext > 0.0f)) return false;
    d.sx[k] = 2.0f / ext;
  }
  const hyrf_mlp* ms[2] = {&f.geo_mlp, &f.col_mlp};
  MlpDev* md[2] = {&d.gm, &d.cm};
  for (int k = 0; k < 2; ++k) {
    const hyrf_mlp& m = *ms[k];
    if (k == 0 && !need_geo) {
      *md[0] = MlpDev{};
      continue;
    }
    if (!((m.n_hidden == 1 && m.width == 32) || (m.n_hidden == 2 && m.width == 64))) return false;
    for (int l = 0; l <= m.n_hidden; ++l)
      if (!m.W[l] || !m.b[l]) return false;
    if (m.dtype != HYRF_F32 && m.dtype != HYRF_BF16 && m.dtype != HYRF_F16) return false;
    MlpDev& o = *md[k];
    for (int l = 0; l < 3; ++l) {
      o.W[l] = l <= m.n_hidden ? m.W[l] : nullptr;
      o.b[l] = l <= m.n_hidden ? m.b[l] : nullptr;
    }
    o.n_in = m.n_in;
    o.width = m.width;
    o.n_hidden = m.n_hidden;
    o.n_out = m.n_out;
    o.bf16 = m.dtype == HYRF_BF16 || m.dtype == HYRF_F16;  // 16-bit: the tensor-core path
    o.f16 = m.dtype == HYRF_F16;
  }
  if (f.pe_freq != kPEFreq || f.pe_pad != kPEPad) return false;
  const int L = f.rad.n_levels;
  if (need_geo) {
    if (f.geo.n_levels != L) return false;
    if (f.geo_mlp.n_in != 2 * L || f.geo_mlp.n_out != 8) return false;
    if (f.geo_mlp.n_hidden != f.col_mlp.n_hidden || f.geo_mlp.width != f.col_mlp.width) return false;
  }
  if (f.col_mlp.n_in != 2 * L + kPEPad || f.col_mlp.n_out != 3) return false;
  d.pe_freq = f.pe_freq;
  d.pe_pad = f.pe_pad;
  return true;
}

int bwd_ctas() { return num_sms() * 3; }

size_t slab_bytes(const FieldsDev& F, bool geo) {
  SlabLayout SL = make_slab_layout(geo ? &F.gm : nullptr, &F.cm);
  return (size_t)bwd_ctas() * SL.total * sizeof(float);
}

SlabTargets slab_targets(const hyrf_field_grads& g, bool geo) {
  SlabTargets T{};
  for (int l = 0; l < 3; ++l) {
    T.W[0][l] = geo ? g.geo_W[l] : nullptr;
    T.b[0][l] = geo ? g.geo_b[l] : nullptr;
    T.W[1][l] = g.col_W[l];
    T.b[1][l] = g.col_b[l];
  }
  return T;
}

hyrf_status launch_slab_reduce(const float* slabs, int nslabs, const SlabLayout& SL,
                               const SlabTargets& T, float scale, cudaStream_t s) {
  if (SL.total <= 0 || nslabs <= 0) return HYRF_OK;
  // columns of 256 elements x 8 parts of the slab range
  const dim3 grid((SL.total + 255) / 256, 8);
  HYRF_LAUNCH("k_slab_reduce", s, k_slab_reduce<<<grid, 256, 0, s>>>(slabs, nslabs, SL, T, scale));
  return HYRF_OK;
}

hyrf_status launch_bg_map_fwd(const FieldsDev& F, const CamDev& cam, float radius, int Hb, int Wb,
                              const float* map, const float* C_fg, const float* T_final, float* C,
                              cudaStream_t s) {
  HYRF_LAUNCH("k_bg_map_fwd", s,
              k_bg_map_fwd<<<fwd_blocks((int64_t)cam.W * cam.H, 256), 256, 0, s>>>(F, cam, radius, Hb, Wb, map,
                                                                      C_fg, T_final, C));
  return HYRF_OK;
}

hyrf_status launch_bg_map_bwd_pix(const FieldsDev& F, const CamDev& cam, float radius, int Hb, int Wb,
                                  const float* map, const float* T_final, const float* dC,
                                  float* dC_fg, float* dT, float* dmap, cudaStream_t s) {
  HYRF_LAUNCH("k_bg_map_bwd_pix", s,
              k_bg_map_bwd_pix<<<fwd_blocks((int64_t)cam.W * cam.H, 256), 256, 0, s>>>(F, cam, radius, Hb, Wb, map,
                                                                          T_final, dC, dC_fg, dT, dmap));
  return HYRF_OK;
}

size_t tc_bwd_workspace(const FieldsDev& F, bool geo, int64_t rows, bool have_features);
size_t tc_bg_fwd_workspace(int64_t P, bool have_features, bool skip);

static int part_of(const hyrf_fields& f, const FieldsDev& F);

// FP32 shapes that take the split path (gather kernel + decoder kernel):
// 16 levels, 2 x 64 decoders (part 2); f32 feature bytes of `rows` rows.
static bool f32_split(const hyrf_fields& f, const FieldsDev& F) { return part_of(f, F) == 2; }
static size_t f32_feature_bytes(int64_t rows, int fields) { return align_up((size_t)fields * rows * 32 * 4); }

size_t query_fwd_workspace_f32(const hyrf_fields& f, const FieldsDev& F, int n) {
  return f32_split(f, F) ? f32_feature_bytes(n, 2) : 0;
}

size_t bg_workspace(const hyrf_composite_background_args& a, const FieldsDev& F, bool backward) {
  if (a.bg.mode == 0 && F.cm.bf16) {  // tensor-core path: gathered features (+ gradients)
    const int64_t P = (int64_t)a.cam.width * a.cam.height;
    const bool have = a.features != nullptr, skip = a.bg.tau_T > 0.0f;
    return backward ? tc_bwd_workspace(F, false, P, have) : tc_bg_fwd_workspace(P, have && !skip, skip);
  }
  if (a.bg.mode == 0 && f32_split(a.fields, F)) {  // split path: features (+ gradients, slabs)
    const int64_t P = (int64_t)a.cam.width * a.cam.height;
    if (!backward) return f32_feature_bytes(P, 1);
    Carver c(nullptr);
    c.take<char>(slab_bytes(F, false));
    c.take<char>(f32_feature_bytes(P, 1));
    c.take<char>(f32_feature_bytes(P, 1));
    return c.size();
  }
  Carver c(nullptr);
  if (a.bg.mode == 1) {
    c.take<float>((size_t)a.bg.map_h * a.bg.map_w * 3);  // map
    if (backward) c.take<float>((size_t)a.bg.map_h * a.bg.map_w * 3);  // dmap
  }
  if (backward) c.take<char>(slab_bytes(F, false));
  return c.size();
}

#define HYRF_DECLARE_PART(P)                                                                      \
  hyrf_status query_fwd_p##P(const FieldsDev&, const CamDev&, const QueryFwdIO&, float*, cudaStream_t); \
  hyrf_status query_bwd_p##P(const FieldsDev&, const CamDev&, const QueryBwdIO&,                  \
                             const hyrf_field_grads&, float*, float*, cudaStream_t);              \
  hyrf_status bg_fwd_p##P(const hyrf_composite_background_args&, const FieldsDev&, void*,          \
                          cudaStream_t);                                                          \
  hyrf_status bg_bwd_p##P(const hyrf_composite_background_backward_args&, const FieldsDev&, void*, \
                          cudaStream_t);
HYRF_DECLARE_PART(1)
HYRF_DECLARE_PART(2)
HYRF_DECLARE_PART(3)

// Shape dispatch: (levels, width, hidden layers, weights) in
// {(8, 32, 1, f32) = part 1, (16, 64, 2, f32) = part 2, (16, 64, 2, bf16) = part 3}.
static int part_of(const hyrf_fields& f, const FieldsDev& F) {
  const int L = f.rad.n_levels;
  if (L == 8 && f.col_mlp.width == 32 && f.col_mlp.n_hidden == 1 && !F.cm.bf16) return 1;
  if (L == 16 && f.col_mlp.width == 64 && f.col_mlp.n_hidden == 2) return F.cm.bf16 ? 3 : 2;
  return 0;
}

size_t precull_workspace(int n);

// ws: the field query's workspace (the pre-cull's part first, then, for the
// split shapes, the f32 features of both fields).
hyrf_status launch_query_fwd(const hyrf_query_fields_args& a, const FieldsDev& F, void* ws, cudaStream_t s) {
  QueryFwdIO io{a.n,      a.pos,   a.alpha_e, a.scale_e, a.color_e, a.vis_ids,
                a.n_vis,  a.alpha, a.scale,   a.quat,    a.color,   a.status};
  const CamDev cam = to_dev(a.cam);
  if (a.n == 0) return HYRF_OK;
  float* X = nullptr;
  if (f32_split(a.fields, F)) {
    Carver c(ws);
    c.take<char>(precull_workspace(a.n));
    X = reinterpret_cast<float*>(c.take<char>(f32_feature_bytes(a.n, 2)));
    const RowSource RS{0, a.n, a.vis_ids, a.n_vis, a.pos, 0.0f, a.status, nullptr, nullptr};
    hyrf_status st = launch_gather_f32(F, cam, RS, a.n, X, X + (size_t)a.n * 32, s);
    if (st != HYRF_OK) return st;
  }
  switch (part_of(a.fields, F)) {
    case 1: return query_fwd_p1(F, cam, io, X, s);
    case 2: return query_fwd_p2(F, cam, io, X, s);
    case 3: return query_fwd_p3(F, cam, io, X, s);
    default: return HYRF_ERR_UNSUPPORTED;
  }
}

size_t active_rows_workspace(int n);
hyrf_status launch_active_rows(int n, const int32_t* n_vis, const float* d_alpha, const float* d_scale,
                               const float* d_quat, const float* d_color, Carver& c, int32_t** list,
                               int32_t** n_list, cudaStream_t s);

// FP32 reverse workspace: CTA slabs, the list of rows with a gradient and,
// for the split shapes, f32 features and feature gradients of both fields.
size_t query_bwd_workspace(const hyrf_fields& f, const FieldsDev& F, int n) {
  Carver c(nullptr);
  c.take<char>(slab_bytes(F, true));
  c.take<char>(active_rows_workspace(n));
  if (f32_split(f, F)) c.take<char>(f32_feature_bytes(n, 4));
  return c.size();
}

hyrf_status launch_query_bwd(const hyrf_query_fields_backward_args& a, const FieldsDev& F,
                             void* ws, cudaStream_t s) {
  QueryBwdIO io{a.n,        a.pos,       a.alpha_e,   a.scale_e,   a.color_e,
                a.vis_ids,  a.n_vis,     a.d_alpha,   a.d_scale,   a.d_quat,
                a.d_color,  a.d_pos,     a.d_alpha_e, a.d_scale_e, a.d_color_e,
                a.grads.geo_table, a.grads.rad_table, a.loss_scale, a.status, nullptr, nullptr};
  const CamDev cam = to_dev(a.cam);
  if (a.n == 0) return HYRF_OK;
  Carver c(ws);
  float* slabs = reinterpret_cast<float*>(c.take<char>(slab_bytes(F, true)));
  Carver ca(c.take<char>(active_rows_workspace(a.n)));
  int32_t *list = nullptr, *n_list = nullptr;
  hyrf_status st = launch_active_rows(a.n, a.n_vis, a.d_alpha, a.d_scale, a.d_quat, a.d_color, ca, &list,
                                      &n_list, s);
  if (st != HYRF_OK) return st;
  io.list = list;
  io.n_list = n_list;
  float* X = f32_split(a.fields, F) ? reinterpret_cast<float*>(c.take<char>(f32_feature_bytes(a.n, 4))) : nullptr;
  switch (part_of(a.fields, F)) {
    case 1: return query_bwd_p1(F, cam, io, a.grads, slabs, X, s);
    case 2: return query_bwd_p2(F, cam, io, a.grads, slabs, X, s);
    case 3: return query_bwd_p3(F, cam, io, a.grads, slabs, X, s);
    default: return HYRF_ERR_UNSUPPORTED;
  }
}

hyrf_status launch_bg_fwd(const hyrf_composite_background_args& a, const FieldsDev& F, void* ws,
                          cudaStream_t s) {
  switch (part_of(a.fields, F)) {
    case 1: return bg_fwd_p1(a, F, ws, s);
    case 2: return bg_fwd_p2(a, F, ws, s);
    case 3: return bg_fwd_p3(a, F, ws, s);
    default: return HYRF_ERR_UNSUPPORTED;
  }
}

hyrf_status launch_bg_bwd(const hyrf_composite_background_backward_args& b, const FieldsDev& F,
                          void* ws, cudaStream_t s) {
  switch (part_of(b.fwd.fields, F)) {
    case 1: return bg_bwd_p1(b, F, ws, s);
    case 2: return bg_bwd_p2(b, F, ws, s);
    case 3: return bg_bwd_p3(b, F, ws, s);
    default: return HYRF_ERR_UNSUPPORTED;
  }
}

#else  // parts 1-3: one shape each

#if HYRF_FIELDS_PART == 1
#define HYRF_SHAPE 8, 32, 1, float
#elif HYRF_FIELDS_PART == 2
#define HYRF_SHAPE 16, 64, 2, float
#else
#define HYRF_SHAPE 16, 64, 2, __nv_bfloat16
#endif

template <int NL, int WID, int NH, class WT>
static hyrf_status query_fwd_impl(const FieldsDev& F, const CamDev& cam, const QueryFwdIO& io, float* X,
                                  cudaStream_t s) {
  if constexpr (std::is_same<WT, __nv_bfloat16>::value) {
    return HYRF_ERR_UNSUPPORTED;  // bf16 decoders run on the tensor cores (fields_tc.cu)
  } else {
    if (X) {  // split path: features gathered by k_gather_f32
      if constexpr (NL == 16 && WID == 64 && NH == 2) {  // register-tiled decoders
        const int tiles = (io.n + kDecRows - 1) / kDecRows, grid = min(tiles, 2 * num_sms());
        const int sg = DecSmemF32<32, 8>::floats * (int)sizeof(float);
        const int sc = DecSmemF32<32 + kPEPad, 4>::floats * (int)sizeof(float);
        set_smem_limit<k_query_dec_f32<true>>(sg);
        set_smem_limit<k_query_dec_f32<false>>(sc);
        HYRF_LAUNCH("k_query_dec_f32<geo>", s, k_query_dec_f32<true><<<grid, kDecRows, sg, s>>>(F, cam, io, X));
        HYRF_LAUNCH("k_query_dec_f32<col>", s,
                    k_query_dec_f32<false><<<grid, kDecRows, sc, s>>>(F, cam, io, X + (size_t)io.n * 2 * NL));
        return HYRF_OK;
      }
      return HYRF_ERR_UNSUPPORTED;  // features are gathered only for the split shape
    }
    HYRF_LAUNCH("k_query_fwd", s,
                k_query_fwd<NL, WID, NH, WT><<<fwd_blocks(io.n, kFwdThreads), kFwdThreads, 0, s>>>(F, cam, io));
    return HYRF_OK;
  }
}

template <int NL, int WID, int NH, class WT>
static hyrf_status query_bwd_impl(const FieldsDev& F, const CamDev& cam, const QueryBwdIO& io,
                                  const hyrf_field_grads& grads, float* slabs, float* X, cudaStream_t s) {
  const SlabLayout SL = make_slab_layout(&F.gm, &F.cm);
  const int ctas = bwd_ctas();
  cudaMemsetAsync(slabs, 0, (size_t)ctas * SL.total * sizeof(float), s);
  const size_t smem = query_bwd_smem_floats<NL, WID, NH>() * sizeof(float);
  if constexpr (NL == 16 && WID == 64 && NH == 2 && std::is_same<WT, float>::value) {
    if (X) {  // split path: the listed rows' features gathered into X, gradients to dX, then scattered
      const size_t rows = (size_t)io.n * 2 * NL;
      float *Xg = X, *Xr = X + rows, *dXg = X + 2 * rows, *dXr = X + 3 * rows;
      const RowSource RS{0, io.n, io.vis_ids, io.n_vis, io.pos, 0.0f, io.status, io.list, io.n_list};
      hyrf_status st = launch_gather_f32(F, cam, RS, io.n, Xg, Xr, s);
      if (st != HYRF_OK) return st;
      const int tiles = (io.n + kBgbRows - 1) / kBgbRows;
      const int grid = max(1, min(tiles, min(num_sms(), ctas / 2)));
      const int sg = QbSmem<32, 8>::floats * (int)sizeof(float);
      const int sc = QbSmem<32 + kPEPad, 4>::floats * (int)sizeof(float);
      set_smem_limit<k_query_dec_bwd_f32<true>>(sg);
      set_smem_limit<k_query_dec_bwd_f32<false>>(sc);
      HYRF_LAUNCH("k_query_dec_bwd_f32<geo>", s,
                  k_query_dec_bwd_f32<true><<<grid, 256, sg, s>>>(F, cam, io, SL, slabs, 0, Xg, dXg));
      HYRF_LAUNCH("k_query_dec_bwd_f32<col>", s,
                  k_query_dec_bwd_f32<false><<<grid, 256, sc, s>>>(F, cam, io, SL, slabs, grid, Xr, dXr));
      st = launch_slab_reduce(slabs, 2 * grid, SL, slab_targets(grads, true), 1.0f / io.loss_scale, s);
      if (st != HYRF_OK) return st;
      return launch_scatter(F, cam, RS, io.n, dXg, dXr, io.g_geo_table, io.g_rad_table, io.d_pos, s);
    }
  }
  set_smem_limit<k_query_bwd<NL, WID, NH, WT>>((int)smem);
  HYRF_LAUNCH("k_query_bwd", s,
              k_query_bwd<NL, WID, NH, WT><<<ctas, kBwdThreads, smem, s>>>(F, cam, io, SL, slabs));
  return launch_slab_reduce(slabs, ctas, SL, slab_targets(grads, true), 1.0f / io.loss_scale, s);
}

template <int NL, int WID, int NH, class WT>
static hyrf_status bg_fwd_impl(const hyrf_composite_background_args& a, const FieldsDev& F, void* ws,
                               cudaStream_t s) {
  const CamDev cam = to_dev(a.cam);
  const int P = cam.W * cam.H;
  if (a.bg.mode == 0) {
    if constexpr (std::is_same<WT, __nv_bfloat16>::value) {
      return HYRF_ERR_UNSUPPORTED;  // bf16 decoders run on the tensor cores (fields_tc.cu)
    } else if constexpr (NL == 16 && WID == 64 && NH == 2) {  // split path
      float* Xb = static_cast<float*>(ws);
      const RowSource RS{1, 0, nullptr, nullptr, nullptr, a.bg.radius, a.status, nullptr, nullptr};
      hyrf_status st = launch_gather_f32(F, cam, RS, P, nullptr, Xb, s);
      if (st != HYRF_OK) return st;
      const int tiles = (P + kDecRows - 1) / kDecRows, grid = min(tiles, 2 * num_sms());
      const int sb = DecSmemF32<2 * NL + kPEPad, 4>::floats * (int)sizeof(float);
      set_smem_limit<k_bg_dec_f32<2 * NL>>(sb);
      HYRF_LAUNCH("k_bg_dec_f32", s,
                  k_bg_dec_f32<2 * NL><<<grid, kDecRows, sb, s>>>(F, cam, a.bg.radius, Xb, a.C_fg, a.T_final, a.C));
      return HYRF_OK;
    } else {
      HYRF_LAUNCH("k_bg_exact_fwd", s,
                  k_bg_exact_fwd<NL, WID, NH, WT><<<fwd_blocks(P, kFwdThreads), kFwdThreads, 0, s>>>(
          F, cam, a.bg.radius, a.C_fg, a.T_final, a.C));
      return HYRF_OK;
    }
  }
  Carver c(ws);
  float* map = c.take<float>((size_t)a.bg.map_h * a.bg.map_w * 3);
  const int nt = a.bg.map_h * a.bg.map_w;
  HYRF_LAUNCH("k_bg_map_texels", s,
              k_bg_map_texels<NL, WID, NH, WT><<<fwd_blocks(nt, 128), 128, 0, s>>>(F, a.bg.map_h, a.bg.map_w,
                                                                        a.bg.radius, map));
  return launch_bg_map_fwd(F, cam, a.bg.radius, a.bg.map_h, a.bg.map_w, map, a.C_fg, a.T_final, a.C, s);
}

template <int NL, int WID, int NH, class WT>
static hyrf_status bg_bwd_impl(const hyrf_composite_background_backward_args& b, const FieldsDev& F,
                               void* ws, cudaStream_t s) {
  const hyrf_composite_background_args& a = b.fwd;
  const CamDev cam = to_dev(a.cam);
  const SlabLayout SL = make_slab_layout(nullptr, &F.cm);
  const int ctas = bwd_ctas();
  if constexpr (NL == 16 && WID == 64 && NH == 2 && std::is_same<WT, float>::value) {
    if (a.bg.mode == 0) {  // split path: gather, decoder reverse, scatter
      const int P = cam.W * cam.H;
      Carver c(ws);
      float* slabs = reinterpret_cast<float*>(c.take<char>(slab_bytes(F, false)));
      float* Xb = reinterpret_cast<float*>(c.take<char>((size_t)P * 32 * 4));
      float* dXb = reinterpret_cast<float*>(c.take<char>((size_t)P * 32 * 4));
      cudaMemsetAsync(slabs, 0, (size_t)ctas * SL.total * sizeof(float), s);
      const RowSource RS{1, 0, nullptr, nullptr, nullptr, a.bg.radius, a.status, nullptr, nullptr};
      hyrf_status st = launch_gather_f32(F, cam, RS, P, nullptr, Xb, s);
      if (st != HYRF_OK) return st;
      const int tiles = (P + kBgbRows - 1) / kBgbRows;
      const int grid = min(min(ctas, num_sms()), tiles);
      const int smem = BgbSmem::floats * (int)sizeof(float);
      set_smem_limit<k_bg_dec_bwd_f32<2 * NL>>(smem);
      HYRF_LAUNCH("k_bg_dec_bwd_f32", s,
                  k_bg_dec_bwd_f32<2 * NL><<<grid, 256, smem, s>>>(F, cam, a.bg.radius, a.T_final, b.d_C, b.d_C_fg,
                                                                b.d_T_final, b.loss_scale, SL, slabs, Xb, dXb));
      st = launch_slab_reduce(slabs, grid, SL, slab_targets(b.grads, false), 1.0f / b.loss_scale, s);
      if (st != HYRF_OK) return st;
      return launch_scatter(F, cam, RS, P, nullptr, dXb, nullptr, b.grads.rad_table, nullptr, s);
    }
  }
  Carver c(ws);
  float* map = nullptr;
  float* dmap = nullptr;
  const int Hb = a.bg.map_h, Wb = a.bg.map_w;
  if (a.bg.mode == 1) {
    map = c.take<float>((size_t)Hb * Wb * 3);
    dmap = c.take<float>((size_t)Hb * Wb * 3);
  }
  float* slabs = c.take<float>((size_t)ctas * SL.total);
  cudaMemsetAsync(slabs, 0, (size_t)ctas * SL.total * sizeof(float), s);
  const size_t smem = query_bwd_smem_floats<NL, WID, NH>() * sizeof(float);
  if (a.bg.mode == 0) {
    set_smem_limit<k_bg_field_bwd<NL, WID, NH, 0, WT>>((int)smem);
    HYRF_LAUNCH("k_bg_field_bwd", s,
                k_bg_field_bwd<NL, WID, NH, 0, WT><<<ctas, kBwdThreads, smem, s>>>(
        F, cam, a.bg.radius, 0, 0, a.T_final, b.d_C, b.d_C_fg, b.d_T_final, nullptr,
        b.grads.rad_table, b.loss_scale, SL, slabs));
  } else {
    const int nt = Hb * Wb;
    HYRF_LAUNCH("k_bg_map_texels", s,
                k_bg_map_texels<NL, WID, NH, WT><<<fwd_blocks(nt, 128), 128, 0, s>>>(F, Hb, Wb, a.bg.radius, map));
    cudaMemsetAsync(dmap, 0, (size_t)nt * 3 * sizeof(float), s);
    hyrf_status st = launch_bg_map_bwd_pix(F, cam, a.bg.radius, Hb, Wb, map, a.T_final, b.d_C,
                                           b.d_C_fg, b.d_T_final, dmap, s);
    if (st != HYRF_OK) return st;
    set_smem_limit<k_bg_field_bwd<NL, WID, NH, 1, WT>>((int)smem);
    HYRF_LAUNCH("k_bg_field_bwd", s,
                k_bg_field_bwd<NL, WID, NH, 1, WT><<<ctas, kBwdThreads, smem, s>>>(
        F, cam, a.bg.radius, Hb, Wb, nullptr, nullptr, nullptr, nullptr, dmap, b.grads.rad_table,
        b.loss_scale, SL, slabs));
  }
  return launch_slab_reduce(slabs, ctas, SL, slab_targets(b.grads, false), 1.0f / b.loss_scale, s);
}

#define HYRF_PASTE2(a, b) a##b
#define HYRF_PASTE(a, b) HYRF_PASTE2(a, b)

hyrf_status HYRF_PASTE(query_fwd_p, HYRF_FIELDS_PART)(const FieldsDev& F, const CamDev& cam,
                                                      const QueryFwdIO& io, float* X, cudaStream_t s) {
  return query_fwd_impl<HYRF_SHAPE>(F, cam, io, X, s);
}
hyrf_status HYRF_PASTE(query_bwd_p, HYRF_FIELDS_PART)(const FieldsDev& F, const CamDev& cam,
                                                      const QueryBwdIO& io,
                                                      const hyrf_field_grads& g, float* slabs, float* X,
                                                      cudaStream_t s) {
  return query_bwd_impl<HYRF_SHAPE>(F, cam, io, g, slabs, X, s);
}
hyrf_status HYRF_PASTE(bg_fwd_p, HYRF_FIELDS_PART)(const hyrf_composite_background_args& a,
                                                   const FieldsDev& F, void* ws, cudaStream_t s) {
  return bg_fwd_impl<HYRF_SHAPE>(a, F, ws, s);
}
hyrf_status HYRF_PASTE(bg_bwd_p, HYRF_FIELDS_PART)(const hyrf_composite_background_backward_args& b,
                                                   const FieldsDev& F, void* ws, cudaStream_t s) {
  return bg_bwd_impl<HYRF_SHAPE>(b, F, ws, s);
}

#endif  // HYRF_FIELDS_PART

}  // namespace hyrf
