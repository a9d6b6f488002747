// Device building blocks of the neural fields (Sec. 3.2): App. A.1
// normalisation, Eq. 2 contraction, Eq. 3 multi-resolution hash encoding
// (gather and gradient scatter), Eq. 5 positional encoding and the decoder
// layers. Shared by the field-query and background kernels.
#pragma once
#include "common.cuh"

namespace hyrf {

constexpr int kPEFreq = 4;  // PE frequencies supported by the kernels (3 + 6*4 = 27 <= 32)

// Eq. 2 contraction of an already normalised point x (|x| <= 1 kept affine),
// with the offset read as +0.5 so that the range is (0, 1).
__device__ __forceinline__ void contract_n(const float x[3], float y[3]) {
  const float n = sqrtf(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  float g = 1.0f;
  if (n > 1.0f) {
    const float inv = 1.0f / n;
    g = 2.0f * inv - inv * inv;
  }
  y[0] = 0.25f * g * x[0] + 0.5f;
  y[1] = 0.25f * g * x[1] + 0.5f;
  y[2] = 0.25f * g * x[2] + 0.5f;
}

// App. A.1 normalisation then contraction; J (row-major dy/dp) if non-null.
__device__ __forceinline__ void contract_p(const FieldsDev& F, const float p[3], float y[3], float* J) {
  float x[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) x[k] = (p[k] - F.lo[k]) * F.sx[k] - 1.0f;
  const float n = sqrtf(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  if (n <= 1.0f) {
#pragma unroll
    for (int k = 0; k < 3; ++k) y[k] = 0.25f * x[k] + 0.5f;
    if (J) {
#pragma unroll
      for (int i = 0; i < 9; ++i) J[i] = (i % 4 == 0) ? 0.25f * F.sx[i / 3] : 0.0f;
    }
  } else {
    const float inv = 1.0f / n;
    const float g = 2.0f * inv - inv * inv;
    const float gp = (-2.0f + 2.0f * inv) * inv * inv;  // dg/dn
#pragma unroll
    for (int k = 0; k < 3; ++k) y[k] = 0.25f * g * x[k] + 0.5f;
    if (J) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          J[3 * i + j] = 0.25f * ((i == j ? g : 0.0f) + gp * x[i] * x[j] * inv) * F.sx[j];
    }
  }
}

// Corner indices and fractional position of point y in level l.
__device__ __forceinline__ void level_cell(const GridDev& G, int l, const float y[3], uint32_t idx[8],
                                           float f[3], uint64_t* cell = nullptr) {
  const int N = G.res[l];
  uint32_t i0[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float u = y[d] * (float)N;
    float fl = floorf(u);
    fl = fminf(fmaxf(fl, 0.0f), (float)(N - 1));
    i0[d] = (uint32_t)fl;
    f[d] = u - fl;
  }
  if (cell) *cell = (uint64_t)i0[0] | ((uint64_t)i0[1] << 21) | ((uint64_t)i0[2] << 42);  // N < 2^21
  const uint32_t n1 = (uint32_t)N + 1u;
  if ((G.dense >> l) & 1u) {  // uniform over a level: one of the two index forms only
    const uint32_t b = i0[0] + i0[1] * n1 + i0[2] * n1 * n1;
#pragma unroll
    for (int c = 0; c < 8; ++c) idx[c] = b + (c & 1) + ((c >> 1) & 1) * n1 + ((c >> 2) & 1) * n1 * n1;
  } else {
    const uint32_t hy0 = i0[1] * 2654435761u, hy1 = (i0[1] + 1u) * 2654435761u;
    const uint32_t hz0 = i0[2] * 805459861u, hz1 = (i0[2] + 1u) * 805459861u;
#pragma unroll
    for (int c = 0; c < 8; ++c)
      idx[c] = ((i0[0] + (c & 1)) ^ ((c & 2) ? hy1 : hy0) ^ ((c & 4) ? hz1 : hz0)) & G.mask;
  }
}

__device__ __forceinline__ float corner_w(const float f[3], int c) {
  return ((c & 1) ? f[0] : 1.0f - f[0]) * ((c & 2) ? f[1] : 1.0f - f[1]) *
         ((c & 4) ? f[2] : 1.0f - f[2]);
}

// Entry e of a table whose type is known at compile time: 0 float32,
// 1 bf16, 2 uint8 codes (value = lo + step * code, per level), 3 f16.
template <int DT>
__device__ __forceinline__ float2 load_entry_t(const GridDev& G, size_t e) {
  if constexpr (DT == 3) {
    return __half22float2(__ldg(reinterpret_cast<const __half2*>(G.table) + e));
  } else if constexpr (DT == 2) {
    const uchar2 c = __ldg(reinterpret_cast<const uchar2*>(G.table) + e);
    const float2 q = __ldg(reinterpret_cast<const float2*>(G.q) + (e >> G.log2T));
    return make_float2(fmaf(q.y, (float)c.x, q.x), fmaf(q.y, (float)c.y, q.x));
  } else if constexpr (DT == 1) {
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(G.table) + e));
  } else {
    return __ldg(reinterpret_cast<const float2*>(G.table) + e);
  }
}

// float32 or bf16 table (runtime flag), for the fused FP32 kernels.
__device__ __forceinline__ float2 load_entry(const GridDev& G, size_t e) {
  if (G.bf16) {
    const __nv_bfloat162 v = __ldg(reinterpret_cast<const __nv_bfloat162*>(G.table) + e);
    return __bfloat1622float2(v);
  }
  return __ldg(reinterpret_cast<const float2*>(G.table) + e);
}

// Eq. 3: level-major features f[2l + k] = sum_c w_c table[l][idx_c][k].
template <int L>
__device__ __forceinline__ void encode(const GridDev& G, const float y[3], float* feat) {
#pragma unroll
  for (int l = 0; l < L; ++l) {
    uint32_t idx[8];
    float f[3];
    level_cell(G, l, y, idx, f);
    float2 e[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) e[c] = load_entry(G, (size_t)l * G.T + idx[c]);
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float w = corner_w(f, c);
      a0 = fmaf(w, e[c].x, a0);
      a1 = fmaf(w, e[c].y, a1);
    }
    feat[2 * l] = a0;
    feat[2 * l + 1] = a1;
  }
}

// Reverse of encode: scatter w_c * df into the float32 table gradient and,
// if dy is given, accumulate dL/dy through the trilinear weights.
// COHERENT: the lanes of a warp hold neighbouring points (e.g. background
// pixels of one image row), so at coarse levels they often share a corner;
// when the whole warp targets one entry its contributions are summed with
// shuffles and added by one atomic instead of 32 serialised ones.
template <int L, bool COHERENT = false>
__device__ __forceinline__ void encode_bwd(const GridDev& G, const float y[3], const float* df,
                                           float* __restrict__ gtab, float* dy) {
  const unsigned am = COHERENT ? __activemask() : 0u;
#pragma unroll 2
  for (int l = 0; l < L; ++l) {
    uint32_t idx[8];
    float f[3];
    level_cell(G, l, y, idx, f);
    const float d0 = df[2 * l], d1 = df[2 * l + 1];
    float g[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const size_t e = (size_t)l * G.T + idx[c];
      const float w = corner_w(f, c);
      if (gtab) {
        float g0 = w * d0, g1 = w * d1;
        bool done = false;
        if (COHERENT && am == 0xffffffffu) {
          const uint32_t e0 = __shfl_sync(am, idx[c], 0);
          if (__all_sync(am, idx[c] == e0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              g0 += __shfl_xor_sync(am, g0, o);
              g1 += __shfl_xor_sync(am, g1, o);
            }
            if ((threadIdx.x & 31) == 0 && (g0 != 0.0f || g1 != 0.0f))
              atomicAdd(reinterpret_cast<float2*>(gtab) + e, make_float2(g0, g1));
            done = true;
          }
        }
        if (!done && (g0 != 0.0f || g1 != 0.0f))
          atomicAdd(reinterpret_cast<float2*>(gtab) + e, make_float2(g0, g1));
      }
      if (dy) {
        const float2 v = load_entry(G, e);
        const float dot = v.x * d0 + v.y * d1;
        const float wx = (c & 1) ? f[0] : 1.0f - f[0];
        const float wy = (c & 2) ? f[1] : 1.0f - f[1];
        const float wz = (c & 4) ? f[2] : 1.0f - f[2];
        g[0] += dot * ((c & 1) ? 1.0f : -1.0f) * wy * wz;
        g[1] += dot * ((c & 2) ? 1.0f : -1.0f) * wx * wz;
        g[2] += dot * ((c & 4) ? 1.0f : -1.0f) * wx * wy;
      }
    }
    if (dy) {
      const float N = (float)G.res[l];
      dy[0] += g[0] * N;
      dy[1] += g[1] * N;
      dy[2] += g[2] * N;
    }
  }
}

// Eq. 5: [d, sin(2^k pi d), cos(2^k pi d)] for k < 4, zero-padded to 32.
__device__ __forceinline__ void pos_enc(const float d[3], float* out) {
#pragma unroll
  for (int j = 0; j < 3; ++j) out[j] = d[j];
#pragma unroll
  for (int k = 0; k < kPEFreq; ++k) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float s, c;
      sincospif((float)(1 << k) * d[j], &s, &c);
      out[3 + 6 * k + j] = s;
      out[3 + 6 * k + 3 + j] = c;
    }
  }
#pragma unroll
  for (int j = 3 + 6 * kPEFreq; j < kPEPad; ++j) out[j] = 0.0f;
}

__device__ __forceinline__ void pos_enc_bwd(const float d[3], const float* dout, float dd[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) dd[j] = dout[j];
#pragma unroll
  for (int k = 0; k < kPEFreq; ++k) {
    const float w = (float)(1 << k) * 3.14159265358979f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float s, c;
      sincospif((float)(1 << k) * d[j], &s, &c);
      dd[j] += w * (dout[3 + 6 * k + j] * c - dout[3 + 6 * k + 3 + j] * s);
    }
  }
}

// ---------------------------------------------------------------- decoder layers (CUDA cores)

// Four consecutive weights as float (float32 or bfloat16 storage). Every
// lane of a warp reads the same weights: one broadcast through the
// read-only path.
__device__ __forceinline__ float4 w4(const float* __restrict__ W, int idx) {
  return __ldg(reinterpret_cast<const float4*>(W + idx));
}
__device__ __forceinline__ float4 w4(const __nv_bfloat16* __restrict__ W, int idx) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(W + idx));
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

// Dot product of weight row o (IN weights) with x (registers).
template <int IN, class WT>
__device__ __forceinline__ float dot_row(const WT* __restrict__ W, int o, const float* x) {
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < IN / 4; ++i) {
    const float4 w = w4(W, o * IN + 4 * i);
    acc = fmaf(w.x, x[4 * i], acc);
    acc = fmaf(w.y, x[4 * i + 1], acc);
    acc = fmaf(w.z, x[4 * i + 2], acc);
    acc = fmaf(w.w, x[4 * i + 3], acc);
  }
  return acc;
}

// Hidden layer: col[o * pitch] = ReLU(W[o] . x + b[o]) for o < OUT. x is in
// registers; the output goes to this thread's shared-memory column.
// Four outputs at a time (four independent accumulation chains; each
// output sums its products in the same order as dot_row).
template <int IN, int OUT, class WT>
__device__ __forceinline__ void dense_col(const WT* __restrict__ W, const float* __restrict__ b,
                                          const float* x, float* col, int pitch) {
  static_assert(IN % 4 == 0 && OUT % 4 == 0, "IN and OUT must be multiples of 4");
#pragma unroll 1
  for (int o = 0; o < OUT; o += 4) {
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < IN / 4; ++i) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 w = w4(W, (o + u) * IN + 4 * i);
        acc[u] = fmaf(w.x, x[4 * i], acc[u]);
        acc[u] = fmaf(w.y, x[4 * i + 1], acc[u]);
        acc[u] = fmaf(w.z, x[4 * i + 2], acc[u]);
        acc[u] = fmaf(w.w, x[4 * i + 3], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) col[(o + u) * pitch] = fmaxf(acc[u] + __ldg(b + o + u), 0.0f);
  }
}

// Output layer (small OUT, registers): y = W x + b.
template <int IN, int OUT, class WT>
__device__ __forceinline__ void dense_out(const WT* __restrict__ W, const float* __restrict__ b,
                                          const float* x, float* y) {
#pragma unroll
  for (int o = 0; o < OUT; ++o) y[o] = dot_row<IN>(W, o, x) + __ldg(b + o);
}

template <int N>
__device__ __forceinline__ void load_col(const float* col, int pitch, float* x) {
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = col[i * pitch];
}

// dx = W^T dz with dz in this thread's shared-memory column (rows < OUT).
template <int IN, int OUT, class WT>
__device__ __forceinline__ void dense_dx_col(const WT* __restrict__ W, const float* dzcol, int pitch,
                                             float* dx) {
#pragma unroll
  for (int i = 0; i < IN; ++i) dx[i] = 0.0f;
#pragma unroll 2
  for (int o = 0; o < OUT; ++o) {
    const float d = dzcol[o * pitch];
#pragma unroll
    for (int i = 0; i < IN / 4; ++i) {
      const float4 w = w4(W, o * IN + 4 * i);
      dx[4 * i] = fmaf(w.x, d, dx[4 * i]);
      dx[4 * i + 1] = fmaf(w.y, d, dx[4 * i + 1]);
      dx[4 * i + 2] = fmaf(w.z, d, dx[4 * i + 2]);
      dx[4 * i + 3] = fmaf(w.w, d, dx[4 * i + 3]);
    }
  }
}

template <class WT>
__device__ __forceinline__ const WT* wptr(const MlpDev& m, int l) {
  return static_cast<const WT*>(m.W[l]);
}

// Whole decoder: IN -> WID (ReLU) [-> WID (ReLU)] -> OUT. `col` is this
// thread's shared-memory column (WID rows, stride `pitch`) for the hidden
// activations.
template <int IN, int WID, int NH, int OUT, class WT>
__device__ __forceinline__ void mlp_fwd(const MlpDev& m, const float* x, float* col, int pitch,
                                        float* out) {
  dense_col<IN, WID>(wptr<WT>(m, 0), m.b[0], x, col, pitch);
  float h[WID];
  load_col<WID>(col, pitch, h);
  if constexpr (NH == 2) {
    dense_col<WID, WID>(wptr<WT>(m, 1), m.b[1], h, col, pitch);
    load_col<WID>(col, pitch, h);
  }
  dense_out<WID, OUT>(wptr<WT>(m, NH), m.b[NH], h, out);
}

// ---------------------------------------------------------------- CTA-level weight gradient

constexpr int kBwdThreads = 64;   // threads (= points) per CTA in the backward kernels
constexpr int kActPitch = 65;     // smem row pitch of [feature][thread] activation tiles

// dW[o][i] += sum_t dz[o][t] x[i][t] over the CTA's 64 points (tiles in smem,
// [row][kActPitch]); the CTA-private float32 slab is updated without atomics.
template <int OUT, int IN>
__device__ __forceinline__ void cta_dw(const float* __restrict__ dz_s, const float* __restrict__ x_s,
                                       float* __restrict__ slab_W, float* __restrict__ slab_b) {
  constexpr int BO = OUT >= 8 ? 8 : OUT;
  constexpr int NOB = OUT / BO;
  constexpr int NIB = (kBwdThreads / NOB) < IN ? (kBwdThreads / NOB) : IN;
  constexpr int BI = IN / NIB;
  static_assert(OUT % BO == 0 && IN % NIB == 0, "unsupported layer shape");
  const int t = threadIdx.x;
  if (t < NOB * NIB) {
    const int ob = t / NIB, ib = t % NIB;
    float acc[BO][BI];
#pragma unroll
    for (int a = 0; a < BO; ++a)
#pragma unroll
      for (int c = 0; c < BI; ++c) acc[a][c] = 0.0f;
#pragma unroll 4
    for (int k = 0; k < kBwdThreads; ++k) {
      float d[BO], xv[BI];
#pragma unroll
      for (int a = 0; a < BO; ++a) d[a] = dz_s[(ob * BO + a) * kActPitch + k];
#pragma unroll
      for (int c = 0; c < BI; ++c) xv[c] = x_s[(ib * BI + c) * kActPitch + k];
#pragma unroll
      for (int a = 0; a < BO; ++a)
#pragma unroll
        for (int c = 0; c < BI; ++c) acc[a][c] = fmaf(d[a], xv[c], acc[a][c]);
    }
#pragma unroll
    for (int a = 0; a < BO; ++a)
#pragma unroll
      for (int c = 0; c < BI; ++c) slab_W[(ob * BO + a) * IN + ib * BI + c] += acc[a][c];
  }
  if (t < OUT) {
    float s = 0.0f;
    for (int k = 0; k < kBwdThreads; ++k) s += dz_s[t * kActPitch + k];
    slab_b[t] += s;
  }
}

// Layout of one CTA's weight-gradient slab: both decoders, W then b per layer.
struct SlabLayout {
  int off_W[2][3], off_b[2][3], n_W[2][3], n_b[2][3];
  int total;
};

// Gradient buffers the slab sums are added to (NULL entries are skipped).
struct SlabTargets {
  float* W[2][3];
  float* b[2][3];
};

inline SlabLayout make_slab_layout(const MlpDev* m0, const MlpDev* m1) {
  SlabLayout s{};
  int off = 0;
  const MlpDev* ms[2] = {m0, m1};
  for (int d = 0; d < 2; ++d)
    for (int l = 0; l < 3; ++l) {
      s.n_W[d][l] = s.n_b[d][l] = 0;
      s.off_W[d][l] = s.off_b[d][l] = off;
      if (!ms[d] || l > ms[d]->n_hidden) continue;
      const int ni = l == 0 ? ms[d]->n_in : ms[d]->width;
      const int no = l == ms[d]->n_hidden ? ms[d]->n_out : ms[d]->width;
      s.off_W[d][l] = off;
      s.n_W[d][l] = no * ni;
      off += no * ni;
      s.off_b[d][l] = off;
      s.n_b[d][l] = no;
      off += no;
      off = (off + 3) & ~3;
    }
  s.total = off;
  return s;
}

}  // namespace hyrf
